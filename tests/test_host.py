"""CPU tests of the CUDA path's host logic and plan-time quadrature (no GPU needed).

Each test pins a routine that runs at plan time (on the device, through the same
__host__ __device__ code) against something independent of it: the CPU oracle's
component integrals, closed forms, scipy quadrature, or numbers printed in the paper.
"""
import ctypes
import json
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2604_07170_gb300 import inputs, wfp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_numbers.json")))


def test_library_exports_every_declared_symbol():
    names = set()
    for h in ("wfp.h", "wfp_debug.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        names |= set(re.findall(r"\b(wfp_[a-z_0-9]+)\s*\(", src))
    assert len(names) >= 15
    lib = ctypes.CDLL(wfp._build.build())
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(wfp.EXPORTS)


def test_invalid_arguments_are_rejected_on_the_host():
    K0 = 12.7
    bad = [dict(dt=0.3), dict(dt=-1.0), dict(tol=0.0), dict(tol=2.0), dict(band_limit=float("nan"))]
    for b in bad:
        args = dict(halfside=10.0, dt=0.1, Nt=100, band_limit=K0, tol=1e-6)
        args.update(b)
        with pytest.raises(wfp.WFPError) as ei:
            wfp.select_params(args["halfside"], args["dt"], args["Nt"], args["band_limit"], args["tol"])
        assert ei.value.code == wfp.WFP_EINVAL
    with pytest.raises(wfp.WFPError):
        wfp.select_params(10.0, 0.1, 100, K0, 1e-6, precision=7)
    for lf in (-1, 3):
        with pytest.raises(wfp.WFPError) as ei:
            wfp.select_params(10.0, 0.1, 100, K0, 1e-6, local_form=lf)
        assert ei.value.code == wfp.WFP_EINVAL


def test_parameters_reproduce_the_papers_printed_example():
    g = GOLD["X2_sec7_2"]
    # the paper's example in normalised units (B = [-1,1]^2): eps = 1e-7, W = 16, dt = 0.00112, K0 = 983
    i = wfp.select_params(1.0, g["dt"], g["N_t"], g["K0"], 100 * g["eps"], eps=g["eps"], W=g["W"], p=g["p"])
    assert i["W"] == 16 and i["p"] == 20
    assert abs(i["delta"] - g["delta"]) < 5e-5                      # delta = W dt
    assert abs(i["A"] - (2 * math.sqrt(2) + 1)) < 1e-15             # Eq. A with Delta = 1
    assert round(i["dk"], 3) == g["dk"]                              # Eq. dk, printed 0.918
    assert abs(i["K"] - g["K"]) / g["K"] < 0.01                      # Eq. K gives 2782; printed 2808
    # reading: A+ = A + a + delta (here rounded up so that A+ - delta is on the step grid);
    # without the rounding, the printed K gives the printed N exactly
    Aplus = i["A"] + 1.0 + g["W"] * g["dt"]
    dk = 2 * math.pi / (Aplus + 2)
    assert 2 * math.ceil(g["K"] / dk) + 1 == g["N"]
    assert i["Aplus"] - Aplus >= 0 and i["Aplus"] - Aplus < g["dt"]
    # N_lambda = n N_g = 20 x 32 for the paper's fixed choice
    lam, q = wfp.debug_soe(36.0, 20, 32)
    assert lam.size == g["N_lambda"]


def test_far_cutoff_table_is_reproduced():
    # Table tab:Kf_estimates; the blend shape b for phi_Delta is not printed: b = ln(1e12) matches
    rows = GOLD["Kf_table"]["rows"]
    for Delta, Kf, ref in rows:
        if Kf > 80:
            continue  # beyond the Kf range the plan's radial rule is built for
        A = 2 * math.sqrt(2) + Delta
        H = wfp.debug_hankel(Kf, A, Delta, 1e-12)
        got = np.abs(H).max()
        assert ref / 5 <= got <= ref * 5, (Delta, Kf, got, ref)


def test_dyadic_sum_of_exponentials_accuracy():
    # Eq. LaplaceApprox with lam_max = 36, n = 20 panels, N_g = 32: near double precision for
    # r in [0, A], t in [A+ - delta, 3e4]; at r = 0 the sum reduces to 1/t
    special = pytest.importorskip("scipy.special")
    lam, q = wfp.debug_soe(36.0, 20, 32)
    A = 2 * math.sqrt(2) + 1
    worst = 0.0
    for r in np.linspace(0, A, 9):
        t = np.geomspace(A + 1.0, 3e4, 300)
        s = (q[None, :] * special.i0e(r * lam)[None, :] * np.exp(-lam[None, :] * (t[:, None] - r))).sum(1)
        worst = max(worst, np.max(np.abs(s * np.sqrt(t * t - r * r) - 1)))
    assert worst < 1e-12


@pytest.mark.parametrize("dlo,T,eps", [(0.1, 300.0, 1e-9), (0.1, 10.0, 1e-9), (1e-3, 8.0, 1e-12),
                                       (0.1, 10000.0, 1e-6)])
def test_self_term_sum_of_exponentials(dlo, T, eps):
    # the self term's sum for 1/d must hold at every grid delay d = m dt in [dlo, T]; checked here at
    # those delays and on a dense geometric sample, in extended precision, with its term count:
    # well under the ~93 terms a trapezoid rule in ln(lambda) from 1e-2 eps / T needs at 1e-9
    lam, q = wfp.debug_self_soe(dlo, T, eps)
    assert np.all(lam > 0) and np.all(q > 0)
    d = np.concatenate([dlo * np.arange(1, int(T / dlo) + 1), np.geomspace(dlo, T, 20000)])
    s = (q[None, :].astype(np.longdouble) * np.exp(-np.outer(d, lam).astype(np.longdouble))).sum(1)
    assert np.max(np.abs(s * d - 1)) <= eps
    if (dlo, T, eps) == (0.1, 300.0, 1e-9):
        assert lam.size <= 50


def test_hankel_and_soe_reproduce_the_truncated_kernel_transform():
    # sum_l H_l e^{A lam_l} e^{-lam_l t} = int_0^A r J0(kappa r) phi_Delta(A - r) / sqrt(t^2 - r^2) dr
    # (Eqs. spectralTK, H, LaplaceApprox), checked against scipy quadrature with the oracle's phi
    integrate = pytest.importorskip("scipy.integrate")
    special = pytest.importorskip("scipy.special")
    Delta, eps = 1.0, 1e-12
    A = 2 * math.sqrt(2) + Delta
    lam, q = wfp.debug_soe(36.0, 12, 32)
    b = math.log(1 / eps)
    for kappa in (0.0, 3.0, 20.0):
        H = wfp.debug_hankel(kappa, A, Delta, eps, 36.0, 12, 32)
        for t in (A + 1.0, 7.0, 15.0):
            got = np.sum(H * np.exp(lam * (A - t)))
            f = lambda r: r * special.j0(kappa * r) * oracle.phi(A - r, Delta, b) / math.sqrt(t * t - r * r)
            ref, _ = integrate.quad(f, 0, A, limit=400, epsabs=1e-15, epsrel=1e-13)
            assert abs(got - ref) <= 1e-11 * max(1.0, abs(ref)), (kappa, t, got, ref)


def test_blending_function_matches_the_oracle():
    for eps in (1e-8, 1e-12):
        b = math.log(1 / eps)
        delta = 0.37
        for t in np.linspace(0, delta, 23):
            phi, dphi, _ = wfp.debug_phi(t, delta, eps)
            assert abs(phi - oracle.phi(t, delta, b)) < 1e-14
            assert abs(dphi - oracle.dphi(t, delta, b)) < 1e-12 * max(1.0, abs(dphi))


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_local_weights_integrate_polynomial_signals_exactly(deg):
    # with p-th order Lagrange interpolation on every interval the local weights are exact for
    # sigma(t) = t^deg (deg < p): eta . sigma(levels) equals the oracle's local component
    dt, W, p, eps = 0.1, 20, 16, 1e-10
    nmax = W + 1 + p // 2
    delta, b = W * dt, math.log(1 / eps)
    par = np.zeros((1, 8))
    par[0, deg] = 1.0
    src = np.array([[0.0, 0.0]])
    n = 60
    lev = np.arange(n - nmax + 1, n + 1) * dt
    sig = lev ** deg
    for r in (1e-6, 0.004, 0.07, 0.33, 1.2, 1.97):
        eta = wfp.debug_eta(r, dt, W, p, eps, -1.0, 20)
        ref = oracle.field(src, par, np.array([[r, 0.0, n * dt]]), family="poly", kind="local", delta=delta,
                           Aplus=100.0, b=b)[0]
        assert abs(eta @ sig - ref) <= 1e-11 * max(1.0, abs(ref)), (r, eta @ sig, ref)


def test_local_weights_on_band_limited_signals():
    # hybrid interpolation (band-limited least squares on the newest four intervals, Lagrange
    # elsewhere) against the oracle's local component for Gaussian-sinusoid signals
    dt, W, p, eps = 0.1, 23, 16, 1e-9
    nmax = W + 1 + p // 2
    delta, b = W * dt, math.log(1 / eps)
    K0 = 2 * math.pi + math.sqrt(2 * math.log(1e9))
    rng = np.random.default_rng(3)
    par = inputs.gauss3_params(1, 20.0, rng)
    src = np.array([[0.0, 0.0]])
    for r in (1e-5, 0.03, 0.08, 0.25, 0.6, 1.5):
        eta = wfp.debug_eta(r, dt, W, p, eps, K0, 20)
        for n in (110, 150):
            sig = inputs.sample_sigma(par, np.arange(n - nmax + 1, n + 1) * dt, "gauss3")[:, 0]
            ref = oracle.field(src, par, np.array([[r, 0.0, n * dt]]), kind="local", delta=delta, Aplus=100.0,
                               b=b)[0]
            tol = 5e-7 if r < 4 * dt else 1e-9
            assert abs(eta @ sig - ref) <= tol, (r, n, eta @ sig, ref)


def test_mode_recurrence_matches_direct_quadrature_and_forgets_removed_signal():
    # Lemma (Eqs. alphakEvolution, ghEquations, alphakF) with the FIR taps of Eq. hggrid against
    # direct quadrature of Eq. alphak: alpha(t) = int sin(k(t-tau))/k phi(t-tau) phi(tau-t+A+) S(tau) dtau
    integrate = pytest.importorskip("scipy.integrate")
    dt, W, eps, L = 0.01, 20, 1e-12, 150  # errors scale with eps (~1e-8 relative at eps = 1e-10)
    b, delta = math.log(1 / eps), W * dt
    Aplus = delta + L * dt
    S = lambda t: math.exp(-((t - 2.0) ** 2) / (2 * 0.2 ** 2)) * math.cos(20 * t) if t > 0 else 0.0
    for kappa in (0.0, 7.5, 30.0):
        taps, rot = wfp.debug_taps(kappa, dt, W, eps, Aplus - delta)
        p, q, pa, qa = taps[:W], taps[W:2 * W], taps[2 * W:3 * W], taps[3 * W:]
        c, sk, ks = rot
        a = ad = 0.0
        hist = {}
        checks = {250: None, 300: None, 400: None, 520: None}
        for n in range(0, 521):
            if n in checks:
                checks[n] = a
            # advance from t_n to t_{n+1} with S at levels n..n-W+1 and n-L..n-L-W+1
            h = sum(p[m] * S((n - m) * dt) - pa[m] * S((n - m - L) * dt) for m in range(W))
            g = sum(q[m] * S((n - m) * dt) - qa[m] * S((n - m - L) * dt) for m in range(W))
            a, ad = c * a + sk * ad + h, -ks * a + c * ad + g
        scale = 0.0
        for n, got in checks.items():
            t = n * dt
            kern = lambda tau: ((math.sin(kappa * (t - tau)) / kappa) if kappa > 0 else (t - tau)) \
                * oracle.phi(t - tau, delta, b) * oracle.phi(tau - t + Aplus, delta, b) * S(tau)
            ref, _ = integrate.quad(kern, max(0.0, t - Aplus), t, limit=800, epsabs=1e-15, epsrel=1e-12,
                                    points=[1.4, 2.0, 2.6])
            scale = max(scale, abs(ref))
            checks[n] = (got, ref)
        for n, (got, ref) in checks.items():
            assert abs(got - ref) <= 1e-9 * scale, (kappa, n, got, ref)
        # at t = 5.2 the pulse (t in [1, 3]) has left the near window [t - A+, t] entirely: the exact
        # value is 0 and the recurrence keeps only eps-level residue of the injected-then-removed pulse
        assert abs(checks[520][1]) < 1e-12 * scale
        assert abs(checks[520][0]) < 1e-9 * scale


def test_server_rejects_bad_requests_on_the_host():
    # submission is host-only: validation happens before any device work
    sv = wfp.Server(1 << 30, 4)
    xy = np.zeros((3, 2))
    xy[:, 0] = [0.0, 1.0, 2.0]
    par = np.zeros((3, 8))
    with pytest.raises(wfp.WFPError) as ei:
        sv.submit(xy, par, 0.1, 10, 5.0, 1e-6, out_steps=[0])          # step outside 1..Nt
    assert ei.value.code == wfp.WFP_EINVAL
    with pytest.raises(wfp.WFPError) as ei:
        sv.submit(xy, par, 0.1, 10, 5.0, 1e-6, out_steps=[11])
    assert ei.value.code == wfp.WFP_EINVAL
    with pytest.raises(wfp.WFPError) as ei:
        sv.submit(xy, par, 0.1, 0, 5.0, 1e-6)                          # Nt < 1
    assert ei.value.code == wfp.WFP_EINVAL
    rid = sv.submit(xy, par, 0.1, 10, 5.0, 1e-6, out_steps=[10, 3])
    st = sv.query(rid)
    assert st["state"] == wfp.REQ_PENDING and st["n_out"] == 2 and st["Mt"] == 3
    with pytest.raises(wfp.WFPError) as ei:
        sv.result(rid)
    assert ei.value.code == wfp.WFP_ESTATE
    q = wfp.wfp_request(M=3, src_xy=wfp._dptr(np.ascontiguousarray(xy)), Mt=3, dt=0.1, Nt=10, band_limit=5.0,
                        tol=1e-6, signal_family=7, signal_params=wfp._dptr(par))
    rid2 = ctypes.c_int64()
    assert wfp.lib().wfp_server_submit(sv._h, ctypes.byref(q), ctypes.byref(rid2)) == wfp.WFP_EUNSUPPORTED
    sv.close()


def test_fixed_delta_sets_W_and_bounds_are_checked():
    i = wfp.select_params(10.0, 0.025, 400, 12.7, 1e-6, delta=1.2)
    assert i["W"] == 48 and i["nmax"] > 32 and i["nmax"] <= 64
    assert abs(i["delta"] / i["scale"] - 48 * 0.025) < 1e-12
    with pytest.raises(wfp.WFPError) as ei:
        wfp.select_params(10.0, 0.025, 400, 12.7, 1e-6, delta=2.0)  # W = 80 > 59
    assert ei.value.code == wfp.WFP_EINVAL
    with pytest.raises(wfp.WFPError):
        wfp.select_params(10.0, 0.1, 400, 12.7, 1e-6, delta=0.3)  # W = 3 violates Eq. dt
    with pytest.raises(wfp.WFPError):
        wfp.select_params(10.0, 0.1, 400, 12.7, 1e-6, local_interp=5)


def test_local_weight_table_matches_the_quadrature():
    # plans evaluate the local weights from a Chebyshev series per delay interval (in sqrt of the
    # distance to the interval's end); it must reproduce the direct quadrature to rounding
    rng = np.random.default_rng(3)
    for dt, W, p, eps, K0 in ((0.0077, 23, 16, 1e-9, 165.4), (0.02, 24, 12, 1e-8, -1.0)):
        worst = 0.0
        for r in np.concatenate([rng.uniform(dt, W * dt, 6), [dt * (1 + 1e-12), 2 * dt, (W - 1) * dt, W * dt * (1 - 1e-9)]]):
            a = wfp.debug_eta(r, dt, W, p, eps, K0)
            b = wfp.debug_eta_table(r, dt, W, p, eps, K0)
            worst = max(worst, float(np.max(np.abs(a - b))))
        assert worst <= 1e-13, (dt, W, worst)


def test_near_weights_are_smooth_on_dyadic_subintervals():
    # below dt the weights carry a logarithm of r; on the sub-intervals [dt/2, dt] (variable
    # sqrt(dt - r), as for the other delay intervals) and [dt/4, dt/2], [dt/8, dt/4] (variable r) they
    # are analytic, so a 16-term Chebyshev series reproduces them with coefficients no larger than the
    # weights themselves (what an FP32 factored form of the near pairs needs)
    from numpy.polynomial import chebyshev as C
    dt, W, p, eps = 0.1, 23, 16, 1e-9
    K0 = 2 * np.pi + np.sqrt(2 * np.log(1 / eps))
    n = 24
    z = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    zt = np.linspace(-1.0, 1.0, 7)
    for a, b, bound in ((0.5, 1.0, 1e-7), (0.25, 0.5, 1e-12), (0.125, 0.25, 1e-12)):
        def r_of(zz):
            if a == 0.5:
                v = 0.5 * (zz + 1) * np.sqrt((b - a) * dt)
                return b * dt - v * v
            return (a + (b - a) * 0.5 * (zz + 1)) * dt
        E = np.array([wfp.debug_eta(r, dt, W, p, eps, K0) for r in r_of(z)])
        coef = np.array([C.chebfit(z, E[:, l], 15) for l in range(E.shape[1])])
        Et = np.array([wfp.debug_eta(r, dt, W, p, eps, K0) for r in r_of(zt)])
        fit = np.array([C.chebval(zt, coef[l]) for l in range(E.shape[1])]).T
        scale = np.abs(E).max()
        assert np.abs(fit - Et).max() <= bound * scale, (a, b)
        assert np.abs(coef).sum(axis=1).max() <= 1.05 * scale, (a, b)


def test_factored_local_series_cut_against_the_quadrature():
    # the factored local part (mixed path) keeps the first NC Chebyshev coefficients of each delay
    # interval's weight series; the dropped tail must bound the error against the direct quadrature
    # of the weights, and the regrouping sum_l eta_l sigma_l = sum_c T_c(x) (sum_l C_lc sigma_l) must
    # hold for the library's own table
    from numpy.polynomial import chebyshev as C
    dt, W, p, eps = 0.1, 23, 16, 1e-9
    K0 = 2 * np.pi + np.sqrt(2 * np.log(1 / eps))
    nc, tail, tab = wfp.debug_factored_table(dt, W, p, eps, K0, 20, precision=wfp.MIXED)
    assert nc == 16 and 0 < tail <= 2.0 ** -25
    nc64, tail64, _ = wfp.debug_factored_table(dt, W, p, eps, K0, 20, precision=wfp.FP64)
    assert nc64 == 36 and tail64 == 0.0
    rng = np.random.default_rng(5)
    sig = rng.standard_normal(tab.shape[1])
    # the table's own accuracy is ~1e-15 of the largest weights (intervals far out carry tiny ones)
    floor = 1e-13 * np.abs(tab).sum(axis=2).max()
    for k in range(1, W):
        scale = np.abs(tab[k - 1]).sum(axis=1).max()
        for r in rng.uniform(k * dt, (k + 1) * dt, 3):
            x = 2 * np.sqrt(((k + 1) * dt - r) / dt) - 1
            quad = wfp.debug_eta(r, dt, W, p, eps, K0)
            full = np.array([C.chebval(x, tab[k - 1, l]) for l in range(tab.shape[1])])
            cut = np.array([C.chebval(x, tab[k - 1, l, :nc]) for l in range(tab.shape[1])])
            assert np.abs(full - quad).max() <= floor
            assert np.abs(cut - quad).max() <= tail * scale + floor
            y = tab[k - 1, :, :nc].T @ sig  # per-coefficient contraction of the window
            assert abs(C.chebval(x, y) - cut @ sig) <= 1e-14 * scale * np.abs(sig).sum()
