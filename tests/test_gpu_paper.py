"""GPU runs in the paper's own setting: erf-switched sine signals (Sec. 7, Eq. exampleDensities),
separate grid targets, and the interpolation-order study of the local part (Sec. 7, first example).
"""
import math

import numpy as np
import pytest

import oracle
from _metric import BAR, rel_errors
from paper_2604_07170_gb300 import inputs

pytestmark = pytest.mark.gpu


def _erf_workload(M=80, box=3.0, n_steps=300, dt=0.02, omega_max=30.0, seed=31, eps=1e-9):
    rng = np.random.Generator(np.random.PCG64(inputs.SEED0 + 7919 * seed))
    src = rng.uniform(0.0, box, (M, 2))
    # switch-on times late enough that the signals are below 1e-16 at t <= 0
    par = inputs.erf_params(M, rng, omega_max, 1.2, 0.5 * n_steps * dt)
    g = np.linspace(0.1 * box, 0.9 * box, 8)
    tgt = np.array([[x, y] for x in g for y in g])
    K0 = inputs.band_limit(par, "erf", eps)
    return src, tgt, par, dt, n_steps, K0


def _oracle(src, par, tgt, steps, dt, box):
    ev = np.array([[x, y, n * dt] for n in steps for (x, y) in tgt])
    return oracle.field(src, par, ev, family="erf", r_coinc=1e-12 * box).reshape(len(steps), -1)


def test_erf_signals_through_the_server():
    from paper_2604_07170_gb300 import wfp
    src, tgt, par, dt, nt, K0 = _erf_workload()
    steps = [150, 300]
    with wfp.Server(8 << 30, 4) as sv:
        rid = sv.submit(src, par[:, :2], dt, nt, K0, 1e-6, tgt_xy=tgt, out_steps=steps, family=wfp.SIGNAL_ERF)
        sv.run()
        got = sv.result(rid)
    ref = _oracle(src, par, tgt, steps, dt, 3.0)
    e = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    print("\nerf server rel L2:", e)
    assert e.max() <= 1e-6


def _x1_error(src, tgt, par, K0, ref, p, N, T=8.0, eps=1e-8):
    from paper_2604_07170_gb300 import wfp
    dt = T / N
    plan = wfp.Plan(src, tgt, dt, N, K0, 1e-5, eps=eps, W=24, p=p, local_interp=wfp.INTERP_LAGRANGE)
    sig = inputs.sample_sigma(par, dt * np.arange(1, N + 1), "erf")
    for k in range(N):
        u = plan.step(sig[k])
    plan.close()
    return float(np.max(np.abs(u - ref)) / np.max(np.abs(ref)))


def test_convergence_study_of_the_first_example():
    # Sec. 7, "Convergence rate": M = 100 sources at random in B = [-1,1]^2, erf-switched sines with
    # t0 in [1.5, 7] and w in [0, 10 pi], eps = 1e-8, W = 24, p-point Lagrange interpolation in the local
    # part; relative max-norm error on a regular 10 x 10 target grid at T = 8 against dt.  The paper finds
    # rates matching the order p and a plateau about a digit above eps.  Eq. dt with W = 24 caps dt at
    # ~0.0216, so the p >= 6 curves reach the plateau within one or two refinements: their order is
    # checked as a lower bound and by their ordering at the coarsest dt.
    rng = np.random.Generator(np.random.PCG64(inputs.SEED0 + 51))
    M = 100
    src = rng.uniform(-1.0, 1.0, (M, 2))
    par = inputs.erf_params(M, rng, 10 * math.pi, 1.5, 7.0, cube_root=False)
    g = np.linspace(-1.0, 1.0, 10)
    tgt = np.array([[x, y] for x in g for y in g])
    K0 = inputs.band_limit(par, "erf", 1e-8)
    ref = oracle.field(src, par, np.column_stack([tgt, np.full(len(tgt), 8.0)]), family="erf", r_coinc=1e-12)
    Ns = [400, 560, 800]
    dts = 8.0 / np.array(Ns)
    slope = {}
    errs = {}
    for p in (2, 4):
        errs[p] = [_x1_error(src, tgt, par, K0, ref, p, N) for N in Ns]
        slope[p] = float(np.polyfit(np.log(dts), np.log(errs[p]), 1)[0])
    errs[6] = [_x1_error(src, tgt, par, K0, ref, 6, N) for N in Ns[:2]]
    slope[6] = math.log(errs[6][0] / errs[6][1]) / math.log(Ns[1] / Ns[0])
    errs[8] = [_x1_error(src, tgt, par, K0, ref, 8, N) for N in (400, 1600)]
    errs[10] = [_x1_error(src, tgt, par, K0, ref, 10, N) for N in (800, 1600)]
    print("\nX1 errors:", {p: [f"{e:.2e}" for e in v] for p, v in errs.items()},
          "slopes:", {p: round(v, 2) for p, v in slope.items()})
    assert abs(slope[2] - 2) <= 0.5 and abs(slope[4] - 4) <= 0.5
    assert slope[6] >= 4.5
    assert errs[2][0] > errs[4][0] > errs[6][0] > errs[8][0]
    plateau = [errs[8][1], errs[10][0], errs[10][1]]
    assert max(plateau) <= 5e-7 and min(plateau) >= 1e-8  # within about a digit and a half of eps


_GRID_REF = {}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind", ["random", "circle", "wiggly"])
def test_paper_grid_target_workloads(kind, precision):
    # the large examples of Sec. 7 (random space-filling sources, sources on a circle, sources on the
    # complicated closed curve) at 10^4 sources with a 100 x 100 target grid, omega_max = 30 pi (about 31
    # wavelengths across B, ~200 sources within delta of a target), T = 8, lag and far history active;
    # 64 grid targets against the oracle at t = 4 and t = 8
    from paper_2604_07170_gb300 import wfp
    wl, tgt = inputs.paper_grid_workload(kind, 10000, 100, 30 * math.pi)
    steps = [wl.n_steps // 2, wl.n_steps]
    idx = np.random.default_rng(61).choice(tgt.shape[0], 64, replace=False)
    if kind not in _GRID_REF:
        ev = np.array([[tgt[i, 0], tgt[i, 1], n * wl.dt] for n in steps for i in idx])
        _GRID_REF[kind] = oracle.field(wl.src_xy, wl.params, ev, family="erf",
                                       r_coinc=1e-12 * 2.0).reshape(len(steps), -1)
    ref = _GRID_REF[kind]
    plan = wfp.Plan(wl.src_xy, tgt, wl.dt, wl.n_steps, wl.band_limit, wl.tol, precision=precision)
    info = plan.info()
    got = []
    for n0 in range(0, wl.n_steps, 256):
        sig = inputs.sample_sigma(wl.params, wl.dt * np.arange(n0 + 1, min(wl.n_steps, n0 + 256) + 1), "erf")
        for k in range(sig.shape[0]):
            u = plan.step(sig[k])
            if n0 + k + 1 in steps:
                got.append(u[idx])
    plan.close()
    assert info["lag_active"] and info["far_active"] and info["n_self"] == 0
    e = rel_errors(np.array(got), ref, precision)
    print(f"\n{kind} precision={precision}: rel L2 at t = 4, 8: {e}, pairs {info['n_pairs']}")
    assert e.max() <= BAR


@pytest.mark.parametrize("precision", [0, 1])
def test_fixed_delta_variant_with_a_64_level_window(precision):
    # fixed blending width delta = 1.2 at dt = 0.025 (40 steps per period): W = 48 and nmax = 59, so
    # the local part runs on the 64-level window; the default plan (W from Eq. dt) is checked too
    from paper_2604_07170_gb300 import wfp
    wl = inputs.small(100, 3.0, 400, seed=41, dt=0.025)
    steps = [120, 250, 400]
    ev = np.array([[x, y, n * wl.dt] for n in steps for (x, y) in wl.src_xy])
    ref = oracle.field(wl.src_xy, wl.params, ev, r_coinc=1e-12 * wl.meta["box"]).reshape(len(steps), -1)
    sig = wl.sigma(1, wl.n_steps + 1)
    for kw in ({"delta": 1.2}, {}):
        plan = wfp.Plan(wl.src_xy, None, wl.dt, wl.n_steps, wl.band_limit, wl.tol, precision=precision, **kw)
        info = plan.info()
        got = []
        for n in range(1, wl.n_steps + 1):
            u = plan.step(sig[n - 1])
            if n in steps:
                got.append(u)
        plan.close()
        e = rel_errors(np.array(got), ref, precision)
        print(f"\n{kw} W={info['W']} nmax={info['nmax']} local_variant={info['local_variant']} rel L2:", e)
        if kw:
            assert info["W"] == 48 and info["nmax"] > 32 and info["local_variant"] == 0
        assert info["lag_active"] and info["far_active"]
        assert e.max() <= BAR
