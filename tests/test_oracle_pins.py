"""Pins for the CPU oracle, against facts fixed by the paper and by mathematics.

The oracle evaluates the exact retarded field of Sec. 1 (Eqs. solnRep, Green) by the
square-root substitution of Sec. 7 (Eq. exactSol).  These tests check it against:
closed forms for non-band-limited signals, an independent quadrature (cosh
substitution, and scipy's adaptive quad on tiny inputs), node doubling,
linearity, reciprocity, rigid-motion / time-shift / space-time-scale invariance,
the blending-function normalisation and Fourier transform of Sec. 2.1
(Eq. KBblending and the formula after it), the partition of unity of Sec. 3
(Eq. split) and the r -> 0 limit that defines the coincident-pair self term.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2604_07170_gb300 import inputs

TWO_PI = 2 * math.pi


def one_source(sig, fam="poly"):
    p = np.zeros(8)
    p[: len(sig)] = sig
    return np.array([[0.0, 0.0]]), p[None, :]


@pytest.mark.parametrize("r,t", [(0.3, 1.7), (1e-7, 0.5), (2.0, 2.5), (0.05, 10.0), (1.0, 30.0)])
def test_closed_forms_polynomial_signals(r, t):
    # sigma = 1:   u = acosh(t/r) / (2 pi)
    # sigma = t:   u = [t acosh(t/r) - sqrt(t^2 - r^2)] / (2 pi)
    # sigma = t^2: u = [(t^2 + r^2/2) acosh(t/r) - 1.5 t sqrt(t^2 - r^2)] / (2 pi)
    ev = np.array([[r, 0.0, t]])
    ac, sq = math.acosh(t / r), math.sqrt(t * t - r * r)
    exact = [ac / TWO_PI, (t * ac - sq) / TWO_PI, ((t * t + 0.5 * r * r) * ac - 1.5 * t * sq) / TWO_PI]
    for k, ex in enumerate(exact):
        coef = [0.0, 0.0, 0.0]
        coef[k] = 1.0
        src, p = one_source(coef)
        for method in (0, 1):
            u = oracle.field(src, p, ev, family="poly", method=method)[0]
            assert abs(u - ex) <= 1e-13 * abs(ex) + 1e-15, (k, method, u, ex)


def test_light_cone_and_coincident_exclusion():
    src, p = one_source([1.0])
    # before the wave arrives (t <= r) the field is exactly zero
    assert oracle.field(src, p, np.array([[1.0, 0.0, 0.999]]), family="poly")[0] == 0.0
    # a coincident pair is excluded (Eq. exactSol sums over r_j != 0)
    assert oracle.field(src, p, np.array([[0.0, 0.0, 3.0]]), family="poly", r_coinc=1e-12)[0] == 0.0


def _random_case(seed, M=6, Ne=8, box=4.0, T=12.0):
    rng = np.random.default_rng(seed)
    src = rng.uniform(0, box, (M, 2))
    par = inputs.gauss3_params(M, T, rng)
    ev = np.column_stack([rng.uniform(0, box, Ne), rng.uniform(0, box, Ne), rng.uniform(4, T, Ne)])
    return src, par, ev


def test_two_independent_quadratures_agree():
    src, par, ev = _random_case(1)
    # include a near-coincident pair (r = 1e-6) to exercise the graded panels
    ev = np.vstack([ev, [src[0, 0] + 1e-6, src[0, 1], 9.0]])
    a = oracle.field(src, par, ev, method=0)
    b = oracle.field(src, par, ev, method=1)
    scale = np.max(np.abs(a))
    assert np.max(np.abs(a - b)) <= 1e-12 * scale


def test_node_doubling():
    src, par, ev = _random_case(2)
    a = oracle.field(src, par, ev)
    try:
        oracle.set_resolution(40, 0.25)
        b = oracle.field(src, par, ev)
    finally:
        oracle.set_resolution(20, 0.5)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


def test_brute_force_scipy_quad():
    integrate = pytest.importorskip("scipy.integrate")
    src, par, ev = _random_case(3, M=2, Ne=2)
    got = oracle.field(src, par, ev)
    for e in range(ev.shape[0]):
        x, y, t = ev[e]
        tot = 0.0
        for j in range(src.shape[0]):
            r = math.hypot(x - src[j, 0], y - src[j, 1])
            if r >= t:
                continue
            f = lambda th: inputs.sample_sigma(par[j:j + 1], np.array([t - r * math.cosh(th)]), "gauss3")[0, 0]
            v, _ = integrate.quad(f, 0.0, math.acosh(t / r), limit=2000, epsabs=1e-14, epsrel=1e-13)
            tot += v / TWO_PI
        assert abs(got[e] - tot) <= 1e-11 * max(1.0, abs(tot)), (got[e], tot)


def test_linearity_in_signal_amplitudes():
    src, par, ev = _random_case(4)
    rng = np.random.default_rng(44)
    pa, pb = par.copy(), par.copy()
    pa[:, 0:3] = rng.uniform(-1, 1, (par.shape[0], 3))
    pb[:, 0:3] = rng.uniform(-1, 1, (par.shape[0], 3))
    ps = par.copy()
    ps[:, 0:3] = 2.0 * pa[:, 0:3] - 3.0 * pb[:, 0:3]
    ua, ub, us = (oracle.field(src, p, ev) for p in (pa, pb, ps))
    assert np.max(np.abs(us - (2 * ua - 3 * ub))) <= 1e-13 * np.max(np.abs(us))


def test_reciprocity():
    rng = np.random.default_rng(5)
    a, b = rng.uniform(0, 3, 2), rng.uniform(0, 3, 2)
    par = inputs.gauss3_params(1, 10.0, rng)
    u_ab = oracle.field(a[None], par, np.array([[b[0], b[1], 11.0]]))[0]
    u_ba = oracle.field(b[None], par, np.array([[a[0], a[1], 11.0]]))[0]
    assert abs(u_ab - u_ba) <= 1e-14 * max(abs(u_ab), 1e-300)


def test_rigid_motion_invariance():
    src, par, ev = _random_case(6)
    base = oracle.field(src, par, ev)
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    shift = np.array([3.3, -1.1])
    src2 = src @ R.T + shift
    ev2 = ev.copy()
    ev2[:, :2] = ev[:, :2] @ R.T + shift
    got = oracle.field(src2, par, ev2)
    assert np.max(np.abs(got - base)) <= 1e-12 * np.max(np.abs(base))


def test_time_shift_equivariance():
    src, par, ev = _random_case(7)
    base = oracle.field(src, par, ev)
    T0 = 2.5
    par2 = par.copy()
    par2[:, 3:6] += T0
    ev2 = ev.copy()
    ev2[:, 2] += T0
    got = oracle.field(src, par2, ev2)
    assert np.max(np.abs(got - base)) <= 1e-12 * np.max(np.abs(base))


def test_space_time_scale_invariance():
    # (x, t) -> (s x, s t) with sigma(t) -> sigma(t / s) leaves the 2D point-source field
    # unchanged: G(s x, s t) = G(x, t) / s and dtau scales by s.
    src, par, ev = _random_case(8)
    base = oracle.field(src, par, ev)
    s = 3.7
    par2 = par.copy()
    par2[:, 3:6] *= s   # pulse centres
    par2[:, 6] *= s     # envelope width
    par2[:, 7] /= s     # carrier
    got = oracle.field(src * s, par2, ev * s)
    assert np.max(np.abs(got - base)) <= 1e-12 * np.max(np.abs(base))


def test_bessel_i0_series():
    special = pytest.importorskip("scipy.special")
    for x in [0.0, 1e-3, 0.5, 3.0, 18.42, 36.0, 50.0]:
        assert abs(oracle.i0(x) - special.i0(x)) <= 1e-14 * special.i0(x)


@pytest.mark.parametrize("b", [math.log(1e8), math.log(1e16)])
def test_blending_function(b):
    delta = 0.37
    # normalisation: int_0^delta phi' = 1 since int_{-1}^{1} I0(b sqrt(1-x^2)) dx = 2 sinh(b)/b
    assert abs(oracle.phi(delta * (1 - 1e-15), delta, b) - 1.0) < 1e-13
    # symmetry of the Kaiser-Bessel bump about delta/2
    assert abs(oracle.phi(0.5 * delta, delta, b) - 0.5) < 1e-14
    for t in [0.1, 0.23]:
        assert abs(oracle.phi(t * delta, delta, b) + oracle.phi((1 - t) * delta, delta, b) - 1.0) < 1e-13
    # Fourier transform of phi' (Sec. 2.1): b e^{-i delta w/2} sinc(sqrt((delta w/2)^2 - b^2)) / sinh b.
    # The printed phase e^{-i delta w / 2} is that of the e^{-i w t} convention (the bump is centred
    # at delta/2); under the e^{+i w t} convention stated beside it the phase is conjugated.  The
    # modulus, which is what the band-limit bound uses, is convention-free.
    x, w = oracle.gl_rule(120)
    tt = 0.5 * delta * (x + 1)
    f = np.array([oracle.dphi(t, delta, b) for t in tt])
    for om in [0.0, 5.0, 40.0, 2 * b / delta, 3 * b / delta]:
        num = np.sum(0.5 * delta * w * f * np.exp(-1j * om * tt))
        z2 = (delta * om / 2) ** 2 - b * b
        if z2 >= 0:
            z = math.sqrt(z2)
            sinc = math.sin(z) / z if z > 0 else 1.0
        else:
            z = math.sqrt(-z2)
            sinc = math.sinh(z) / z
        ex = b * np.exp(-1j * delta * om / 2) / math.sinh(b) * sinc
        assert abs(num - ex) <= 1e-12, (om, num, ex)


def test_split_components_sum_to_full_field():
    # u = u_l + u_nh + u_fh (Sec. 3, Eq. split); needs A+ >= 2 delta
    src, par, ev = _random_case(9, M=4, Ne=6, T=14.0)
    ev[:, 2] = np.linspace(6, 14, ev.shape[0])
    delta, Aplus, b = 0.9, 4.1, math.log(1e8)
    full = oracle.field(src, par, ev)
    parts = sum(oracle.field(src, par, ev, kind=k, delta=delta, Aplus=Aplus, b=b) for k in ("local", "near", "far"))
    assert np.max(np.abs(parts - full)) <= 1e-12 * np.max(np.abs(full))
    # and the pieces are genuinely non-trivial
    loc = oracle.field(src, par, ev, kind="local", delta=delta, Aplus=Aplus, b=b)
    far = oracle.field(src, par, ev, kind="far", delta=delta, Aplus=Aplus, b=b)
    assert np.max(np.abs(loc)) > 1e-3 * np.max(np.abs(full))
    assert np.max(np.abs(far)) > 1e-3 * np.max(np.abs(full))


def test_self_term_is_the_r_to_zero_limit_of_the_history_field():
    # history = full - local is smooth in r; at r -> 0 it tends to (1/2pi) int phi(d) sigma(t-d)/d dd
    rng = np.random.default_rng(10)
    par = inputs.gauss3_params(1, 8.0, rng)
    delta, b = 0.8, math.log(1e8)
    src = np.array([[0.0, 0.0]])
    ts = np.array([7.0, 9.5, 12.0])
    r = 1e-6 * delta
    ev = np.column_stack([np.full(3, r), np.zeros(3), ts])
    hist = oracle.field(src, par, ev) - oracle.field(src, par, ev, kind="local", delta=delta, Aplus=100.0, b=b)
    self_ = oracle.self_term(np.repeat(par, 3, axis=0), ts, delta, b)
    assert np.max(np.abs(hist - self_)) <= 1e-10 * max(1.0, np.max(np.abs(self_)))
    assert np.max(np.abs(self_)) > 1e-3


def test_signal_formula_matches_input_generator():
    # the oracle's C signal evaluation and the numpy input generator are independent implementations
    rng = np.random.default_rng(11)
    par = inputs.gauss3_params(5, 20.0, rng)
    t = np.linspace(-1, 25, 37)
    ref = inputs.sample_sigma(par, t, "gauss3")
    for j in range(5):
        got = np.array([oracle.sigma(par[j], tt) for tt in t])
        assert np.max(np.abs(got - ref[:, j])) <= 1e-15
    pe = inputs.erf_params(3, rng, 30.0, 1.5, 7.0)
    ref = inputs.sample_sigma(pe, t, "erf")
    for j in range(3):
        got = np.array([oracle.sigma(pe[j], tt, family="erf") for tt in t])
        assert np.max(np.abs(got - ref[:, j])) <= 1e-15


# ------------------------------------------------------------------ erf-switched signals
# The paper's own signal family (Sec. 7, Eq. exampleDensities): 0.5 (erf(5 (t - t0)) + 1) sin(w (t - t0)),
# with t0 in [1.5, 7] and w up to 10 pi as in its convergence study.  Its switch-on is the sharpest
# feature any workload here has, so the quadrature is pinned on it separately.
def _erf_case(seed, omega_max, M=6, Ne=10, box=3.0, T=8.0):
    rng = np.random.default_rng(seed)
    src = rng.uniform(0, box, (M, 2))
    par = inputs.erf_params(M, rng, omega_max, 1.5, 7.0, cube_root=False)
    par[0, 1] = omega_max  # one source at the top frequency
    ev = np.column_stack([rng.uniform(0, box, Ne), rng.uniform(0, box, Ne), rng.uniform(2.0, T, Ne)])
    return src, par, ev


@pytest.mark.parametrize("seed,omega_max", [(1, 10 * math.pi), (2, 10 * math.pi), (3, 30.0), (4, 2.0)])
def test_erf_family_node_doubling_and_cosh_quadrature(seed, omega_max):
    src, par, ev = _erf_case(seed, omega_max)
    a = oracle.field(src, par, ev, family="erf")
    c = oracle.field(src, par, ev, family="erf", method=1)
    try:
        oracle.set_resolution(40, 0.25)
        b = oracle.field(src, par, ev, family="erf")
    finally:
        oracle.set_resolution(20, 0.5)
    scale = np.max(np.abs(b))
    assert scale > 1e-2
    assert np.max(np.abs(a - b)) <= 1e-13 * scale
    assert np.max(np.abs(a - c)) <= 1e-13 * scale


def test_erf_family_brute_force_scipy_quad():
    integrate = pytest.importorskip("scipy.integrate")
    special = pytest.importorskip("scipy.special")
    src, par, ev = _erf_case(5, 10 * math.pi, M=2, Ne=3)
    got = oracle.field(src, par, ev, family="erf")
    for e in range(ev.shape[0]):
        x, y, t = ev[e]
        tot = 0.0
        for j in range(src.shape[0]):
            r = math.hypot(x - src[j, 0], y - src[j, 1])
            if r >= t:
                continue
            t0, w = par[j, 0], par[j, 1]

            def f(th):
                tau = t - r * math.cosh(th)
                return 0.5 * (special.erf(5 * (tau - t0)) + 1) * math.sin(w * (tau - t0)) if tau > 0 else 0.0

            # break the theta range where the emission time crosses the switch-on and zero
            pts = [math.acosh(d / r) for d in (t - t0 - 0.5, t - t0, t - t0 + 0.5, t) if r < d < t]
            v, _ = integrate.quad(f, 0.0, math.acosh(t / r), points=pts or None, limit=4000, epsabs=1e-14,
                                  epsrel=1e-13)
            tot += v / TWO_PI
        assert abs(got[e] - tot) <= 1e-11 * max(1.0, abs(tot)), (got[e], tot)


# ------------------------------------------------------- split components, one by one
# Each component oracle against scipy's adaptive quadrature of its own defining integral (Sec. 3,
# Eqs. ul, unh, ufh) in the cosh variable, with the blending function built independently from
# scipy's I0: phi(d) = int_0^d b/(delta sinh b) I0(b sqrt(1 - (2s/delta - 1)^2)) ds (Eq. KBblending).
@pytest.mark.parametrize("kind", ["local", "near", "far"])
def test_each_split_component_against_scipy(kind):
    integrate = pytest.importorskip("scipy.integrate")
    special = pytest.importorskip("scipy.special")
    delta, Aplus, b = 0.9, 4.1, math.log(1e8)
    rng = np.random.default_rng(12)
    par = inputs.gauss3_params(1, 8.0, rng)
    par[0, 3:6] = [4.0, 5.5, 7.0]
    src = np.array([[0.0, 0.0]])

    def phi(d):
        if d <= 0:
            return 0.0
        if d >= delta:
            return 1.0
        g = lambda s: b / (delta * math.sinh(b)) * special.i0(b * math.sqrt(max(0.0, 1 - (2 * s / delta - 1) ** 2)))
        return integrate.quad(g, 0.0, d, epsabs=1e-15, epsrel=1e-14)[0]

    def weight(d):
        if kind == "local":
            return 1.0 - phi(d) if d < delta else 0.0
        if kind == "near":
            return phi(d) * phi(Aplus - d) if d < Aplus else 0.0
        return 1.0 - phi(Aplus - d) if d > Aplus - delta else 0.0

    for (r, t) in [(0.35, 9.0), (0.05, 8.2), (0.7, 10.5)]:
        got = oracle.field(src, par, np.array([[r, 0.0, t]]), kind=kind, delta=delta, Aplus=Aplus, b=b)[0]
        f = lambda th: weight(r * math.cosh(th)) * inputs.sample_sigma(par, np.array([t - r * math.cosh(th)]),
                                                                          "gauss3")[0, 0]
        brk = [math.acosh(d / r) for d in (delta, Aplus - delta, Aplus) if r < d < t]
        ref = integrate.quad(f, 0.0, math.acosh(t / r), points=brk or None, limit=2000, epsabs=1e-13,
                             epsrel=1e-11)[0] / TWO_PI
        full = oracle.field(src, par, np.array([[r, 0.0, t]]))[0]
        assert abs(got - ref) <= 1e-10 * max(abs(full), 1e-3), (kind, r, t, got, ref)
        assert abs(got) > 1e-4 * abs(full) or kind == "far"
