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


def test_local_interpolation_order_convergence():
    # Lagrange-only local interpolation (the paper's form), eps = 1e-8, W = 24: the error falls with
    # the interpolation order p until it meets the eps floor of the history parts
    from paper_2604_07170_gb300 import wfp
    src, tgt, par, dt, nt, K0 = _erf_workload(omega_max=30.0, eps=1e-8)
    n = 250
    sig = inputs.sample_sigma(par, dt * np.arange(1, n + 1), "erf")
    ref = _oracle(src, par, tgt, [n], dt, 3.0)[0]
    errs = {}
    for p in (4, 6, 8, 10, 12):
        plan = wfp.Plan(src, tgt, dt, nt, K0, 1e-5, eps=1e-8, W=24, p=p, local_interp=wfp.INTERP_LAGRANGE)
        for k in range(n):
            u = plan.step(sig[k])
        plan.close()
        errs[p] = float(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    print("\nrel L2 by interpolation order:", {p: f"{e:.2e}" for p, e in errs.items()})
    assert errs[4] > errs[6] > errs[8]
    assert errs[4] > 100 * errs[10]
    assert errs[12] < 1e-6


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
