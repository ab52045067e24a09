"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

The oracle evaluates the exact retarded field (Eq. exactSol) at sampled (target, step)
pairs; the CUDA path steps the 2D TK-WFP method (Secs. 3-6) through every step.  Bar:
relative L2 error per step <= 1e-6 (FP64 path), with the error measure
e_n = ||u~_n - u_n||_2 / max(||u_n||_2, 1e-2 max_m ||u_m||_2):
steps whose field is below 1% of its peak (the leading edge of the pulses) are held to an
absolute error of 1e-8 of the peak field.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2604_07170_gb300 import inputs

pytestmark = pytest.mark.gpu


def run_plan(wl, tgt_xy=None, steps=None, **opts):
    from paper_2604_07170_gb300 import wfp
    tgt = wl.src_xy if tgt_xy is None else tgt_xy
    steps = wl.n_steps if steps is None else steps
    plan = wfp.Plan(wl.src_xy, tgt, wl.dt, wl.n_steps, wl.band_limit, wl.tol, **opts)
    sig = wl.sigma(1, steps + 1)
    out = np.zeros((steps, tgt.shape[0]))
    comps = {}
    for n in range(1, steps + 1):
        out[n - 1] = plan.step(sig[n - 1])
    info = plan.info()
    comps["last"] = plan.components()
    plan.close()
    return out, info, comps


def oracle_at(wl, tgt_xy, steps_idx, tgt_idx=None):
    tgt = wl.src_xy if tgt_xy is None else tgt_xy
    ti = np.arange(tgt.shape[0]) if tgt_idx is None else np.asarray(tgt_idx)
    ev = np.array([[tgt[i, 0], tgt[i, 1], n * wl.dt] for n in steps_idx for i in ti])
    u = oracle.field(wl.src_xy, wl.params, ev, r_coinc=1e-12 * wl.meta["box"])
    return u.reshape(len(steps_idx), len(ti))


def rel_errors(got, ref):
    norms = np.linalg.norm(ref, axis=1)
    floor = 1e-2 * norms.max()
    return np.linalg.norm(got - ref, axis=1) / np.maximum(norms, floor)


def test_small_uniform_coincident_all_parts_active():
    # box 3 x 3 wavelengths, 250 steps: lagged type-1 and far history switch on after ~75 steps
    wl = inputs.small(150, 3.0, 250, seed=1)
    got, info, _ = run_plan(wl)
    assert info["lag_active"] and info["far_active"] and info["n_self"] == 150
    steps = [20, 60, 90, 130, 170, 210, 250]
    ref = oracle_at(wl, None, steps)
    e = rel_errors(got[np.array(steps) - 1], ref)
    print("\nrel L2 per step:", dict(zip(steps, np.round(e, 10))), info["L"], info["n_modes"])
    assert e.max() <= 1e-6


def test_cfg1_all_steps_all_targets():
    # M = 200 coincident sources/targets uniform in a 5 x 5-wavelength square, N_t = 100
    wl = inputs.make("cfg1")
    got, info, _ = run_plan(wl)
    steps = list(range(5, 101, 5))
    ref = oracle_at(wl, None, steps)
    e = rel_errors(got[np.array(steps) - 1], ref)
    print("\ncfg1 rel L2:", np.array2string(e, precision=2))
    assert e.max() <= 1e-6


def test_separate_targets_on_curve():
    # targets distinct from sources (no self term), sources on ellipses
    wl = inputs.small(200, 4.0, 220, seed=2, curve=True)
    rng = np.random.default_rng(5)
    tgt = rng.uniform(0.0, 4.0, (80, 2))
    got, info, _ = run_plan(wl, tgt_xy=tgt)
    assert info["n_self"] == 0
    steps = [40, 100, 160, 220]
    ref = oracle_at(wl, tgt, steps)
    e = rel_errors(got[np.array(steps) - 1], ref)
    print("\ncurve/targets rel L2:", np.array2string(e, precision=2))
    assert e.max() <= 1e-6


def test_mixed_precision_small():
    # FP32 spreading / FFT / taps / weights, FP64 state and accumulation (wfp_opts.precision = MIXED)
    wl = inputs.small(150, 3.0, 250, seed=1)
    got, info, _ = run_plan(wl, precision=1)
    steps = [60, 130, 200, 250]
    ref = oracle_at(wl, None, steps)
    e = rel_errors(got[np.array(steps) - 1], ref)
    print("\nmixed rel L2:", np.array2string(e, precision=2))
    assert e.max() <= 1e-5
