"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

The oracle evaluates the exact retarded field (Eq. exactSol) at sampled (target, step)
pairs; the CUDA path steps the 2D TK-WFP method (Secs. 3-6) through every step.  Bar:
relative L2 error per step <= 1e-6 with the floor of tests/_metric.py (1% of the peak field
on the FP64 path, 10% on the mixed path).
"""
import math

import numpy as np
import pytest

import oracle
from _metric import BAR, rel_errors
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


def test_small_uniform_coincident_all_parts_active():
    # box 3 x 3 wavelengths, 250 steps: lagged type-1 and far history switch on after ~75 steps
    wl = inputs.small(150, 3.0, 250, seed=1)
    got, info, _ = run_plan(wl)
    assert info["lag_active"] and info["far_active"] and info["n_self"] == 150
    steps = [20, 60, 90, 130, 170, 210, 250]
    ref = oracle_at(wl, None, steps)
    e = rel_errors(got[np.array(steps) - 1], ref)
    print("\nrel L2 per step:", dict(zip(steps, np.round(e, 10))), info["L"], info["n_modes"])
    assert e.max() <= BAR


def test_cfg1_all_steps_all_targets():
    # M = 200 coincident sources/targets uniform in a 5 x 5-wavelength square, N_t = 100
    wl = inputs.make("cfg1")
    got, info, _ = run_plan(wl)
    steps = list(range(5, 101, 5))
    ref = oracle_at(wl, None, steps)
    e = rel_errors(got[np.array(steps) - 1], ref)
    print("\ncfg1 rel L2:", np.array2string(e, precision=2))
    assert e.max() <= BAR


@pytest.mark.parametrize("precision", [0, 1])
def test_cfg1_geometry_through_the_whole_pulses(precision):
    # cfg1's 200 points with its signals (pulse centres at t = 8..13) stepped to T = 25: the pulses rise,
    # pass and leave their tail, and the lag and far history switch on; every 5th step, every target
    wl = inputs.make("cfg1")
    wl.n_steps = 250
    got, info, _ = run_plan(wl, precision=precision)
    assert info["lag_active"] and info["far_active"] and info["n_self"] == 200
    steps = list(range(5, 251, 5))
    ref = oracle_at(wl, None, steps)
    e = rel_errors(got[np.array(steps) - 1], ref, precision)
    print(f"\ncfg1 geometry to T = 25, precision {precision}, rel L2:", np.array2string(e, precision=2))
    assert e.max() <= BAR


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
    assert e.max() <= BAR


def test_mixed_precision_small():
    # FP32 spreading / FFT / taps / weights, FP64 state and accumulation (wfp_opts.precision = MIXED)
    wl = inputs.small(150, 3.0, 250, seed=1)
    got, info, _ = run_plan(wl, precision=1)
    assert info["local_form"] == 2 and 12 <= info["local_nc"] <= 36
    steps = [60, 130, 200, 250]
    ref = oracle_at(wl, None, steps)
    e = rel_errors(got[np.array(steps) - 1], ref, precision=1)
    print("\nmixed rel L2:", np.array2string(e, precision=2))
    assert e.max() <= BAR


def test_factored_local_part_fp64_equals_stored_rows():
    # the factored local part (each interval's weight series contracted with the source windows
    # first, then summed against T_c(x_ij) per pair) regroups the same table weights as the stored
    # rows: in FP64 with every coefficient kept, the two agree to rounding.  Targets: on the
    # sources (rows with near pairs, r < dt) and off the curve (rows without)
    from paper_2604_07170_gb300 import wfp
    wl = inputs.small(200, 4.0, 120, seed=2, curve=True)
    rng = np.random.default_rng(7)
    tgt = np.vstack([wl.src_xy[::3], rng.uniform(0.0, 4.0, (40, 2))])
    a, ia, ca = run_plan(wl, tgt_xy=tgt, local_form=wfp.LOCAL_STORED)
    b, ib, cb = run_plan(wl, tgt_xy=tgt, local_form=wfp.LOCAL_FACTORED)
    assert ia["local_form"] == 1 and ib["local_form"] == 2 and ib["local_nc"] == 36
    assert 0 < ib["n_near_pairs"] < ib["n_pairs"] == ia["n_pairs"]
    ul_a, ul_b = ca["last"][0], cb["last"][0]
    d_loc = np.linalg.norm(ul_b - ul_a) / np.linalg.norm(ul_a)
    d_all = np.linalg.norm(b - a) / np.linalg.norm(a)
    print(f"\nfactored vs stored FP64: local {d_loc:.2e}, field {d_all:.2e}")
    assert d_loc <= 1e-13 and d_all <= 1e-13


def test_factored_local_part_mixed_against_oracle():
    # the mixed path's factored local part (series cut where its tail drops below FP32 rounding,
    # FP32 contraction and recurrences, compensated sums) against the oracle and beside the stored
    # FP32 rows: same error level
    from paper_2604_07170_gb300 import wfp
    wl = inputs.small(300, 4.0, 220, seed=3, curve=True)
    steps = [60, 120, 180, 220]
    ref = oracle_at(wl, None, steps)
    e = {}
    for form in (wfp.LOCAL_STORED, wfp.LOCAL_FACTORED):
        got, info, _ = run_plan(wl, precision=1, local_form=form)
        assert info["local_form"] == form
        e[form] = rel_errors(got[np.array(steps) - 1], ref, precision=1)
    print("\nmixed stored / factored rel L2:", np.array2string(e[1], precision=2), np.array2string(e[2], precision=2))
    assert e[2].max() <= max(2 * e[1].max(), 1e-7)
    assert e[2].max() <= BAR
