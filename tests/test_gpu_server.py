"""GPU tests of the request server (wfp_server_* in include/wfp.h), through the C ABI.

A request's field must not depend on what else the server runs: run alone and run among
other requests of different sizes (admitted at different ticks), its outputs are bitwise
equal.  Its field is also checked against the FP64 oracle, and admission against the budget.
"""
import numpy as np
import pytest

import oracle
from _metric import BAR, rel_errors
from paper_2604_07170_gb300 import inputs

pytestmark = pytest.mark.gpu


def _req(M, box, n_steps, seed, curve=False):
    return inputs.small(M, box, n_steps, seed=seed, curve=curve)


def _submit(sv, wl, out_steps=None, tgt=None):
    return sv.submit(wl.src_xy, wl.params, wl.dt, wl.n_steps, wl.band_limit, wl.tol, tgt_xy=tgt,
                     out_steps=out_steps)


def test_request_alone_equals_request_in_a_mix():
    from paper_2604_07170_gb300 import wfp
    a = _req(150, 3.0, 250, seed=21)
    steps = [40, 130, 250]
    with wfp.Server(8 << 30, 16) as sv:
        ida = _submit(sv, a, steps)
        sv.run()
        alone = sv.result(ida)
        st = sv.query(ida)
    assert st["state"] == wfp.REQ_DONE and st["steps_done"] == 250
    others = [_req(400, 5.0, 180, seed=22), _req(60, 4.0, 300, seed=23, curve=True), _req(900, 8.0, 90, seed=24)]
    with wfp.Server(8 << 30, 16) as sv:
        ids = [_submit(sv, others[0]), _submit(sv, others[1])]
        for _ in range(17):  # a enters while others are part-way through
            sv.tick()
        ida = _submit(sv, a, steps)
        sv.tick()
        ids.append(_submit(sv, others[2]))
        sv.run()
        mixed = sv.result(ida)
        for i in ids:
            sv.result(i)  # raises with the request's error if it failed
    assert np.array_equal(alone, mixed)
    # and the field is right (signals are generated on the device from the same parameters)
    ev = np.array([[x, y, n * a.dt] for n in steps for (x, y) in a.src_xy])
    ref = oracle.field(a.src_xy, a.params, ev, r_coinc=1e-12 * a.meta["box"]).reshape(len(steps), -1)
    floor = 1e-2 * np.linalg.norm(ref, axis=1).max()
    e = np.linalg.norm(alone - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), floor)
    print("\nserver request rel L2:", e)
    assert e.max() <= 1e-6


def test_admission_respects_the_budget_and_arrival_order():
    from paper_2604_07170_gb300 import wfp
    wls = [_req(300, 4.0, 60, seed=30 + i) for i in range(4)]
    with wfp.Server(64 << 30, 16) as probe:  # learn one request's footprint
        i0 = _submit(probe, wls[0])
        probe.tick()
        assert probe.query(i0)["state"] in (wfp.REQ_BUILDING, wfp.REQ_ACTIVE)
        while probe.query(i0)["state"] == wfp.REQ_BUILDING:  # the plan is built on a worker thread
            probe.tick()
        need = probe.query(i0)["device_bytes"]
        plan_bytes = probe.query(i0)["plan_bytes"]
    # the admission estimate covers what the plan really holds (plus the cuFFT work areas)
    assert plan_bytes <= need <= 3 * plan_bytes, (need, plan_bytes)
    with wfp.Server(int(1.5 * need), 16) as sv:  # room for one request at a time
        ids = [_submit(sv, w) for w in wls]
        active, pending = sv.tick()
        assert active == 1 and pending == 3
        sv.run()
        st = [sv.query(i) for i in ids]
    assert all(s["state"] == wfp.REQ_DONE for s in st)
    for s0, s1 in zip(st, st[1:]):
        assert s1["t_admit"] >= s0["t_done"] - 1e-3  # served one after another, in order
    with wfp.Server(need // 4, 4) as sv:  # never fits: fails, the server carries on
        rid = _submit(sv, wls[0])
        sv.tick()
        assert sv.query(rid)["state"] == wfp.REQ_FAILED
        with pytest.raises(wfp.WFPError):
            sv.result(rid)


def test_separate_targets_and_mixed_precision_requests():
    from paper_2604_07170_gb300 import wfp
    wl = _req(200, 4.0, 160, seed=40, curve=True)
    tgt = np.random.default_rng(41).uniform(0.0, 4.0, (70, 2))
    with wfp.Server(8 << 30, 8, precision=wfp.MIXED) as sv:
        rid = _submit(sv, wl, [80, 160], tgt=tgt)
        sv.run()
        got = sv.result(rid)
    ev = np.array([[x, y, n * wl.dt] for n in (80, 160) for (x, y) in tgt])
    ref = oracle.field(wl.src_xy, wl.params, ev, r_coinc=1e-12 * wl.meta["box"]).reshape(2, -1)
    e = rel_errors(got, ref, precision=1)
    print("\nserver mixed rel L2:", e)
    assert e.max() <= BAR
