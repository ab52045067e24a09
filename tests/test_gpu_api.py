"""GPU tests of the C ABI's behaviour and of full-size workloads (through the C ABI)."""
import math

import numpy as np
import pytest

import oracle
from _metric import BAR, FLOOR
from paper_2604_07170_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(wl, steps, tgt=None, **opts):
    from paper_2604_07170_gb300 import wfp
    plan = wfp.Plan(wl.src_xy, tgt, wl.dt, wl.n_steps, wl.band_limit, wl.tol, **opts)
    sig = wl.sigma(1, steps + 1)
    out = np.stack([plan.step(sig[n]) for n in range(steps)])
    info = plan.info()
    plan.close()
    return out, info


def test_stored_history_and_lagged_nufft_give_identical_fields():
    # the lagged type-1 NUFFT reproduces the stored S levels bit for bit (deterministic spreading,
    # same cuFFT plan), so both ways of feeding the removal term give the same field
    from paper_2604_07170_gb300 import wfp
    wl = inputs.small(120, 3.0, 200, seed=11)
    a, ia = _run(wl, 200, lag_mode=wfp.LAG_STORE)
    b, ib = _run(wl, 200, lag_mode=wfp.LAG_RECOMPUTE)
    assert ia["lag_store"] == 1 and ib["lag_store"] == 0 and ia["lag_active"]
    assert np.array_equal(a, b)


def test_mixed_lag_modes_agree():
    from paper_2604_07170_gb300 import wfp
    wl = inputs.small(120, 3.0, 200, seed=12)
    a, _ = _run(wl, 200, precision=1, lag_mode=wfp.LAG_STORE)
    b, _ = _run(wl, 200, precision=1, lag_mode=wfp.LAG_RECOMPUTE)
    assert np.array_equal(a, b)


def test_graph_replay_equals_direct_launches():
    wl = inputs.small(90, 3.0, 160, seed=13)
    a, _ = _run(wl, 160, use_graph=1)
    b, _ = _run(wl, 160, use_graph=0)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [0, 1])
def test_serial_and_concurrent_step_orders_give_the_same_bits(precision):
    # the local branch and the advance share no written buffer, so issuing them one after the other
    # or on concurrent streams changes no bit (every part active: lag, far history, self term)
    from paper_2604_07170_gb300 import wfp
    wl = inputs.small(140, 3.0, 200, seed=23)
    a, ia = _run(wl, 200, precision=precision, step_order=wfp.ORDER_CONCURRENT)
    b, ib = _run(wl, 200, precision=precision, step_order=wfp.ORDER_SERIAL)
    assert ia["step_order"] == wfp.ORDER_CONCURRENT and ib["step_order"] == wfp.ORDER_SERIAL
    assert ia["lag_active"] and ia["far_active"] and ia["n_self"] > 0
    assert np.array_equal(a, b)


def test_device_and_host_pointers_give_the_same_field():
    import torch
    from paper_2604_07170_gb300 import wfp
    wl = inputs.small(80, 3.0, 60, seed=14)
    a, _ = _run(wl, 60)
    # device pointers: the step is ordered on the plan's stream (here a torch stream), so the
    # caller synchronises that stream before reading the output
    stream = torch.cuda.Stream()
    plan = wfp.Plan(wl.src_xy, None, wl.dt, wl.n_steps, wl.band_limit, wl.tol, stream=stream.cuda_stream)
    sig = torch.from_numpy(wl.sigma(1, 61)).cuda()
    out = torch.empty(wl.M, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    got = []
    for n in range(60):
        plan.step(sig[n], out)
        stream.synchronize()
        got.append(out.cpu().numpy().copy())
    plan.close()
    assert np.array_equal(a, np.stack(got))


def test_page_locked_host_buffers_give_the_same_field():
    # page-locked host buffers are copied by the DMA engines directly (no staging copy); pinned
    # input with pageable output, and the reverse, take the staged path for one side
    import torch
    from paper_2604_07170_gb300 import wfp
    wl = inputs.small(80, 3.0, 60, seed=14)
    a, _ = _run(wl, 60)
    sig = torch.from_numpy(wl.sigma(1, 61)).pin_memory().numpy()
    out_pin = torch.empty(wl.M, dtype=torch.float64, pin_memory=True).numpy()
    plan = wfp.Plan(wl.src_xy, None, wl.dt, wl.n_steps, wl.band_limit, wl.tol)
    got = []
    for n in range(60):
        if n % 3 == 0:
            got.append(plan.step(sig[n], out_pin).copy())
        elif n % 3 == 1:
            got.append(plan.step(sig[n]).copy())              # pinned in, pageable out
        else:
            got.append(plan.step(np.array(sig[n]), out_pin).copy())  # pageable in, pinned out
    plan.close()
    assert np.array_equal(a, np.stack(got))


def test_stepping_past_Nt_is_an_error_and_the_plan_survives():
    from paper_2604_07170_gb300 import wfp
    wl = inputs.small(30, 2.0, 5, seed=15)
    plan = wfp.Plan(wl.src_xy, None, wl.dt, 5, wl.band_limit, wl.tol)
    sig = wl.sigma(1, 6)
    for n in range(5):
        plan.step(sig[n])
    with pytest.raises(wfp.WFPError) as ei:
        plan.step(sig[0])
    assert ei.value.code == wfp.WFP_ESTATE
    assert plan.info()["n_modes"] > 0
    plan.close()


def test_single_coincident_source_has_zero_field():
    # one source at the only target: the self term is excluded (Eq. exactSol), the field is 0
    wl = inputs.small(1, 1.0, 120, seed=16)
    out, info = _run(wl, 120)
    assert info["n_self"] == 1 and info["n_pairs"] == 0
    assert np.max(np.abs(out)) < 1e-8


def test_self_term_included_when_not_excluded():
    # exclude_self = 0 returns the method's raw field: oracle field + the coincident self term
    wl = inputs.small(40, 2.5, 150, seed=17)
    a, info_a = _run(wl, 150)
    b, info_b = _run(wl, 150, exclude_self=0)
    assert info_a["n_self"] == 40 and info_b["n_self"] == 0
    n = 150
    delta = info_a["delta"] / info_a["scale"]
    selfv = oracle.self_term(wl.params, np.full(wl.M, n * wl.dt), delta, info_a["b"])
    assert np.linalg.norm((b[-1] - a[-1]) - selfv) <= 1e-6 * np.linalg.norm(a[-1])


def test_profiling_reports_every_part():
    from paper_2604_07170_gb300 import wfp
    wl = inputs.small(100, 3.0, 120, seed=18)
    plan = wfp.Plan(wl.src_xy, None, wl.dt, wl.n_steps, wl.band_limit, wl.tol)
    sig = wl.sigma(1, 121)
    plan.profile(True)
    for n in range(120):
        plan.step(sig[n])
    parts = plan.profile_read()
    plan.close()
    for name in ("ingest", "local", "self", "combine", "spread", "fft_type1", "modes", "far", "fft_type2", "interp"):
        assert parts[name][1] > 0, name


def _full_size_parity(name, precision, steps_check, n_tgt, bound):
    from paper_2604_07170_gb300 import wfp
    wl = inputs.make(name)
    plan = wfp.Plan(wl.src_xy, None, wl.dt, wl.n_steps, wl.band_limit, wl.tol, precision=precision)
    rng = np.random.default_rng(5)
    idx = rng.choice(wl.M, n_tgt, replace=False)
    got = {}
    last = max(steps_check)
    chunk = 200
    for n0 in range(0, last, chunk):
        sig = wl.sigma(n0 + 1, min(last, n0 + chunk) + 1)
        for k in range(sig.shape[0]):
            u = plan.step(sig[k])
            if n0 + k + 1 in steps_check:
                got[n0 + k + 1] = u[idx]
    info = plan.info()
    plan.close()
    refs = {}
    for n in steps_check:
        ev = np.column_stack([wl.src_xy[idx], np.full(n_tgt, n * wl.dt)])
        refs[n] = oracle.field(wl.src_xy, wl.params, ev, r_coinc=1e-12 * wl.meta["box"])
    floor = FLOOR[precision] * max(np.linalg.norm(r) for r in refs.values())
    errs = [np.linalg.norm(got[n] - refs[n]) / max(np.linalg.norm(refs[n]), floor) for n in steps_check]
    print(f"\n{name} precision={precision} sampled rel L2:", np.array2string(np.array(errs), precision=2),
          "lag_store", info["lag_store"])
    assert info["lag_active"] and info["far_active"]
    assert max(errs) <= bound


def test_cfg2_full_size_fp64_sampled():
    # 10^4 coincident points on ellipses, box 30, N_t = 2000 (lagged S / far history on after ~630
    # steps; the last pulses arrive near step 1080, after which the field is a decaying tail)
    _full_size_parity("cfg2", 0, [400, 800, 1060, 1254, 1400, 1800], 24, BAR)


def test_cfg2_full_size_mixed_sampled():
    # mixed path, the same steps: active ones, the last pulses' passage (1254) and the tail (1400, 1800,
    # field ~1e-9 of its peak) where the FP32 type-2 rounding of the outgoing waves' amplitudes sets an
    # absolute floor (tests/_metric.py)
    _full_size_parity("cfg2", 1, [400, 800, 1060, 1254, 1400, 1800], 24, BAR)


def test_spreading_tilings_give_identical_fields():
    # every grid point sums its sources in ascending order whatever the tile side or staging chunk,
    # so the autotuner's choice cannot change a bit of the result
    wl = inputs.small(300, 4.0, 120, seed=19, curve=True)
    outs = []
    for ts, ch in ((8, 32), (8, 64), (16, 32), (16, 64), (32, 32), (32, 64)):
        o, info = _run(wl, 120, spread_tile=ts, spread_chunk=ch)
        assert info["spread_tile"] == ts and info["spread_chunk"] == ch
        outs.append(o)
    auto, info = _run(wl, 120)
    assert info["spread_tile"] in (8, 16, 32) and info["spread_chunk"] in (32, 64)
    for o in outs[1:] + [auto]:
        assert np.array_equal(outs[0], o)


@pytest.mark.parametrize("precision", [0, 1])
def test_local_variants_give_identical_fields(precision):
    # the warp-vector kernel and every bulk-staged configuration sum each lane's pairs in the same
    # order with the same arithmetic, so the autotuner's pick cannot change a bit
    wl = inputs.small(400, 5.0, 90, seed=20, curve=True)
    outs = []
    for v in range(1, 6):
        o, info = _run(wl, 90, precision=precision, local_variant=v, local_form=1)
        assert info["local_variant"] == v and info["local_form"] == 1
        outs.append(o)
    auto, info = _run(wl, 90, precision=precision, local_form=1)
    assert 1 <= info["local_variant"] <= 5
    for o in outs[1:] + [auto]:
        assert np.array_equal(outs[0], o)


def test_bounded_device_wait_runs_out_and_reports():
    # the wall-time bound of every mbarrier wait in the CUDA path: a phase nothing completes must
    # make the wait give up after its limit and report it; a completed phase must pass at once
    from paper_2604_07170_gb300 import wfp
    timed_out, waited = wfp.debug_bounded_wait(0.2, arrive=False)
    assert timed_out and 0.2 <= waited < 1.0
    timed_out, waited = wfp.debug_bounded_wait(0.2, arrive=True)
    assert not timed_out and waited < 0.01


@pytest.mark.parametrize("precision,lag_mode", [(0, 2), (1, 2), (0, 1)])
def test_checkpoint_resume_gives_the_same_bits(precision, lag_mode):
    # save mid-run (lagged S and far history active), resume in a fresh plan of the same inputs
    from paper_2604_07170_gb300 import wfp
    wl = inputs.small(120, 3.0, 220, seed=21)
    sig = wl.sigma(1, 221)
    kw = dict(precision=precision, lag_mode=lag_mode)
    a = wfp.Plan(wl.src_xy, None, wl.dt, wl.n_steps, wl.band_limit, wl.tol, **kw)
    for n in range(150):
        a.step(sig[n])
    assert a.info()["lag_active"]
    ck = a.checkpoint()
    ref = np.stack([a.step(sig[n]) for n in range(150, 220)])
    a.close()
    b = wfp.Plan(wl.src_xy, None, wl.dt, wl.n_steps, wl.band_limit, wl.tol, **kw)
    b.restore(ck)
    got = np.stack([b.step(sig[n]) for n in range(150, 220)])
    b.close()
    assert np.array_equal(ref, got)
    # a plan of other inputs refuses the state and stays usable: another N_t, or the same sizes and
    # derived parameters with one source moved (caught by the checkpoint's fingerprint of the inputs)
    moved = wl.src_xy.copy()
    moved[7] += 1e-3
    for c in (wfp.Plan(wl.src_xy, None, wl.dt, wl.n_steps + 1, wl.band_limit, wl.tol, **kw),
              wfp.Plan(moved, None, wl.dt, wl.n_steps, wl.band_limit, wl.tol, **kw)):
        with pytest.raises(wfp.WFPError) as ei:
            c.restore(ck)
        assert ei.value.code == wfp.WFP_EINVAL
        c.step(sig[0])
        c.close()


def test_one_step_plan_and_zero_signals():
    from paper_2604_07170_gb300 import wfp
    # N_t = 1: the only step has no advance phase (signals start smoothly, so the field is ~0)
    wl = inputs.small(50, 2.5, 1, seed=22)
    plan = wfp.Plan(wl.src_xy, None, wl.dt, 1, wl.band_limit, wl.tol)
    u = plan.step(wl.sigma(1, 2)[0])
    with pytest.raises(wfp.WFPError) as ei:
        plan.step(wl.sigma(1, 2)[0])
    assert ei.value.code == wfp.WFP_ESTATE
    plan.close()
    ev = np.column_stack([wl.src_xy, np.full(wl.M, wl.dt)])
    ref = oracle.field(wl.src_xy, wl.params, ev, r_coinc=1e-12 * wl.meta["box"])
    assert np.all(np.isfinite(u)) and np.max(np.abs(u - ref)) <= 1e-12
    # identically zero signals through every part (lag and far history active): exactly zero field
    wl = inputs.small(60, 3.0, 200, seed=23)
    for precision in (0, 1):
        plan = wfp.Plan(wl.src_xy, None, wl.dt, 200, wl.band_limit, wl.tol, precision=precision)
        z = np.zeros(wl.M)
        out = [plan.step(z) for _ in range(200)]
        assert plan.info()["lag_active"]
        plan.close()
        assert not np.any(np.stack(out))


@pytest.mark.parametrize("precision", [0, 1])
def test_isolated_target_has_only_history_contributions(precision):
    # a target farther than delta from every source has an empty local row (both local forms: the
    # mixed path uses the factored one)
    wl = inputs.small(80, 3.0, 150, seed=24)
    tgt = np.array([[1.5, 1.5], [-4.0, -4.0], [9.0, 1.0]])
    out, info = _run(wl, 150, tgt=tgt, precision=precision)
    assert info["local_form"] == (2 if precision else 1)
    ev = np.array([[x, y, n * wl.dt] for n in (60, 150) for (x, y) in tgt])
    ref = oracle.field(wl.src_xy, wl.params, ev).reshape(2, -1)
    got = out[[59, 149]]
    assert info["n_self"] == 0
    assert np.linalg.norm(got - ref) <= (1e-6 if precision == 0 else 1e-5) * np.linalg.norm(ref)
