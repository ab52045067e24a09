"""GPU test of wfp_local_noalloc, the entry point that allocates nothing.

Callers whose device memory all comes from a fixed arena they may not grow, or real-time loops
that may not pay for an allocation and the synchronisation it can cause, get the local part of a
step from this entry point instead of from a plan (a plan allocates in wfp_plan_create).  Its
result must equal the local part that a plan computes for the same points and signal window
(wfp_step_components), on two calls in a row with different point sets, so that the shared
scratch array carries nothing from one call into the next; both calls are also checked against
the oracle's local component of the exact field.  The file is named so that pytest collects it
after every other test.
"""
import numpy as np
import pytest

from paper_2604_07170_gb300 import inputs

pytestmark = pytest.mark.gpu


def _plan_local(wl, tgt, n):
    from paper_2604_07170_gb300 import wfp
    plan = wfp.Plan(wl.src_xy, tgt, wl.dt, wl.n_steps, wl.band_limit, wl.tol)
    nmax = plan.info()["nmax"]
    sig = wl.sigma(1, n + 1)
    for k in range(n):
        plan.step(sig[k])
    ul, _, _ = plan.components()
    plan.close()
    win = np.zeros((nmax, wl.M))
    lev = np.arange(n - nmax + 1, n + 1)
    ok = lev >= 1
    win[ok] = sig[lev[ok] - 1]
    return ul, win, nmax


def test_local_noalloc_matches_plan_two_calls():
    import torch
    from paper_2604_07170_gb300 import wfp
    dev = torch.device("cuda", 0)
    wl = inputs.small(140, 3.0, 70, seed=4)
    rng = np.random.default_rng(9)
    tgt_b = rng.uniform(0.0, 3.0, (57, 2))
    n = 70
    ul_a, win, nmax = _plan_local(wl, None, n)     # targets = sources (coincident pairs excluded)
    ul_b, win_b, _ = _plan_local(wl, tgt_b, n)     # separate targets
    src = torch.from_numpy(np.ascontiguousarray(wl.src_xy)).to(dev)
    tb = torch.from_numpy(np.ascontiguousarray(tgt_b)).to(dev)
    w = torch.from_numpy(win).to(dev)
    out_a = torch.empty(wl.M, dtype=torch.float64, device=dev)
    out_b = torch.empty(tgt_b.shape[0], dtype=torch.float64, device=dev)
    # two calls in a row: different target sets share the one scratch array
    wfp.local_noalloc(src, src, w, nmax, wl.dt, wl.band_limit, wl.tol, out_a)
    wfp.local_noalloc(src, tb, w, nmax, wl.dt, wl.band_limit, wl.tol, out_b)
    torch.cuda.synchronize(dev)
    got_a, got_b = out_a.cpu().numpy(), out_b.cpu().numpy()
    for got, ref in ((got_a, ul_a), (got_b, ul_b)):
        assert np.max(np.abs(ref)) > 0
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    # against the oracle: the local component of the exact field, weight 1 - phi(d) on delays below
    # delta = W dt (the split of the field into local and history parts)
    import oracle
    pr = wfp.select_params(1.5, wl.dt, wl.n_steps, wl.band_limit, wl.tol)
    delta = pr["W"] * wl.dt
    for got, tgt in ((got_a, wl.src_xy), (got_b, tgt_b)):
        ev = np.column_stack([tgt, np.full(tgt.shape[0], n * wl.dt)])
        ref = oracle.field(wl.src_xy, wl.params, ev, kind="local", delta=delta, Aplus=1e3, b=pr["b"],
                           r_coinc=1e-12 * wl.meta["box"])
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print(f"\nno-alloc local part vs oracle local component: rel L2 {err:.2e}")
        assert err <= 1e-6


def test_local_noalloc_rejects_oversize():
    import torch
    from paper_2604_07170_gb300 import wfp
    dev = torch.device("cuda", 0)
    M = 70000  # beyond the fixed scratch's 65536 sources
    src = torch.zeros((M, 2), dtype=torch.float64, device=dev)
    w = torch.zeros((32, M), dtype=torch.float64, device=dev)
    out = torch.empty(10, dtype=torch.float64, device=dev)
    with pytest.raises(wfp.WFPError) as ei:
        wfp.local_noalloc(src, src[:10], w, 32, 0.1, 12.7, 1e-6, out)
    assert ei.value.code == wfp.WFP_EINVAL


def test_local_noalloc_rejects_a_target_on_two_sources():
    # a plan rejects a target that coincides with two sources; so does the allocation-free call
    import torch
    from paper_2604_07170_gb300 import wfp
    dev = torch.device("cuda", 0)
    wl = inputs.small(40, 3.0, 70, seed=4)
    src = np.ascontiguousarray(wl.src_xy.copy())
    src[1] = src[0]
    pr = wfp.select_params(1.5, wl.dt, wl.n_steps, wl.band_limit, wl.tol)
    s = torch.from_numpy(src).to(dev)
    w = torch.zeros((pr["nmax"], wl.M), dtype=torch.float64, device=dev)
    out = torch.empty(wl.M, dtype=torch.float64, device=dev)
    with pytest.raises(wfp.WFPError) as ei:
        wfp.local_noalloc(s, s, w, pr["nmax"], wl.dt, wl.band_limit, wl.tol, out)
    assert ei.value.code == wfp.WFP_EUNSUPPORTED
    with pytest.raises(wfp.WFPError) as ei:
        wfp.Plan(src, None, wl.dt, wl.n_steps, wl.band_limit, wl.tol)
    assert ei.value.code == wfp.WFP_EUNSUPPORTED
