"""GPU test of wfp_local_noalloc, the entry point that allocates nothing.

Callers that cannot allocate (code inside a stream capture, code bound to a fixed memory
arena, real-time loops) get the local part of a step from this entry point instead of from a
plan.  Its result must equal the local part that a plan computes for the same points and
signal window (wfp_step_components), on two calls in a row with different point sets, so that
the shared scratch array carries nothing from one call into the next.  The file is named so
that pytest collects it after every other test.
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
    for got, ref in ((out_a.cpu().numpy(), ul_a), (out_b.cpu().numpy(), ul_b)):
        assert np.max(np.abs(ref)) > 0
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


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
