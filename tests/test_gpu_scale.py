"""GPU parity at the larger workloads (mixed precision), sampled against the FP64 oracle.

cfg3: 10^5 coincident points on 40 ellipses in a 100 x 100-wavelength box, N_t = 4000 (the lagged
S and the far history switch on after step 2403).  cfg4: 10^6 points on 100 ellipses in a
300 x 300-wavelength box, N_t = 3000 (T below A+: local part and near history only).  The plan is
the one the bench times; a few random targets are compared with the oracle at sampled steps.
"""
import numpy as np
import pytest

import oracle
from _metric import BAR, rel_errors
from paper_2604_07170_gb300 import inputs

pytestmark = pytest.mark.gpu


def _sampled(name, steps, n_tgt, bound):
    from paper_2604_07170_gb300 import wfp
    wl = inputs.make(name)
    plan = wfp.Plan(wl.src_xy, None, wl.dt, wl.n_steps, wl.band_limit, wl.tol, precision=1)
    rng = np.random.default_rng(7)
    idx = rng.choice(wl.M, n_tgt, replace=False)
    got = {}
    last = max(steps)
    for n0 in range(0, last, 200):
        sig = wl.sigma(n0 + 1, min(last, n0 + 200) + 1)
        for k in range(sig.shape[0]):
            u = plan.step(sig[k])
            if n0 + k + 1 in steps:
                got[n0 + k + 1] = u[idx]
    info = plan.info()
    plan.close()
    ev = np.array([[wl.src_xy[i, 0], wl.src_xy[i, 1], n * wl.dt] for n in steps for i in idx])
    ref = oracle.field(wl.src_xy, wl.params, ev, r_coinc=1e-12 * wl.meta["box"]).reshape(len(steps), -1)
    errs = rel_errors(np.array([got[n] for n in steps]), ref, precision=1)
    print(f"\n{name} mixed sampled rel L2:", np.array2string(np.array(errs), precision=2),
          "device GB", round(info["device_bytes"] / 1e9, 1), "lag", info["lag_active"], info["lag_store"])
    assert max(errs) <= bound
    return info


def test_cfg3_mixed_sampled():
    info = _sampled("cfg3", [1200, 2600], 24, BAR)
    assert info["lag_active"] and info["far_active"]


def test_cfg4_mixed_sampled():
    info = _sampled("cfg4", [150, 400], 32, BAR)
    assert not info["lag_active"]
