"""The per-step error measure of the parity tests (relative L2 against the oracle, with a floor).

    e_n = ||u~_n - u_n||_2 / max(||u_n||_2, f * max_m ||u_m||_2)

over the sampled steps m.  Bar: e_n <= 1e-6 on both paths.  The floor f keeps steps whose field is
nearly zero (the leading edge of the pulses, the tail after they pass) from being divided by ~0:

* FP64 path: f = 1e-2, i.e. those steps are held to an absolute error of 1e-8 of the peak field.
* Mixed path: f = 1e-1, i.e. an absolute 1e-7 of the peak field.  Its type-2 evaluation rounds the
  mode amplitudes to FP32 and transforms them in FP32, so its error is relative to the amplitude of
  the whole near-history field in the periodic box, which stays near its peak for A+ after the
  pulses pass (the outgoing waves), while the field at the targets falls by orders of magnitude.
  Measured at 10^4 points: 4e-7 of the field at active steps, an absolute ~8e-8 of the peak field in
  the tail (history part only; the local part and the self term are exact zeros there).
"""
import numpy as np

BAR = 1e-6
FLOOR = {0: 1e-2, 1: 1e-1}  # by precision: WFP_FP64, WFP_MIXED


def rel_errors(got, ref, precision=0):
    """e_n per row (step) of got / ref, arrays [steps][targets]."""
    got, ref = np.asarray(got), np.asarray(ref)
    norms = np.linalg.norm(ref, axis=1)
    floor = FLOOR[precision] * norms.max()
    return np.linalg.norm(got - ref, axis=1) / np.maximum(norms, floor)
