/*
 * wfp_debug.h -- diagnostics of the 2D TK-WFP evaluator.
 *
 * All but the last expose the plan-time quadrature routines that the CUDA path runs on the
 * device, so that tests on a machine without a GPU can check them against closed forms and
 * against the independent CPU oracle; they allocate only host memory.  wfp_debug_bounded_wait
 * runs on the GPU.  All return WFP_EINVAL on bad arguments; output arrays are owned by the caller.
 */
#ifndef WFP_DEBUG_H
#define WFP_DEBUG_H

#include "wfp.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Local-part weights eta_l(r), l = 0..nmax-1 with nmax = W + 1 + p/2 (Sec. 6, Eqs. local2,
 * sigInterp, ul_GL): u_l(t_n) = sum_l eta_l(r) sigma(t_{n-nmax+1+l}) for one source-target pair
 * at distance r in (0, W dt), including the factor 1/(2 pi).  eps sets the blending-function
 * shape b = ln(1/eps); band_limit (rad per unit of dt's time) sets the band of the least-squares
 * interpolation used on the newest delay intervals (a negative value selects Lagrange interpolation
 * there too); ng is the number of Gauss-Legendre nodes per panel.  eta: nmax doubles.
 */
wfp_status wfp_debug_eta(double r, double dt, int W, int p, double eps, double band_limit, int ng, double* eta);

/*
 * The same weights as plans compute them: for r >= dt from the Chebyshev table of each delay
 * interval [k dt, (k+1) dt] (series in sqrt((k+1) dt - r), built from eta_weights at Chebyshev
 * points), for r < dt by the direct quadrature above.  Arguments as wfp_debug_eta.
 */
wfp_status wfp_debug_eta_table(double r, double dt, int W, int p, double eps, double band_limit, int ng, double* eta);

/*
 * The per-interval Chebyshev table behind wfp_debug_eta_table and the coefficient count the factored
 * local part keeps (wfp_opts.local_form): coefficients of the weights on the delay intervals
 * k = 1..W-1, tab[((k - 1) nmax + l) 33 + c] for the series sum_c tab[..][c] T_c(x) in
 * x = 2 sqrt(((k+1) dt - r) / dt) - 1 (nmax = W + 1 + p/2).  *nc = the coefficients kept by a plan
 * of the given precision (WFP_MIXED: the first multiple of 4, at least 16 and at most 32, whose
 * dropped tail is within 2^-25 of the interval's weight scale; WFP_FP64: all, reported as 36 with
 * zero padding); *tail = the largest dropped tail over intervals and levels relative to the
 * interval's weight scale max_l sum_c |tab|.  tab may be NULL; else (W - 1) * nmax * 33 doubles.
 * Arguments otherwise as wfp_debug_eta; host only.
 */
wfp_status wfp_debug_factored_table(double dt, int W, int p, double eps, double band_limit, int ng, int precision,
                                    int* nc, double* tail, double* tab);

/*
 * Near-history FIR taps at wavenumber magnitude kappa (Lemma 4.2, Eq. hggrid), dt folded in:
 * taps[0..W) = p_m, [W..2W) = q_m, [2W..3W) = pA_m, [3W..4W) = qA_m; lagshift = A+ - delta.
 * rot = {cos(kappa dt), sin(kappa dt)/kappa, kappa sin(kappa dt)}.  taps: 4W doubles, rot: 3.
 */
wfp_status wfp_debug_taps(double kappa, double dt, int W, double eps, double lagshift, double* taps, double* rot);

/* Blending function phi_delta(t) and its first two derivatives (Eq. KBblending), b = ln(1/eps). */
wfp_status wfp_debug_phi(double t, double delta, double eps, double* phi, double* dphi, double* d2phi);

/*
 * Nodes and weights of the dyadic-panel sum of exponentials (Sec. 2.3, Eq. LaplaceApprox):
 * panels [0, lmax/2^(panels-1)], ..., [lmax/2, lmax] with ng Gauss-Legendre nodes each.
 * lam, q: panels*ng doubles each.
 */
wfp_status wfp_debug_soe(double lam_max, int panels, int ng, double* lam, double* q);

/*
 * Nodes and weights of the self term's sum of exponentials for 1/d on [dlo, T] (the regularised
 * self history of coincident pairs, whose kernel at r = 0 is 1/(2 pi d); its recurrence follows the
 * far history's, Sec. 5): Gauss-Legendre in lambda on [0, 8/T] and composite Gauss-Legendre in
 * ln(lambda) above, the fewest terms found with relative error <= 0.8 eps on [dlo, T].  Host only.
 * lam, q: cap doubles each; *n = the number of terms (also set when it exceeds cap, which returns
 * WFP_EINVAL).
 */
wfp_status wfp_debug_self_soe(double dlo, double T, double eps, int cap, double* lam, double* q, int* n);

/*
 * Hankel coefficients of the far history (Sec. 5, Eq. H) at wavenumber magnitude kappa:
 * H_l = q_l exp(-A lam_l) int_0^A J0(kappa r) I0(lam_l r) phi_Delta(A - r) r dr for the dyadic
 * sum of exponentials (lam_max, panels, ng) above, with the composite Gauss-Legendre rule in r
 * that plans use.  H: panels*ng doubles.
 */
wfp_status wfp_debug_hankel(double kappa, double A, double Delta, double eps, double lam_max, int panels, int ng,
                            double* H);

/*
 * The bounded wait that every mbarrier wait of the CUDA path uses (the bulk-copy pipeline of the
 * local part), run once on the current GPU by one warp on an mbarrier of its own shared memory
 * (no copies involved): with arrive = 0 nothing completes the barrier's phase and the wait must
 * run out after limit_s seconds (0.001 .. 1); with arrive = 1 the phase is completed first and the
 * wait must succeed at once.  *timed_out receives 1 if the wait ran out, *waited_s the wall time
 * the wait took (device global timer).  Requires a GPU; WFP_ECUDA if the launch fails.
 */
wfp_status wfp_debug_bounded_wait(double limit_s, int arrive, int* timed_out, double* waited_s);

/*
 * Measured arithmetic peak of the current GPU (no counterpart in the paper: the denominator of the
 * roofline of the parts bound by arithmetic rather than memory).  A grid of 8 blocks of 256 threads
 * per SM runs 8 independent fused multiply-add chains per thread, in FP64 (fp64 = 1) or FP32 (0),
 * timed with CUDA events on the calling thread's default stream; the best of three launches after
 * one warm-up is reported.  *tflops = 2 flops per FMA over that time, *ms = its duration.
 * Allocates and frees a small device buffer; synchronises.  Requires a GPU; WFP_ECUDA on failure.
 */
wfp_status wfp_debug_alu_peak(int fp64, double* tflops, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* WFP_DEBUG_H */
