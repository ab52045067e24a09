// Plan-time quadrature of the 2D TK-WFP evaluator, usable on host and device:
// local-part weights (Sec. 6) and near-history FIR taps (Sec. 4.2, Eq. hggrid).
#pragma once

#include <math.h>

#include "wfp_internal.h"

namespace wfp {

constexpr int kMaxP = 32;        // interpolation order p <= 32

// Lagrange basis of the equispaced nodes k0, ..., k0+p-1 evaluated at X, by prefix/suffix
// products (no divisions); wl[i] = 1 / prod_{j != i} (i - j).
WFP_HD inline void lagrange_eq(double X, int k0, int p, const double* wl, double* xi) {
    double pre[kMaxP + 1];
    pre[0] = 1.0;
    for (int i = 0; i < p; i++) pre[i + 1] = pre[i] * (X - (double)(k0 + i));
    double suf = 1.0;
    for (int i = p - 1; i >= 0; i--) {
        xi[i] = wl[i] * pre[i] * suf;
        suf *= (X - (double)(k0 + i));
    }
}

WFP_HD inline void lagrange_ref_weights(int p, double* wl) {
    for (int i = 0; i < p; i++) {
        double d = 1.0;
        for (int j = 0; j < p; j++)
            if (j != i) d *= (double)(i - j);
        wl[i] = 1.0 / d;
    }
}

// Weights eta_l(r), l = 0..nmax-1, of the local part at source-target distance r in (0, delta):
//   u_l(t_n) = sum_l eta_l(r) sigma(t_{n-nmax+1+l})
//   eta_l(r) = (1/2pi) int_r^delta [1 - phi(tau)] a_l(tau) / sqrt(tau^2 - r^2) dtau        (Eq. local2)
// where a_l(tau) interpolates sigma(t_n - tau) from the nmax stored levels (Eq. sigInterp).
// On delay intervals [m dt, (m+1) dt] with m >= kLsIntervals, a_l is p-th order Lagrange
// interpolation from the p nearest levels (Sec. 6).  On the newest kLsIntervals intervals those p
// levels are one-sided and that stencil loses accuracy (Lebesgue constant ~6e3 for p = 20); there
// a_l(tau) is the band-limited least-squares interpolant over all nmax levels, given as Chebyshev
// series Cls[l][c] on [0, kLsIntervals dt]: the kernel's Chebyshev moments are accumulated over
// the quadrature nodes and contracted with Cls once per pair.
// The delay integral is split at the step grid; on each piece tau = r + s^2 (Sec. 6) removes the
// inverse square root; Gauss-Legendre panels (ng nodes) are graded geometrically towards s = 0,
// where 1/sqrt(s^2 + 2r) peaks for small r.
WFP_HD inline void eta_weights(double r, double dt, int W, int p, int nmax, const double* phicoef, const double* gx,
                               const double* gw, int ng, const double* wl, const double* Cls, double* eta) {
    for (int l = 0; l < nmax; l++) eta[l] = 0.0;
    const double delta = W * dt;
    if (!(r > 0.0) || !(r < delta)) return;
    const double c = sqrt(2.0 * r);
    const double inv_pi = 0.31830988618379067154;
    const double span = kLsIntervals * dt;
    double xi[kMaxP];
    double mom[kLsDeg + 1];
    for (int k = 0; k <= kLsDeg; k++) mom[k] = 0.0;
    bool used_ls = false;
    int m0 = (int)floor(r / dt);
    for (int m = m0; m < W; m++) {
        double ta = fmax(r, m * dt), tb = (m + 1) * dt;
        if (!(tb > ta)) continue;
        const bool ls = (m < kLsIntervals) && Cls != nullptr;
        used_ls = used_ls || ls;
        int k0 = nmax - 1 - m - p / 2;
        if (k0 > nmax - p) k0 = nmax - p;
        if (k0 < 0) k0 = 0;
        double sa = sqrt(fmax(0.0, ta - r)), sb = sqrt(tb - r);
        double hi = sb;
        for (int lev = 0; lev < 200; lev++) {
            double lo = 0.5 * hi;
            bool last = (lo <= sa) || (lo < 0.25 * c);
            if (last) lo = sa;
            double half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
            for (int q = 0; q < ng; q++) {
                double s = mid + half * gx[q];
                double tau = r + s * s;
                double ph = (tau <= 0.0) ? 0.0 : (tau >= delta ? 1.0 : cheb_phi(phicoef, 2.0 * tau / delta - 1.0));
                double wt = half * gw[q] * inv_pi * (1.0 - ph) / sqrt(s * s + 2.0 * r);
                if (ls) {
                    double x = 2.0 * tau / span - 1.0, t0 = 1.0, t1 = x;
                    mom[0] += wt;
                    mom[1] += wt * x;
                    for (int k = 2; k <= kLsDeg; k++) {
                        double t2 = 2.0 * x * t1 - t0;
                        mom[k] += wt * t2;
                        t0 = t1;
                        t1 = t2;
                    }
                } else {
                    double X = (nmax - 1) - tau / dt;
                    lagrange_eq(X, k0, p, wl, xi);
                    for (int i = 0; i < p; i++) eta[k0 + i] += wt * xi[i];
                }
            }
            if (last) break;
            hi = lo;
        }
    }
    if (used_ls)
        for (int l = 0; l < nmax; l++) {
            double a = 0.0;
            for (int k = 0; k <= kLsDeg; k++) a = fma(Cls[l * (kLsDeg + 1) + k], mom[k], a);
            eta[l] += a;
        }
}

// sin(k x)/k, continuous at k = 0
// Chebyshev table of the local weights.  On each delay interval r in [k dt, (k+1) dt], k >= 1, the
// weights are analytic in v = sqrt((k+1) dt - r) (the square-root behaviour where a quadrature
// sub-interval opens at r = (k+1) dt is absorbed by the variable), so a degree-kEtaChebDeg
// Chebyshev series in v per interval and level replaces the per-pair quadrature; r < dt (a
// logarithmic singularity at r = 0) keeps eta_weights.  tab[((k - 1) * nmax + l) * (D + 1) + d].
constexpr int kEtaChebDeg = 32;

WFP_HD inline void eta_from_table(double r, double dt, int W, int nmax, const double* tab, double* eta) {
    constexpr int N = kEtaChebDeg + 1;
    int k = (int)floor(r / dt);
    k = k < 1 ? 1 : (k > W - 1 ? W - 1 : k);
    const double v = sqrt(fmax(0.0, (k + 1) * dt - r));
    const double x = 2.0 * v / sqrt(dt) - 1.0;
    const double* t = tab + (size_t)(k - 1) * nmax * N;
    for (int l = 0; l < nmax; l++) {
        const double* c = t + (size_t)l * N;
        double b1 = 0.0, b2 = 0.0;
        for (int d = N - 1; d >= 1; d--) {
            const double b0 = fma(2.0 * x, b1, c[d] - b2);
            b2 = b1;
            b1 = b0;
        }
        eta[l] = fma(x, b1, c[0] - b2);
    }
}

WFP_HD inline double sin_over(double k, double x) {
    double a = k * x;
    if (fabs(a) < 1e-3) {
        double a2 = a * a;
        return x * (1.0 - a2 / 6.0 * (1.0 - a2 / 20.0));
    }
    return sin(a) / k;
}

// Near-history FIR taps at |k| = kappa (Lemma 4.2 and Eq. hggrid), dt folded in:
//   p_m  = dt int_0^dt sin(kappa (dt - s))/kappa Psi(s + m dt) ds,  q_m  = same with cos(kappa (dt - s)),
//   pA_m, qA_m with Psi_A in place of Psi, where
//   Psi(d)   = 2 cos(kappa d) phi'(d) + sin(kappa d)/kappa phi''(d),
//   Psi_A(d) = 2 cos(kappa (d + A+ - delta)) phi'(d) + sin(kappa (d + A+ - delta))/kappa phi''(d).
// The trapezoid rule on the step grid for F (Eq. alphakF) gives one tap per level m = 0..W-1.
// s nodes (sq, wq on [0, dt]) and phi', phi'' at s + m dt (f1, f2: [W][ngt]) are precomputed.
// rot = {cos(kappa dt), sin(kappa dt)/kappa, kappa sin(kappa dt)}.
// Tap writers: planar [p | q | pA | qA] (W each, FP64), or interleaved per level m: FP64
// {p, q, pA, qA}; FP32 hi/lo pairs (rounded value and its rounding residual) grouped by FIR.
struct TapsPlanar {
    double* t;
    int W;
    WFP_HD void operator()(int m, double p, double q, double pa, double qa) const {
        t[m] = p;
        t[W + m] = q;
        t[2 * W + m] = pa;
        t[3 * W + m] = qa;
    }
};
template <typename TT>
struct TapsInterleaved;
template <>
struct TapsInterleaved<double> {
    double* t;
    WFP_HD void operator()(int m, double p, double q, double pa, double qa) const {
        t[4 * m] = p;
        t[4 * m + 1] = q;
        t[4 * m + 2] = pa;
        t[4 * m + 3] = qa;
    }
};
template <>
struct TapsInterleaved<float> {
    float* t;
    // per level: {p, pA} hi, {p, pA} lo, {q, qA} hi, {q, qA} lo -- one float4 per FIR (h or g)
    WFP_HD void operator()(int m, double p, double q, double pa, double qa) const {
        const double v[4] = {p, pa, q, qa};
        for (int i = 0; i < 2; i++)
            for (int k = 0; k < 2; k++) {
                const double x = v[2 * i + k];
                const float hi = (float)x;
                t[8 * m + 4 * i + k] = hi;
                t[8 * m + 4 * i + 2 + k] = (float)(x - (double)hi);
            }
    }
};

// FP32 hi/lo pairs of p and q only (plans whose lag never activates): per level {p hi, p lo},
// {q hi, q lo} -- one float2 per FIR
struct TapsCompact {
    float* t;
    WFP_HD void operator()(int m, double p, double q, double, double) const {
        const double v[2] = {p, q};
        for (int i = 0; i < 2; i++) {
            const float hi = (float)v[i];
            t[4 * m + 2 * i] = hi;
            t[4 * m + 2 * i + 1] = (float)(v[i] - (double)hi);
        }
    }
};

template <typename Put>
WFP_HD inline void mode_taps(double kappa, double dt, int W, double lagshift, int ngt, const double* sq,
                             const double* wq, const double* f1, const double* f2, const Put& put, double* rot) {
    for (int m = 0; m < W; m++) {
        double P = 0, Q = 0, PA = 0, QA = 0;
        for (int q = 0; q < ngt; q++) {
            double s = sq[q], wgt = wq[q];
            double d = s + m * dt;
            double a1 = f1[m * ngt + q], a2 = f2[m * ngt + q];
            double sk = sin_over(kappa, dt - s), ck = cos(kappa * (dt - s));
            double psi = 2.0 * cos(kappa * d) * a1 + sin_over(kappa, d) * a2;
            double dA = d + lagshift;
            double psiA = 2.0 * cos(kappa * dA) * a1 + sin_over(kappa, dA) * a2;
            P += wgt * sk * psi;
            Q += wgt * ck * psi;
            PA += wgt * sk * psiA;
            QA += wgt * ck * psiA;
        }
        put(m, dt * P, dt * Q, dt * PA, dt * QA);
    }
    rot[0] = cos(kappa * dt);
    rot[1] = sin_over(kappa, dt);
    rot[2] = kappa * sin(kappa * dt);
}

}  // namespace wfp
