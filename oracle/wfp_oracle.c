/*
 * wfp_oracle.c -- plain, slow, FP64 CPU oracle for the 2D free-space wave field
 * radiated by point sources (Al Hassanieh, Greengard & Barnett, "A spectral method
 * for the rapid evaluation of hyperbolic potentials in two dimensions using
 * windowed Fourier projection").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * helper with the CUDA path; it carries its own Gauss-Legendre rule, its own
 * Bessel I0 and its own blending function.
 *
 * What it computes (all in the caller's units, unit wave speed):
 *
 *   u(x,t) = sum_j int_0^t G(x - y_j, t - tau) sigma_j(tau) dtau,         (Sec. 1, Eq. solnRep)
 *   G(x,t) = H(t - |x|) / (2 pi sqrt(t^2 - |x|^2))                        (Eq. Green)
 *
 * evaluated, as the paper does for its own error checks (Sec. 7, Eq. exactSol),
 * through the substitution tau' = r + s^2 of the delay, which removes the inverse
 * square-root singularity on the light cone:
 *
 *   u(x,t) = (1/pi) sum_{j: 0 < r_j < t} int_0^{sqrt(t - r_j)}
 *                 sigma_j(t - r_j - s^2) / sqrt(s^2 + 2 r_j) ds .
 *
 * Coincident pairs (r_j <= r_coinc) are excluded, as in Eq. exactSol.
 *
 * A second, independent quadrature of the same integral uses the substitution
 * d = r cosh(theta) of the delay (the form the paper uses for tiny r in Sec. 6):
 *
 *   u(x,t) = (1/(2 pi)) sum_j int_0^{acosh(t/r_j)} sigma_j(t - r_j cosh theta) dtheta .
 *
 * Component oracles weight the delay integral by the blending functions of the
 * three-way split (Sec. 3, Eqs. ul, unh, ufh), with the temporal blending function
 * phi of Eq. KBblending:
 *     LOCAL : 1 - phi(d)              (0 <= d <= delta)
 *     NEAR  : phi(d) phi(A+ - d)      (0 <= d <= A+)
 *     FAR   : 1 - phi(A+ - d)         (d >= A+ - delta)
 * The spatial truncation phi_Delta(A - r) of the far kernel (Eq. TKdef) equals 1
 * for every source-target distance inside the computational domain, so FAR uses
 * the untruncated kernel.  The three weights sum to 1 for every delay when
 * A+ >= 2 delta.
 *
 * The self term of a coincident source/target pair is the part of the history
 * field that the Fourier representation carries at r = 0 (G(0,d) = 1/(2 pi d)):
 *     u_self(t) = (1/(2 pi)) int_0^t phi(d) sigma(t - d) / d dd .
 *
 * Signals sigma_j are analytic (evaluated at any time), zero for t <= 0:
 *   family 0 (GAUSS3): sum_{q=1..3} a_q exp(-(t-c_q)^2/(2 s^2)) sin(w (t - c_q))
 *                      params [a1 a2 a3 c1 c2 c3 s w]
 *   family 1 (ERF)   : 0.5 (erf(5 (t - t0)) + 1) sin(w (t - t0))   (Sec. 7, Eq. exampleDensities)
 *                      params [t0 w]
 *   family 2 (POLY)  : p0 + p1 t + p2 t^2 (t > 0), params [p0 p1 p2]; used only for closed-form checks.
 *
 * Quadrature: composite Gauss-Legendre, panels uniform in the delay d of width at
 * most half a carrier period (and half the envelope scale), restricted to each
 * pulse's support (|t - d - c_q| <= 8.5 s, outside which the Gaussian is below
 * 2e-16), with geometric refinement towards s = 0 where the factor
 * 1/sqrt(s^2 + 2r) peaks for small r.  Sums over sources are plain FP64 sums.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NPAR 8
#define NGL 20
#define NGL_HI 40

/* ---------------------------------------------------------------- GL rule */
/* Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_n. */
static void gl_rule(int n, double* x, double* w) {
    for (int i = 0; i < n; i++) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double pp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; k++) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            pp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute derivative at the converged node */
        double p0 = 1.0, p1 = 0.0;
        for (int k = 1; k <= n; k++) {
            double p2 = p1;
            p1 = p0;
            p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
        }
        pp = n * (z * p0 - p1) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

static double GX[NGL_HI], GW[NGL_HI];
static int g_n = 0;
static double g_hfac = 0.5;

static void ensure_rule(int n) {
    if (g_n != n) {
        gl_rule(n, GX, GW);
        g_n = n;
    }
}

/* -------------------------------------------------------------- signals */
double wfo_sigma(int fam, const double* p, double t) {
    if (!(t > 0.0)) return 0.0;
    switch (fam) {
        case 0: {
            double s = p[6], w = p[7], v = 0.0;
            for (int q = 0; q < 3; q++) {
                double z = t - p[3 + q];
                v += p[q] * exp(-z * z / (2.0 * s * s)) * sin(w * z);
            }
            return v;
        }
        case 1:
            return 0.5 * (erf(5.0 * (t - p[0])) + 1.0) * sin(p[1] * (t - p[0]));
        case 2:
            return p[0] + t * (p[1] + t * p[2]);
        default:
            return 0.0;
    }
}

/* One smooth piece of a signal: support [lo, hi] in emission time, feature scale. */
typedef struct {
    int fam;
    const double* p;
    int q;          /* pulse index for GAUSS3, -1 = whole signal */
    double lo, hi;  /* support in emission time tau */
    double scale;   /* panel width cap in delay */
} piece_t;

static double piece_eval(const piece_t* pc, double tau) {
    if (!(tau > 0.0)) return 0.0;
    if (pc->fam == 0 && pc->q >= 0) {
        double z = tau - pc->p[3 + pc->q], s = pc->p[6];
        return pc->p[pc->q] * exp(-z * z / (2.0 * s * s)) * sin(pc->p[7] * z);
    }
    return wfo_sigma(pc->fam, pc->p, tau);
}

static int signal_pieces(int fam, const double* p, piece_t* out) {
    if (fam == 0) {
        double s = p[6], w = fabs(p[7]);
        double per = (w > 0) ? 2.0 * M_PI / w : 1e30;
        double sc = fmin(per, 2.0 * s);
        for (int q = 0; q < 3; q++) {
            out[q].fam = 0;
            out[q].p = p;
            out[q].q = q;
            out[q].lo = fmax(0.0, p[3 + q] - 8.5 * s);
            out[q].hi = p[3 + q] + 8.5 * s;
            out[q].scale = sc;
        }
        return 3;
    }
    if (fam == 1) {
        /* the switch-on 0.5 (erf(5 z) + 1) rises with derivative (5/sqrt(pi)) exp(-25 z^2), a Gaussian
         * of standard deviation s = 1/(5 sqrt 2): the same cap min(period, 2 s) as the Gaussian pulses */
        double w = fabs(p[1]);
        double per = (w > 0) ? 2.0 * M_PI / w : 1e30;
        out[0].fam = 1;
        out[0].p = p;
        out[0].q = -1;
        out[0].lo = 0.0;
        out[0].hi = 1e300;
        out[0].scale = fmin(per, 2.0 / (5.0 * sqrt(2.0)));
        return 1;
    }
    out[0].fam = fam;
    out[0].p = p;
    out[0].q = -1;
    out[0].lo = 0.0;
    out[0].hi = 1e300;
    out[0].scale = 1.0;
    return 1;
}

/* ------------------------------------------------- Bessel I0 and blending */
/* I0 by its power series sum_k (x/2)^{2k} / (k!)^2; all terms positive, so the
 * partial sums are accurate to rounding for the arguments used here (x <= 60). */
double wfo_i0(double x) {
    double q = 0.25 * x * x, term = 1.0, sum = 1.0;
    for (int k = 1; k < 500; k++) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

/* phi'_delta(t) = b / (delta sinh b) I0(b sqrt(1 - (2t/delta - 1)^2)) on [0, delta] (Eq. KBblending). */
double wfo_dphi(double t, double delta, double b) {
    if (t < 0.0 || t > delta) return 0.0;
    double z = 2.0 * t / delta - 1.0;
    double a = 1.0 - z * z;
    if (a < 0) a = 0;
    return b / (delta * sinh(b)) * wfo_i0(b * sqrt(a));
}

/* phi_delta(t) = int_0^t phi'_delta, by composite 20-point GL on 16 panels. */
static double PX[NGL], PW[NGL];
static int p_init = 0;

static void ensure_phi_rule(void) {
    if (!p_init) {
        gl_rule(NGL, PX, PW);
        p_init = 1;
    }
}

double wfo_phi(double t, double delta, double b) {
    if (t <= 0.0) return 0.0;
    if (t >= delta) return 1.0;
    ensure_phi_rule();
    const double* x = PX;
    const double* w = PW;
    const int np = 16;
    double h = t / np, sum = 0.0;
    for (int k = 0; k < np; k++) {
        double a = k * h;
        for (int i = 0; i < NGL; i++) {
            double tt = a + 0.5 * h * (x[i] + 1.0);
            sum += 0.5 * h * w[i] * wfo_dphi(tt, delta, b);
        }
    }
    return sum;
}

/* ------------------------------------------------------------ weights */
enum { K_FULL = 0, K_LOCAL = 1, K_NEAR = 2, K_FAR = 3 };

typedef struct {
    int kind;
    double delta, Aplus, b;
} wparam_t;

static double weight(const wparam_t* wp, double d) {
    switch (wp->kind) {
        case K_LOCAL:
            return (d >= wp->delta) ? 0.0 : 1.0 - wfo_phi(d, wp->delta, wp->b);
        case K_NEAR:
            if (d >= wp->Aplus) return 0.0;
            return wfo_phi(d, wp->delta, wp->b) * wfo_phi(wp->Aplus - d, wp->delta, wp->b);
        case K_FAR:
            if (d <= wp->Aplus - wp->delta) return 0.0;
            return 1.0 - wfo_phi(wp->Aplus - d, wp->delta, wp->b);
        default:
            return 1.0;
    }
}

/* delay interval [lo, hi] where the weight can be nonzero */
static void weight_support(const wparam_t* wp, double* lo, double* hi) {
    *lo = 0.0;
    *hi = 1e300;
    if (wp->kind == K_LOCAL) *hi = wp->delta;
    if (wp->kind == K_NEAR) *hi = wp->Aplus;
    if (wp->kind == K_FAR) *lo = wp->Aplus - wp->delta;
}

/* breakpoints of the weight (transition regions are refined to delta/16) */
static int weight_breaks(const wparam_t* wp, double* br) {
    int n = 0;
    if (wp->kind == K_FULL) return 0;
    double a[2] = {0.0, wp->Aplus - wp->delta};
    int na = (wp->kind == K_LOCAL) ? 1 : (wp->kind == K_FAR ? 1 : 2);
    int off = (wp->kind == K_FAR) ? 1 : 0;
    for (int k = 0; k < na; k++) {
        double s0 = a[k + off];
        for (int i = 0; i <= 16; i++) br[n++] = s0 + wp->delta * i / 16.0;
    }
    return n;
}

/* ---------------------------------------------- s-substitution quadrature */
/* (1/pi) int over s in [sa, sb] of f(t - r - s^2) W(r + s^2) / sqrt(s^2 + 2r) */
static double s_panel(const piece_t* pc, const wparam_t* wp, double t, double r, double sa, double sb) {
    double sum = 0.0, h = 0.5 * (sb - sa), m = 0.5 * (sb + sa);
    for (int i = 0; i < g_n; i++) {
        double s = m + h * GX[i];
        double d = r + s * s;
        double f = piece_eval(pc, t - d);
        if (f != 0.0) {
            double wgt = weight(wp, d);
            sum += GW[i] * f * wgt / sqrt(s * s + 2.0 * r);
        }
    }
    return h * sum;
}

static int cmpd(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x < y) ? -1 : (x > y);
}

/* integral over delay d in [dlo, dhi] (dlo >= r) for one piece, one pair */
static double pair_piece_s(const piece_t* pc, const wparam_t* wp, double t, double r) {
    double dlo = fmax(r, t - pc->hi), dhi = fmin(t, t - pc->lo);
    double wl, wh;
    weight_support(wp, &wl, &wh);
    dlo = fmax(dlo, wl);
    dhi = fmin(dhi, wh);
    if (!(dhi > dlo)) return 0.0;
    double h = g_hfac * pc->scale;
    int np = (int)ceil((dhi - dlo) / h);
    if (np < 1) np = 1;
    /* breakpoints in d: uniform panels plus the weight's transition breakpoints */
    int cap = np + 1 + 40;
    double* br = (double*)malloc(sizeof(double) * cap);
    int nb = 0;
    for (int k = 0; k <= np; k++) br[nb++] = dlo + (dhi - dlo) * k / np;
    double wb[40];
    int nw = weight_breaks(wp, wb);
    for (int k = 0; k < nw; k++)
        if (wb[k] > dlo && wb[k] < dhi) br[nb++] = wb[k];
    qsort(br, nb, sizeof(double), cmpd);
    double total = 0.0;
    for (int k = 0; k + 1 < nb; k++) {
        double da = br[k], db = br[k + 1];
        if (!(db > da)) continue;
        double sa = sqrt(fmax(0.0, da - r)), sb = sqrt(db - r);
        double c = sqrt(2.0 * r);
        if (sa == 0.0 && sb > 0.25 * c) {
            /* geometric refinement towards s = 0 where 1/sqrt(s^2+2r) peaks */
            double hi = sb;
            int lev = 0;
            while (hi > 0.25 * c && lev < 80) {
                double lo = 0.5 * hi;
                total += s_panel(pc, wp, t, r, lo, hi);
                hi = lo;
                lev++;
            }
            total += s_panel(pc, wp, t, r, 0.0, hi);
        } else {
            total += s_panel(pc, wp, t, r, sa, sb);
        }
    }
    free(br);
    return total / M_PI;
}

/* -------------------------------------------- cosh-substitution quadrature */
/* (1/(2pi)) int over theta of f(t - r cosh theta) W(r cosh theta) */
static double pair_piece_cosh(const piece_t* pc, const wparam_t* wp, double t, double r) {
    double dlo = fmax(r, t - pc->hi), dhi = fmin(t, t - pc->lo);
    double wl, wh;
    weight_support(wp, &wl, &wh);
    dlo = fmax(dlo, wl);
    dhi = fmin(dhi, wh);
    if (!(dhi > dlo)) return 0.0;
    double h = g_hfac * pc->scale;
    int np = (int)ceil((dhi - dlo) / h);
    if (np < 1) np = 1;
    double total = 0.0;
    for (int k = 0; k < np; k++) {
        double da = dlo + (dhi - dlo) * k / np, db = dlo + (dhi - dlo) * (k + 1) / np;
        double ta = acosh(fmax(1.0, da / r)), tb = acosh(db / r);
        int nsub = (int)ceil((tb - ta) / 0.5);
        if (nsub < 1) nsub = 1;
        for (int u = 0; u < nsub; u++) {
            double a = ta + (tb - ta) * u / nsub, b2 = ta + (tb - ta) * (u + 1) / nsub;
            double hh = 0.5 * (b2 - a), m = 0.5 * (b2 + a), sum = 0.0;
            for (int i = 0; i < g_n; i++) {
                double th = m + hh * GX[i];
                double d = r * cosh(th);
                double f = piece_eval(pc, t - d);
                if (f != 0.0) sum += GW[i] * f * weight(wp, d);
            }
            total += hh * sum;
        }
    }
    return total / (2.0 * M_PI);
}

/* ------------------------------------------------------------- drivers */
static int g_threads = 0;

int wfo_set_threads(int n) {
    g_threads = n;
    return 0;
}

int wfo_num_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/* Quadrature resolution: nodes per panel (20 or 40) and the panel-width factor
 * (fraction of the feature scale).  Used by the self-checks that double the work. */
int wfo_set_resolution(int nodes, double hfac) {
    if (nodes != NGL && nodes != NGL_HI) return -1;
    ensure_rule(nodes);
    g_hfac = hfac;
    return 0;
}

/*
 * Field at n_eval (x, y, t) triples from M sources.
 *   fam      signal family (all sources share it)
 *   src_xy   2*M coordinates (interleaved)
 *   par      NPAR*M signal parameters
 *   eval_xyt 3*n_eval (x, y, t)
 *   kind     0 FULL, 1 LOCAL, 2 NEAR, 3 FAR
 *   delta, Aplus, b  blending parameters (ignored for FULL)
 *   method   0 = s-substitution (Eq. exactSol), 1 = cosh substitution
 *   r_coinc  pairs with r <= r_coinc are excluded
 *   out      n_eval values
 */
int wfo_field(int fam, int M, const double* src_xy, const double* par, int n_eval, const double* eval_xyt,
              int kind, double delta, double Aplus, double b, int method, double r_coinc, double* out) {
    if (g_n == 0) ensure_rule(NGL);
    ensure_phi_rule();
    wparam_t wp = {kind, delta, Aplus, b};
#ifdef _OPENMP
    int nth = wfo_num_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth)
#endif
    for (int e = 0; e < n_eval; e++) {
        double x = eval_xyt[3 * e], y = eval_xyt[3 * e + 1], t = eval_xyt[3 * e + 2];
        double acc = 0.0;
        for (int j = 0; j < M; j++) {
            double dx = x - src_xy[2 * j], dy = y - src_xy[2 * j + 1];
            double r = sqrt(dx * dx + dy * dy);
            if (r <= r_coinc || !(r < t)) continue;
            piece_t pcs[3];
            int np = signal_pieces(fam, par + (size_t)NPAR * j, pcs);
            for (int q = 0; q < np; q++)
                acc += (method == 0) ? pair_piece_s(&pcs[q], &wp, t, r) : pair_piece_cosh(&pcs[q], &wp, t, r);
        }
        out[e] = acc;
    }
    return 0;
}

/*
 * Self term at coincident pairs: u_self(t) = (1/(2 pi)) int_0^t phi(d) sigma(t - d) / d dd,
 * for n_eval (signal, time) pairs.  par: NPAR*n_eval, times: n_eval.
 */
int wfo_self(int fam, int n_eval, const double* par, const double* times, double delta, double b, double* out) {
    if (g_n == 0) ensure_rule(NGL);
    ensure_phi_rule();
#ifdef _OPENMP
    int nth = wfo_num_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth)
#endif
    for (int e = 0; e < n_eval; e++) {
        double t = times[e];
        piece_t pcs[3];
        int np = signal_pieces(fam, par + (size_t)NPAR * e, pcs);
        double acc = 0.0;
        for (int q = 0; q < np; q++) {
            double dlo = fmax(0.0, t - pcs[q].hi), dhi = fmin(t, t - pcs[q].lo);
            if (!(dhi > dlo)) continue;
            double h = g_hfac * pcs[q].scale;
            /* breakpoints: uniform panels plus delta/16 refinement of [0, delta] */
            int npn = (int)ceil((dhi - dlo) / h);
            if (npn < 1) npn = 1;
            double* br = (double*)malloc(sizeof(double) * (npn + 20));
            int nb = 0;
            for (int k = 0; k <= npn; k++) br[nb++] = dlo + (dhi - dlo) * k / npn;
            for (int i = 1; i <= 16; i++) {
                double v = delta * i / 16.0;
                if (v > dlo && v < dhi) br[nb++] = v;
            }
            qsort(br, nb, sizeof(double), cmpd);
            for (int k = 0; k + 1 < nb; k++) {
                double a = br[k], c = br[k + 1];
                if (!(c > a)) continue;
                double hh = 0.5 * (c - a), m = 0.5 * (c + a), sum = 0.0;
                for (int i = 0; i < g_n; i++) {
                    double d = m + hh * GX[i];
                    double f = piece_eval(&pcs[q], t - d);
                    if (f != 0.0) sum += GW[i] * f * wfo_phi(d, delta, b) / d;
                }
                acc += hh * sum;
            }
            free(br);
        }
        out[e] = acc / (2.0 * M_PI);
    }
    return 0;
}

/* Gauss-Legendre rule export, for the oracle's own self-checks. */
int wfo_gl_rule(int n, double* x, double* w) {
    if (n < 1 || n > 200) return -1;
    gl_rule(n, x, w);
    return 0;
}
