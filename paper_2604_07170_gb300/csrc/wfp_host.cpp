// Host-side parameter selection and plan-time quadrature helpers of the 2D TK-WFP evaluator.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "wfp_internal.h"

namespace wfp {

static thread_local std::string g_last_error;

void set_error(const std::string& s) { g_last_error = s; }
const char* last_error_cstr() { return g_last_error.c_str(); }

// Gauss-Legendre rule on [-1,1]: Newton iteration on the Legendre three-term recurrence.
void gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; i++) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; k++) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            double dp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = 0.0;
        for (int k = 1; k <= n; k++) {
            double p2 = p1;
            p1 = p0;
            p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
        }
        double dp = n * (z * p0 - p1) / (z * z - 1.0);
        x[n - 1 - i] = z;  // ascending order
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// ---------------------------------------------------------------- blending function
// phi'_delta(t) = b/(delta sinh b) I0(b sqrt(1 - (2t/delta - 1)^2)) on [0, delta]   (Eq. KBblending)
double dphi_host(double t, double delta, double b) {
    if (t < 0.0 || t > delta) return 0.0;
    double x = 2.0 * t / delta - 1.0;
    double a = std::max(0.0, 1.0 - x * x);
    return b / (delta * std::sinh(b)) * std::cyl_bessel_i(0.0, b * std::sqrt(a));
}

// phi'' = b/(delta sinh b) * d/dt I0(z),  z = b sqrt(1-x^2):  dI0/dt = -(2 b^2 x / delta) I1(z)/z
double d2phi_host(double t, double delta, double b) {
    if (t < 0.0 || t > delta) return 0.0;
    double x = 2.0 * t / delta - 1.0;
    double a = std::max(0.0, 1.0 - x * x);
    double z = b * std::sqrt(a);
    double i1z = (z > 1e-8) ? std::cyl_bessel_i(1.0, z) / z : 0.5 + z * z / 16.0;
    return b / (delta * std::sinh(b)) * (-2.0 * b * b * x / delta) * i1z;
}

// F(x) = int_{-1}^{x} (b / (2 sinh b)) I0(b sqrt(1 - y^2)) dy, so phi_delta(t) = F(2t/delta - 1).
// Tabulated as kPhiPanels Chebyshev interpolants of degree kPhiDeg; the values at the
// Chebyshev points come from composite Gauss-Legendre quadrature of the Kaiser-Bessel bump.
void build_phi_table(double b, std::vector<double>& coef) {
    coef.assign((size_t)kPhiPanels * (kPhiDeg + 1), 0.0);
    build_phi_table_into(b, coef.data());
}

void build_phi_table_into(double b, double* coef) {
    const int np = kPhiPanels, deg = kPhiDeg, ng = 30;
    double gx[ng], gw[ng];
    gauss_legendre(ng, gx, gw);
    auto bump = [&](double y) {
        double a = std::max(0.0, 1.0 - y * y);
        return b / (2.0 * std::sinh(b)) * std::cyl_bessel_i(0.0, b * std::sqrt(a));
    };
    // integral of the bump over [lo, hi] (composite: 4 sub-panels)
    auto integ = [&](double lo, double hi) {
        double s = 0.0;
        const int ns = 4;
        for (int k = 0; k < ns; k++) {
            double a = lo + (hi - lo) * k / ns, c = lo + (hi - lo) * (k + 1) / ns;
            for (int i = 0; i < ng; i++) s += 0.5 * (c - a) * gw[i] * bump(0.5 * (c - a) * gx[i] + 0.5 * (c + a));
        }
        return s;
    };
    double base = 0.0;  // F at the panel's left end
    for (int k = 0; k < np; k++) {
        double xl = -1.0 + 2.0 * k / np, xr = -1.0 + 2.0 * (k + 1) / np;
        double f[kPhiDeg + 1];
        for (int j = 0; j <= deg; j++) {
            double sj = std::cos(kPi * (j + 0.5) / (deg + 1));  // Chebyshev points of the first kind
            double xx = 0.5 * (xr - xl) * sj + 0.5 * (xr + xl);
            f[j] = base + integ(xl, xx);
        }
        for (int m = 0; m <= deg; m++) {
            double c = 0.0;
            for (int j = 0; j <= deg; j++) c += f[j] * std::cos(m * kPi * (j + 0.5) / (deg + 1));
            coef[(size_t)k * (deg + 1) + m] = c * (m == 0 ? 1.0 : 2.0) / (deg + 1);
        }
        base += integ(xl, xr);
    }
}

double phi_host(const double* coef, double t, double delta) {
    if (t <= 0.0) return 0.0;
    if (t >= delta) return 1.0;
    return cheb_phi(coef, 2.0 * t / delta - 1.0);
}

// One-sided Jacobi SVD of the m x n (m >= n) column-major matrix A: on return the columns of A
// are s_j u_j, V (n x n, column-major) holds the right singular vectors and s the singular values.
static void jacobi_svd(int m, int n, double* A, double* V, double* s) {
    for (int i = 0; i < n * n; i++) V[i] = 0.0;
    for (int j = 0; j < n; j++) V[(size_t)j * n + j] = 1.0;
    for (int sweep = 0; sweep < 80; sweep++) {
        int rotated = 0;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                double al = 0, be = 0, ga = 0;
                for (int i = 0; i < m; i++) {
                    double x = A[(size_t)p * m + i], y = A[(size_t)q * m + i];
                    al += x * x;
                    be += y * y;
                    ga += x * y;
                }
                if (std::fabs(ga) <= 1e-16 * std::sqrt(al * be) || ga == 0.0) continue;
                rotated++;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
                for (int i = 0; i < m; i++) {
                    double x = A[(size_t)p * m + i], y = A[(size_t)q * m + i];
                    A[(size_t)p * m + i] = c * x - sn * y;
                    A[(size_t)q * m + i] = sn * x + c * y;
                }
                for (int i = 0; i < n; i++) {
                    double x = V[(size_t)p * n + i], y = V[(size_t)q * n + i];
                    V[(size_t)p * n + i] = c * x - sn * y;
                    V[(size_t)q * n + i] = sn * x + c * y;
                }
            }
        if (!rotated) break;
    }
    for (int j = 0; j < n; j++) {
        double t = 0;
        for (int i = 0; i < m; i++) t += A[(size_t)j * m + i] * A[(size_t)j * m + i];
        s[j] = std::sqrt(t);
    }
}

// Band-limited least-squares interpolation weights a_l(tau), l = 0..nmax-1, for sigma(t_n - tau)
// from the levels t_l = -(nmax-1-l) dt, tau in [0, span]:
//   a(tau) = argmin int_0^Omega |sum_l a_l e^{i w t_l} - e^{-i w tau}|^2 dw + mu Omega |a|^2,
// discretised with Gauss-Legendre nodes in w and solved through the SVD of the real (cos, sin)
// design matrix (condition ~ sqrt of the normal equations').  Returned as Chebyshev coefficients
// C[l][c], c = 0..kLsDeg, of a_l on [0, span].
void build_ls_cheb(int nmax, double dt, double Omega, double span, std::vector<double>& C) {
    C.assign((size_t)nmax * (kLsDeg + 1), 0.0);
    build_ls_cheb_into(nmax, dt, Omega, span, C.data());
}

void build_ls_cheb_into(int nmax, double dt, double Omega, double span, double* C) {
    constexpr int Q = 96, m = 2 * Q, deg = kLsDeg;
    const int n = nmax;
    const double mu = 1e-16;
    double gx[Q], gw[Q], om[Q], sw[Q];
    gauss_legendre(Q, gx, gw);
    for (int q = 0; q < Q; q++) {
        om[q] = 0.5 * Omega * (gx[q] + 1.0);
        sw[q] = std::sqrt(0.5 * Omega * gw[q]);
    }
    // fixed-size work arrays (nmax <= kMaxLevels): no heap allocation
    static_assert(kMaxLevels <= 64, "work arrays sized for 64 levels");
    double A[m * kMaxLevels], V[kMaxLevels * kMaxLevels], s[kMaxLevels];
    for (int l = 0; l < n; l++) {
        double tl = -(double)(n - 1 - l) * dt;
        for (int q = 0; q < Q; q++) {
            A[(size_t)l * m + q] = sw[q] * std::cos(om[q] * tl);
            A[(size_t)l * m + Q + q] = sw[q] * std::sin(om[q] * tl);
        }
    }
    jacobi_svd(m, n, A, V, s);
    const double reg = mu * Omega;
    double av[(kLsDeg + 1) * kMaxLevels], b[m];
    for (int c = 0; c <= deg; c++) {
        double x = std::cos(kPi * (c + 0.5) / (deg + 1));
        double tau = 0.5 * span * (x + 1.0);
        for (int q = 0; q < Q; q++) {
            b[q] = sw[q] * std::cos(om[q] * tau);
            b[Q + q] = -sw[q] * std::sin(om[q] * tau);
        }
        for (int l = 0; l < n; l++) av[(size_t)c * n + l] = 0.0;
        for (int j = 0; j < n; j++) {
            double proj = 0;  // (s_j u_j)^T b
            for (int i = 0; i < m; i++) proj += A[(size_t)j * m + i] * b[i];
            double f = proj / (s[j] * s[j] + reg);
            for (int l = 0; l < n; l++) av[(size_t)c * n + l] += V[(size_t)j * n + l] * f;
        }
    }
    for (int l = 0; l < n; l++)
        for (int k = 0; k <= deg; k++) {
            double t = 0;
            for (int c = 0; c <= deg; c++) t += av[(size_t)c * n + l] * std::cos(k * kPi * (c + 0.5) / (deg + 1));
            C[(size_t)l * (deg + 1) + k] = t * (k == 0 ? 1.0 : 2.0) / (deg + 1);
        }
}

// ---------------------------------------------------------------- sum of exponentials
void soe_nodes(double lam_max, int panels, int ng, std::vector<double>& lam, std::vector<double>& q) {
    std::vector<double> gx(ng), gw(ng);
    gauss_legendre(ng, gx.data(), gw.data());
    lam.clear();
    q.clear();
    for (int k = 0; k < panels; k++) {
        // panel k: [lo, hi]; k = 0 is [0, lmax/2^(panels-1)]
        double hi = lam_max / std::ldexp(1.0, panels - 1 - k);
        double lo = (k == 0) ? 0.0 : 0.5 * hi;
        for (int i = 0; i < ng; i++) {
            lam.push_back(0.5 * (hi - lo) * gx[i] + 0.5 * (hi + lo));
            q.push_back(0.5 * (hi - lo) * gw[i]);
        }
    }
}

// Sum of exponentials for 1/d on [dlo, T] (r = 0) from 1/d = int_0^inf exp(-lambda d) dlambda, split
// at lc (a few times 1/T).  Below lc the integrand is an entire function of lambda with d lc of order
// one for every d <= T, so n0-point Gauss-Legendre in lambda resolves it: these few terms stand in for
// the many slowly decaying terms a rule in ln(lambda) would spend there.  Above lc the integrand
// exp(s - e^s d) in s = ln(lambda) is analytic in the strip |Im s| < pi/2; composite Gauss-Legendre in
// s (panels of equal width <= ds, n1 nodes each) over [ln lc, ln lmax].  Beyond lmax the dropped tail
// is exp(-lmax d) / d.  The caller checks the sum against 1/d before using it.
void soe_inverse(double lc, int n0, double lmax, double ds, int n1, std::vector<double>& lam,
                 std::vector<double>& q) {
    lam.clear();
    q.clear();
    std::vector<double> gx(std::max(n0, n1)), gw(gx.size());
    gauss_legendre(n0, gx.data(), gw.data());
    for (int i = 0; i < n0; i++) {
        lam.push_back(0.5 * lc * (gx[i] + 1.0));
        q.push_back(0.5 * lc * gw[i]);
    }
    const double s0 = std::log(lc), s1 = std::max(std::log(lmax), s0 + 1.0);
    const int P = std::max(1, (int)std::ceil((s1 - s0) / ds));
    const double hs = (s1 - s0) / P;
    gauss_legendre(n1, gx.data(), gw.data());
    for (int pnl = 0; pnl < P; pnl++)
        for (int i = 0; i < n1; i++) {
            const double sv = s0 + hs * (pnl + 0.5 * (gx[i] + 1.0));
            lam.push_back(std::exp(sv));
            q.push_back(0.5 * hs * gw[i] * std::exp(sv));
        }
}

// The self term's sum of exponentials for 1/d on [dlo, T]: soe_inverse with lc = 8 / T and lmax =
// (ln(1/eps) + 3) / dlo (dropped tail below e^-3 eps), the fewest terms over the node counts and
// panel widths tried whose relative error on [dlo, T] is within 0.8 eps.  Each term costs the self
// term two FP64 FMAs per coincident target and step.  False if none meets the tolerance.
bool self_soe(double dlo, double T, double eps, std::vector<double>& lam, std::vector<double>& q) {
    lam.clear();
    q.clear();
    std::vector<double> tl, tq;
    const double lmax = (std::log(1.0 / eps) + 3.0) / dlo;
    bool ok = false;
    for (int n0 : {8, 10, 12, 14, 16})
        for (double ds : {2.0, 3.0, 4.0})
            for (int n1 = 6; n1 <= 24; n1++) {
                soe_inverse(8.0 / T, n0, lmax, ds, n1, tl, tq);
                if (ok && tl.size() >= lam.size()) continue;
                if (soe_max_rel_error(tl, tq, 0.0, dlo, T) <= 0.8 * eps) {
                    lam.swap(tl);
                    q.swap(tq);
                    ok = true;
                }
            }
    return ok;
}

double soe_max_rel_error(const std::vector<double>& lam, const std::vector<double>& q, double rmax, double tlo,
                         double thi) {
    double worst = 0.0;
    const int nr = (rmax > 0) ? 24 : 1, nt = 160;
    const size_t nl = lam.size();
    std::vector<double> qi(nl);
    for (int ir = 0; ir < nr; ir++) {
        double r = (nr == 1) ? 0.0 : rmax * ir / (nr - 1);
        // q_l I0(r lam_l) e^{-r lam_l}, so that each term is q_l [I0 e^{-r lam}] e^{-lam (t - r)}
        for (size_t l = 0; l < nl; l++) {
            double x = r * lam[l];
            qi[l] = q[l] * ((x < 700.0) ? std::cyl_bessel_i(0.0, x) * std::exp(-x) : 1.0 / std::sqrt(2 * kPi * x));
        }
        for (int it = 0; it < nt; it++) {
            double t = tlo * std::pow(thi / tlo, (double)it / (nt - 1));  // geometric sampling
            if (t <= r) continue;
            double s = 0.0;
            for (size_t l = 0; l < nl; l++) s += qi[l] * std::exp(-lam[l] * (t - r));
            double ex = 1.0 / std::sqrt(t * t - r * r);
            worst = std::max(worst, std::fabs(s - ex) / ex);
        }
    }
    return worst;
}

// ---------------------------------------------------------------- spreading kernel transform
// psihat(n) = int psi(x) e^{i n x} dx over |x| <= w h / 2, psi(x) = es_kernel(2x/(w h), beta).
void es_kernel_ft(int w, double beta, double h, int nmax, std::vector<double>& out) {
    const int ng = 200;
    std::vector<double> gx(ng), gw(ng);
    gauss_legendre(ng, gx.data(), gw.data());
    double half = 0.5 * w * h;
    out.assign(nmax + 1, 0.0);
    for (int n = 0; n <= nmax; n++) {
        double s = 0.0;
        for (int i = 0; i < ng; i++) s += gw[i] * es_kernel(gx[i], beta) * std::cos(n * half * gx[i]);
        out[n] = half * s;
    }
}

// ---------------------------------------------------------------- parameters
// FFT-friendly grid size: the smallest 2^a, 3 * 2^a or 9 * 2^a at or above n (cuFFT runs these
// sizes markedly faster than sizes with factors 5 or 7 in double precision)
static int next_fft_size(int n) {
    int best = 1 << 30;
    for (int f : {1, 3, 9}) {
        int m = f * 2;
        while (m < n) m *= 2;
        best = std::min(best, m);
    }
    return best;
}

wfp_status local_params(double dt, double K0, double tol, const wfp_opts& o, double* eps, int* W, int* p, int* nmax,
                        const char** why) {
    *why = "";
    if (!(dt > 0) || !std::isfinite(dt)) {
        *why = "dt must be positive and finite";
        return WFP_EINVAL;
    }
    if (!(K0 >= 0) || !std::isfinite(K0)) {
        *why = "band_limit must be >= 0 and finite";
        return WFP_EINVAL;
    }
    if (!(tol > 0 && tol < 1)) {
        *why = "tol must be in (0, 1)";
        return WFP_EINVAL;
    }
    // the history parts carry absolute errors ~eps |sigma|, which must stay below tol times the
    // smallest per-step field norm of interest (tail steps of a pulse are ~1e-2 of the peak)
    double e = (o.eps > 0) ? o.eps : tol / 1000.0;
    if (!(e > 0 && e < 1)) {
        *why = "eps must be in (0, 1)";
        return WFP_EINVAL;
    }
    double b = std::log(1.0 / e);
    double K0dt = K0 * dt;  // scale-free
    if (!(K0dt < kPi)) {
        *why = "band_limit * dt must be below pi (Eq. dt)";
        return WFP_EINVAL;
    }
    // Eq. dt: dt <= (pi - 2b/W)/K0  <=>  W >= 2b / (pi - K0 dt).  A fixed blending width delta
    // (the fixed-delta variant of the paper's remark on small time steps) sets W = ceil(delta / dt).
    if (!(o.delta >= 0) || !std::isfinite(o.delta)) {
        *why = "delta must be >= 0 and finite";
        return WFP_EINVAL;
    }
    int w = (o.W > 0) ? o.W
                      : (o.delta > 0 ? (int)std::ceil(o.delta / dt - 1e-9)
                                     : (int)std::ceil(2.0 * b / (kPi - K0dt) - 1e-12));
    if (w < 2) w = 2;
    if (2.0 * b / w >= kPi - K0dt) {
        *why = "W too small for band_limit * dt (Eq. dt)";
        return WFP_EINVAL;
    }
    if (w > 59) {
        *why = "W must be <= 59 (dt too coarse for the band limit, or delta / dt too large)";
        return WFP_EINVAL;
    }
    // default order 20 (Sec. 7), reduced if needed so that nmax = W + 1 + p/2 fits a 32-level window,
    // else a 64-level one
    const int cap = (2 * (31 - w) >= 8) ? 31 : 63;
    int pp = (o.p > 0) ? o.p : std::max(8, std::min(20, 2 * (cap - w)));
    if (pp % 2) pp += 1;
    if (pp > 32) {
        *why = "interpolation order p must be <= 32";
        return WFP_EINVAL;
    }
    if (w + 1 + pp / 2 > kMaxLevels) {
        *why = "W + 1 + p/2 exceeds the supported number of levels";
        return WFP_EINVAL;
    }
    *eps = e;
    *W = w;
    *p = pp;
    *nmax = w + 1 + pp / 2;
    return WFP_OK;
}

wfp_status select_params(double halfside, double dt, int64_t Nt, double K0, double tol, const wfp_opts& o,
                         Params& P, std::string& err) {
    if (!(halfside > 0) || !std::isfinite(halfside)) {
        err = "degenerate or non-finite bounding box";
        return WFP_EINVAL;
    }
    if (!(dt > 0) || !std::isfinite(dt)) {
        err = "dt must be positive and finite";
        return WFP_EINVAL;
    }
    if (Nt < 1) {
        err = "Nt must be >= 1";
        return WFP_EINVAL;
    }
    if (!(K0 >= 0) || !std::isfinite(K0)) {
        err = "band_limit must be >= 0 and finite";
        return WFP_EINVAL;
    }
    if (!(tol > 0 && tol < 1)) {
        err = "tol must be in (0, 1)";
        return WFP_EINVAL;
    }
    if (o.precision != WFP_FP64 && o.precision != WFP_MIXED) {
        err = "precision must be WFP_FP64 or WFP_MIXED";
        return WFP_EINVAL;
    }
    if (o.local_interp != WFP_INTERP_HYBRID && o.local_interp != WFP_INTERP_LAGRANGE) {
        err = "local_interp must be WFP_INTERP_HYBRID or WFP_INTERP_LAGRANGE";
        return WFP_EINVAL;
    }
    if (o.local_form < WFP_LOCAL_AUTO || o.local_form > WFP_LOCAL_FACTORED) {
        err = "local_form must be WFP_LOCAL_AUTO, WFP_LOCAL_STORED or WFP_LOCAL_FACTORED";
        return WFP_EINVAL;
    }
    P.precision = o.precision;
    P.exclude_self = o.exclude_self != 0;
    P.scale = 1.0 / halfside;
    P.dt_user = dt;
    P.K0_user = K0;
    P.tol = tol;
    P.Nt = Nt;
    P.dt = dt * P.scale;
    P.K0 = K0 / P.scale;
    P.T = (double)Nt * P.dt;
    {
        const char* why = "";
        wfp_status st = local_params(dt, K0, tol, o, &P.eps, &P.W, &P.p, &P.nmax, &why);
        if (st != WFP_OK) {
            err = why;
            return st;
        }
    }
    P.b = std::log(1.0 / P.eps);
    P.delta = P.W * P.dt;        // Eq. W
    P.K = P.K0 + 2.0 * P.b / P.delta;  // Eq. K
    P.Delta = 1.0;
    P.a = 1.0;
    P.A = 2.0 * std::sqrt(2.0) + P.Delta;  // Eq. A
    // A+ - delta sits on the time grid and is at least A + a, so the far history starts at
    // least a after the light cone of the truncated kernel (Sec. 2.3).
    P.L = (int)std::ceil((P.A + P.a) / P.dt - 1e-9);
    P.Aplus = P.delta + P.L * P.dt;
    if (!(P.delta < P.A + P.a)) {
        err = "blending width delta exceeds the domain passage time";
        return WFP_EINVAL;
    }
    P.dk = 2.0 * kPi / (P.Aplus + 2.0);  // Eq. dk
    if (o.Kf > 0)
        P.Kf = o.Kf;
    else  // far cut-off from the paper's Table (Delta = 1): 55 -> ~1e-12, 67 -> ~1e-14, 80 -> ~1e-16
        P.Kf = (P.eps >= 1e-10) ? 55.0 : (P.eps >= 1e-13 ? 67.0 : 80.0);
    P.Km = std::max(P.K, P.Kf);
    P.Nh = (int)std::ceil(P.Km / P.dk);
    // lag / far active if some advance n <= Nt-1 sees a lagged level n - L >= 1
    P.lag_active = (Nt - 1 >= P.L + 1);
    P.far_active = P.lag_active;
    // far SOE: n panels with lam_max/2^(n-1) ~ 1/T (Sec. 2.3), ng nodes per panel chosen to meet eps/10
    P.lam_max = 36.0;
    double Tsoe = std::max(P.T, P.Aplus);
    P.soe_panels = std::max(2, (int)std::ceil(std::log2(P.lam_max * Tsoe)));
    if (o.soe_nodes > 0) {
        P.soe_nodes = o.soe_nodes;
    } else if (!P.far_active) {
        P.soe_nodes = 0;
    } else {
        P.soe_nodes = 32;
        for (int ng : {12, 16, 20, 24, 28}) {
            std::vector<double> lam, q;
            soe_nodes(P.lam_max, P.soe_panels, ng, lam, q);
            if (soe_max_rel_error(lam, q, P.A, P.Aplus - P.delta, Tsoe) <= 0.1 * P.eps) {
                P.soe_nodes = ng;
                break;
            }
        }
    }
    P.n_lambda = P.soe_panels * P.soe_nodes;
    // NUFFT: exponential-of-semicircle kernel, width from the tolerance and upsampling factor
    // default upsampling: 1.25 on the FP64 path (FP64 FFTs dominate there); on the mixed path 2 while
    // the grid stays at most 4096 points a side (FP32 FFTs are cheap there and a narrower kernel
    // saves spreading), 1.25 beyond (the FFTs dominate large grids)
    double sig_req = o.upsampfac;
    if (!(sig_req > 0)) sig_req = (P.precision == WFP_FP64 || 2.0 * (2 * P.Nh + 1) > 4096) ? 1.25 : 2.0;
    if (sig_req < 1.2 || sig_req > 4.0) {
        err = "upsampfac must be in [1.2, 4]";
        return WFP_EINVAL;
    }
    double eps_nufft = (P.precision == WFP_MIXED) ? std::max(P.eps, 1e-7) : P.eps;
    P.nf = next_fft_size(std::max((int)std::ceil(sig_req * (2 * P.Nh + 1)), 64));
    // band of grid rows/columns touched by points x' = dk x + pi, x in [-1, 1] (a multiple of the
    // spreading tile); the fine grid grows until the band fits inside one period.  The kernel width
    // and shape follow the effective upsampling n_f / (2 N_h + 1) of the grid chosen.
    for (;;) {
        P.upsamp = (double)P.nf / (2 * P.Nh + 1);
        P.w = (o.kernel_width > 0)
                  ? o.kernel_width
                  : (int)std::ceil(std::log(1.0 / eps_nufft) / (kPi * std::sqrt(1.0 - 1.0 / P.upsamp))) + 1;
        if (P.w < 2 || P.w > 24) {
            err = "kernel_width must be in [2, 24]";
            return WFP_EINVAL;
        }
        P.beta = 0.97 * kPi * (1.0 - 0.5 / P.upsamp) * P.w;
        P.h = 2.0 * kPi / P.nf;
        int lo = (int)std::floor((kPi - P.dk) / P.h - 0.5 * P.w) - 1;
        int hi = (int)std::ceil((kPi + P.dk) / P.h + 0.5 * P.w) + 1;
        int nb = (hi - lo + 1 + kTile - 1) / kTile * kTile;
        if (lo >= 0 && lo + nb <= P.nf) {
            P.lb0 = lo;
            P.nb = nb;
            break;
        }
        P.nf = next_fft_size(P.nf + 2);
    }
    return WFP_OK;
}

void fill_info(const Params& P, wfp_info& I) {
    std::memset(&I, 0, sizeof(I));
    I.scale = P.scale;
    I.cx = P.cx;
    I.cy = P.cy;
    I.dt = P.dt;
    I.T = P.T;
    I.K0 = P.K0;
    I.eps = P.eps;
    I.b = P.b;
    I.W = P.W;
    I.p = P.p;
    I.nmax = P.nmax;
    I.delta = P.delta;
    I.K = P.K;
    I.A = P.A;
    I.Aplus = P.Aplus;
    I.dk = P.dk;
    I.L = P.L;
    I.Kf = P.Kf;
    I.Nh = P.Nh;
    I.n_lambda = P.n_lambda;
    I.soe_panels = P.soe_panels;
    I.soe_nodes = P.soe_nodes;
    I.nf = P.nf;
    I.nb = P.nb;
    I.kernel_width = P.w;
    I.upsampfac = P.upsamp;
    I.lag_active = P.lag_active;
    I.far_active = P.far_active;
    I.precision = P.precision;
}


}  // namespace wfp
