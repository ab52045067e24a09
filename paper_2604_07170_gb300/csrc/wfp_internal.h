// Internal declarations of the 2D TK-WFP evaluator (CUDA path).  Not part of the ABI.
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "wfp.h"

#ifdef __CUDACC__
#define WFP_HD __host__ __device__
#else
#define WFP_HD
#endif

namespace wfp {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxLevels = 64;      // n_max = W + 1 + p/2 must not exceed this
constexpr int kTile = 32;           // spreading tile (grid points per side)
constexpr int kPhiPanels = 32;      // piecewise Chebyshev representation of phi
constexpr int kPhiDeg = 24;

// Parameters of a plan, in normalised units (Secs. 2-6).
struct Params {
    // caller-side
    int64_t M = 0, Mt = 0, Nt = 0;
    double dt_user = 0, K0_user = 0, tol = 0;
    // normalisation x_n = (x - c) * scale, t_n = t * scale
    double cx = 0, cy = 0, scale = 1;
    // normalised
    double dt = 0, K0 = 0, T = 0;
    double eps = 0, b = 0;
    int W = 0, p = 0, nmax = 0;
    double delta = 0, K = 0;
    double Delta = 1.0, A = 0, a = 1.0, Aplus = 0;
    int L = 0;
    double dk = 0;
    double Kf = 0, Km = 0;
    int Nh = 0;
    // far sum of exponentials (Sec. 2.3)
    double lam_max = 36.0;
    int soe_panels = 0, soe_nodes = 0, n_lambda = 0;
    // NUFFT
    double upsamp = 2.0;
    int w = 0;
    double beta = 0;
    int nf = 0, nb = 0, lb0 = 0;
    double h = 0;
    bool lag_active = false, far_active = false;
    int precision = WFP_FP64;
    bool exclude_self = true;
};

// ---------------------------------------------------------------- host helpers
void gauss_legendre(int n, double* x, double* w);                 // nodes/weights on [-1,1]
wfp_status select_params(double halfside, double dt, int64_t Nt, double K0, double tol, const wfp_opts& o,
                         Params& P, std::string& err);
void fill_info(const Params& P, wfp_info& info);

// phi(t) = F(2t/delta - 1); F tabulated as kPhiPanels Chebyshev pieces of degree kPhiDeg on [-1,1].
void build_phi_table(double b, std::vector<double>& coef);
void build_phi_table_into(double b, double* coef);  // kPhiPanels * (kPhiDeg + 1) doubles, no heap use
double phi_host(const double* coef, double t, double delta);
double dphi_host(double t, double delta, double b);                // phi'
double d2phi_host(double t, double delta, double b);               // phi''

constexpr int kLsIntervals = 4;  // newest delay intervals interpolated by band-limited least squares
constexpr int kLsDeg = 28;       // Chebyshev degree of the least-squares weights over those intervals
void build_ls_cheb(int nmax, double dt, double Omega, double span, std::vector<double>& C);
// Chebyshev table of the local weights on the delay intervals k = 1..W-1 (see eta_from_table)
void build_eta_table(double dt, int W, int p, int nmax, const double* phicoef, const double* gx, const double* gw,
                     int ng, const double* wl, const double* Cls, std::vector<double>& tab);
void build_ls_cheb_into(int nmax, double dt, double Omega, double span, double* C);  // no heap use
// coefficients the factored local part keeps from that table, and the relative tail it drops (see
// wfp_debug_factored_table)
int factored_nc_choice(const std::vector<double>& tab, int W, int nmax, bool fp64);
double factored_tail(const std::vector<double>& tab, int W, int nmax, int nc);
// W, p, nmax and eps of the local part from dt, K0 (band limit) and tol (no heap use)
wfp_status local_params(double dt, double K0, double tol, const wfp_opts& o, double* eps, int* W, int* p, int* nmax,
                        const char** why);

// Dyadic-panel Gauss-Legendre discretisation of the Laplace integral
// 1/sqrt(t^2 - r^2) = int_0^inf exp(-lambda t) I0(r lambda) dlambda (Eq. LaplaceIntegral):
// panels [0, lmax/2^(n-1)], [lmax/2^(n-1), lmax/2^(n-2)], ..., [lmax/2, lmax], ng nodes each.
void soe_nodes(double lam_max, int panels, int ng, std::vector<double>& lam, std::vector<double>& q);
// 1/d (r = 0): n0-point Gauss-Legendre in lambda on [0, lc], composite Gauss-Legendre in ln(lambda)
// (panels of width <= ds, n1 nodes each) on [lc, lmax]
void soe_inverse(double lc, int n0, double lmax, double ds, int n1, std::vector<double>& lam,
                 std::vector<double>& q);
// the self term's sum for 1/d on [dlo, T] to relative eps (false if none of the candidates meets it)
bool self_soe(double dlo, double T, double eps, std::vector<double>& lam, std::vector<double>& q);
// max over r in [0, rmax], t in [tlo, thi] of |SOE - 1/sqrt(t^2-r^2)| * sqrt(t^2-r^2)
double soe_max_rel_error(const std::vector<double>& lam, const std::vector<double>& q, double rmax, double tlo,
                         double thi);

// Fourier transform of the exponential-of-semicircle spreading kernel psi at integer n.
void es_kernel_ft(int w, double beta, double h, int nmax, std::vector<double>& out);
WFP_HD inline double es_kernel(double z, double beta) {  // z in [-1, 1]
    double a = 1.0 - z * z;
#ifdef __CUDA_ARCH__
    return a > 0.0 ? exp(beta * (sqrt(a) - 1.0)) : 0.0;
#else
    return a > 0.0 ? std::exp(beta * (std::sqrt(a) - 1.0)) : 0.0;
#endif
}

// Piecewise-Chebyshev evaluation of F(x), x in [-1, 1] (host and device).
WFP_HD inline double cheb_phi(const double* coef, double x) {
    if (x <= -1.0) return 0.0;
    if (x >= 1.0) return 1.0;
    double u = (x + 1.0) * 0.5 * kPhiPanels;
    int k = (int)u;
    if (k >= kPhiPanels) k = kPhiPanels - 1;
    double s = 2.0 * (u - k) - 1.0;
    const double* c = coef + k * (kPhiDeg + 1);
    double b0 = 0, b1 = 0, b2 = 0;
    for (int j = kPhiDeg; j >= 1; j--) {
        b2 = b1;
        b1 = b0;
        b0 = 2.0 * s * b1 - b2 + c[j];
    }
    return s * b0 - b1 + c[0];
}

// Form of the local weights a plan uses (wfp_opts.local_form): WFP_LOCAL_STORED or
// WFP_LOCAL_FACTORED, or -1 when the factored form is asked for but cannot serve the plan.  The
// factored form needs a 32-level window (nmax <= 32), at least one table interval (W >= 2), and
// (W - 1) M coefficient blocks indexable in 32 bits (with room for 16-byte vector indices).
inline int local_form_of(const Params& P, const wfp_opts& o) {
    const bool fits = P.nmax <= 32 && P.W >= 2 && (double)(P.W - 1) * (double)P.M * 8.0 < 4294967296.0;
    if (o.local_form == WFP_LOCAL_FACTORED) return fits ? WFP_LOCAL_FACTORED : -1;
    if (o.local_form == WFP_LOCAL_STORED) return WFP_LOCAL_STORED;
    return (fits && P.precision == WFP_MIXED) ? WFP_LOCAL_FACTORED : WFP_LOCAL_STORED;
}

// Thread-local last-error message.
void set_error(const std::string& s);

}  // namespace wfp
