// Plan-time precomputation of the 2D TK-WFP evaluator (boundary of the per-step path).
//
// Normalises the geometry onto B = [-1,1]^2, finds the local source-target pairs, builds the
// local quadrature weights (Sec. 6), enumerates the near/far Fourier modes with their FIR taps
// (Sec. 4.2) and Hankel coefficients (Sec. 5, Eq. H), the sums of exponentials (Sec. 2.3), the
// NUFFT spreading tables and cuFFT plans, and allocates the device state.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "wfp_local_factored.cuh"
#include "wfp_plan.h"
#include "wfp_quad.h"

namespace wfp {

#define CK(x)                                                                      \
    do {                                                                           \
        cudaError_t e_ = (x);                                                      \
        if (e_ != cudaSuccess) {                                                   \
            err = std::string(#x) + ": " + cudaGetErrorString(e_);                 \
            return (e_ == cudaErrorMemoryAllocation) ? WFP_ENOMEM : WFP_ECUDA;     \
        }                                                                          \
    } while (0)
#define CKF(x)                                                                     \
    do {                                                                           \
        cufftResult r_ = (x);                                                      \
        if (r_ != CUFFT_SUCCESS) {                                                 \
            err = std::string(#x) + ": cufft error " + std::to_string((int)r_);    \
            return (r_ == CUFFT_ALLOC_FAILED) ? WFP_ENOMEM : WFP_ECUDA;            \
        }                                                                          \
    } while (0)

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// scoped temporary device buffer
template <typename T>
struct Tmp {
    T* p = nullptr;
    cudaError_t alloc(size_t n) { return cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)); }
    ~Tmp() {
        if (p) cudaFree(p);
    }
};

// ------------------------------------------------------------------- neighbour search
// pass 0: count pairs with 0 < r < delta and record a coincident source (r <= rc);
// pass 1: write the pairs (source index and FP64 distance) in cell-scan order.
__global__ void k_nbr(int pass, int64_t Mt, const double2* __restrict__ tgt, const double2* __restrict__ src,
                      const int* __restrict__ cell_start, int nc, double cs, double delta, double rc,
                      int* __restrict__ count, int* __restrict__ selfj, int* __restrict__ nself,
                      const int64_t* __restrict__ rowptr, int* __restrict__ col, double* __restrict__ rr) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Mt) return;
    double2 x = tgt[i];
    int cx = min(nc - 1, max(0, (int)floor((x.x + 1.0) / cs)));
    int cy = min(nc - 1, max(0, (int)floor((x.y + 1.0) / cs)));
    int cnt = 0, sj = -1, ns = 0;
    int64_t o = pass ? rowptr[i] : 0;
    double d2max = delta * delta, rc2 = rc * rc;
    for (int gy = max(0, cy - 1); gy <= min(nc - 1, cy + 1); gy++)
        for (int gx = max(0, cx - 1); gx <= min(nc - 1, cx + 1); gx++) {
            int c = gy * nc + gx;
            for (int k = cell_start[c]; k < cell_start[c + 1]; k++) {
                double dx = x.x - src[k].x, dy = x.y - src[k].y;
                double d2 = dx * dx + dy * dy;
                if (d2 <= rc2) {
                    sj = k;
                    ns++;
                    continue;
                }
                if (d2 < d2max) {
                    if (pass) {
                        col[o + cnt] = k;
                        rr[o + cnt] = sqrt(d2);
                    }
                    cnt++;
                }
            }
        }
    if (!pass) {
        count[i] = cnt;
        selfj[i] = sj;
        nself[i] = ns;
    }
}

// ------------------------------------------------------------------- local weights
// weights of each pair slot: from the per-interval Chebyshev table for r >= dt, by the direct
// quadrature below (and for the zero-weight padding slots, r = 0)
template <typename TW>
__global__ void __launch_bounds__(128) k_eta(int64_t npairs, const double* __restrict__ rr, double dt, int W, int p,
                                             int nmax, int NW, const double* __restrict__ phicoef,
                                             const double* __restrict__ gx, const double* __restrict__ gw, int ng,
                                             const double* __restrict__ wl, const double* __restrict__ Cls,
                                             const double* __restrict__ tab, TW* __restrict__ eta) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npairs) return;
    double e[kMaxLevels];
    const double r = rr[k];
    if (tab && r >= dt && r < W * dt)
        eta_from_table(r, dt, W, nmax, tab, e);
    else
        eta_weights(r, dt, W, p, nmax, phicoef, gx, gw, ng, wl, Cls, e);
    // with NW = 32 the row is aligned with the linear window (position NW - nmax + l holds level l)
    const int off = (NW == 32) ? NW - nmax : 0;
    for (int i = 0; i < NW; i++) eta[k * NW + i] = (i >= off && i - off < nmax) ? (TW)e[i - off] : (TW)0;
}

// direct weights at the table's Chebyshev nodes: out[i][l], FP64
__global__ void k_eta_nodes(int nn, const double* __restrict__ rn, double dt, int W, int p, int nmax,
                            const double* __restrict__ phicoef, const double* __restrict__ gx,
                            const double* __restrict__ gw, int ng, const double* __restrict__ wl,
                            const double* __restrict__ Cls, double* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    double e[kMaxLevels];
    eta_weights(rn[i], dt, W, p, nmax, phicoef, gx, gw, ng, wl, Cls, e);
    for (int l = 0; l < nmax; l++) out[(size_t)i * nmax + l] = e[l];
}

// Chebyshev coefficients of the table from the node values (host)
static void eta_table_coefficients(int W, int nmax, const std::vector<double>& vals, std::vector<double>& tab) {
    const int N = kEtaChebDeg + 1;
    tab.assign((size_t)std::max(W - 1, 0) * nmax * N, 0.0);
    for (int k = 1; k < W; k++)
        for (int l = 0; l < nmax; l++)
            for (int d = 0; d < N; d++) {
                double c = 0.0;
                for (int j = 0; j < N; j++)
                    c += vals[((size_t)(k - 1) * N + j) * nmax + l] * std::cos(kPi * d * (j + 0.5) / N);
                tab[((size_t)(k - 1) * nmax + l) * N + d] = (d == 0 ? 1.0 : 2.0) * c / N;
            }
}

void build_eta_table(double dt, int W, int p, int nmax, const double* phicoef, const double* gx, const double* gw,
                     int ng, const double* wl, const double* Cls, std::vector<double>& tab) {
    const int N = kEtaChebDeg + 1;
    std::vector<double> vals((size_t)std::max(W - 1, 0) * N * nmax);
    double e[kMaxLevels];
    for (int k = 1; k < W; k++)
        for (int j = 0; j < N; j++) {  // Chebyshev points of the first kind in v on [0, sqrt(dt)]
            const double v = 0.5 * (std::cos(kPi * (j + 0.5) / N) + 1.0) * std::sqrt(dt);
            eta_weights((k + 1) * dt - v * v, dt, W, p, nmax, phicoef, gx, gw, ng, wl, Cls, e);
            for (int l = 0; l < nmax; l++) vals[((size_t)(k - 1) * N + j) * nmax + l] = e[l];
        }
    eta_table_coefficients(W, nmax, vals, tab);
}

// Factored form: split the pairs of each target row by delay interval -- r >= dt to the table
// pairs (the block (k - 1) M + j of interval k = floor(r / dt) and its Chebyshev variable, exactly
// as eta_from_table forms them), r < dt to the near pairs that keep stored weight rows; row order
// is kept.  Pass 0 counts,
// pass 1 writes.
template <typename T>
__global__ void k_split(int pass, int64_t Mt, int64_t M, const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                        const double* __restrict__ rr, double dt, int W, int* __restrict__ ntab,
                        int* __restrict__ nnear, const int64_t* __restrict__ trow, const int64_t* __restrict__ nrow,
                        TabPair<T>* __restrict__ tp, int* __restrict__ ncol, double* __restrict__ nr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Mt) return;
    const int64_t a = pass ? trow[i] : 0, b = pass ? nrow[i] : 0;
    int ca = 0, cb = 0;
    for (int64_t s = rowptr[i]; s < rowptr[i + 1]; s++) {
        const double r = rr[s];
        if (!(r > 0.0)) continue;
        if (r >= dt && r < W * dt) {
            if (pass) {
                int k = (int)floor(r / dt);
                k = k < 1 ? 1 : (k > W - 1 ? W - 1 : k);
                const double v = sqrt(fmax(0.0, (k + 1) * dt - r));
                TabPair<T> e;
                e.blk = (unsigned)((int64_t)(k - 1) * M + col[s]);
                if constexpr (sizeof(T) == 8) e.pad = 0u;
                e.x = (T)(2.0 * v / sqrt(dt) - 1.0);
                tp[a + ca] = e;
            }
            ca++;
        } else {
            if (pass) {
                ncol[b + cb] = col[s];
                nr[b + cb] = r;
            }
            cb++;
        }
    }
    if (!pass) {
        ntab[i] = ca;
        nnear[i] = cb;
    }
}

// Largest dropped tail sum_{c >= nc} |C[k][l][c]| of the factored form's per-interval series, over
// intervals and levels, relative to the interval's weight scale max_l sum_c |C[k][l][c]|.
double factored_tail(const std::vector<double>& tab, int W, int nmax, int nc) {
    const int N = kEtaChebDeg + 1;
    double w = 0.0;
    for (int kk = 0; kk < W - 1; kk++) {
        double scale = 0.0;
        for (int l = 0; l < nmax; l++) {
            double a = 0.0;
            for (int c = 0; c < N; c++) a += std::fabs(tab[((size_t)kk * nmax + l) * N + c]);
            scale = std::max(scale, a);
        }
        for (int l = 0; l < nmax; l++) {
            double t = 0.0;
            for (int c = nc; c < N; c++) t += std::fabs(tab[((size_t)kk * nmax + l) * N + c]);
            if (scale > 0.0) w = std::max(w, t / scale);
        }
    }
    return w;
}

// Coefficients to keep per interval in the factored form: the smallest multiple of 4 whose dropped
// tail is at most 2^-25 of the interval's weight scale (reduced precision; 36 if even 32 are not
// enough); every coefficient (36, zero-padded) in FP64.
int factored_nc_choice(const std::vector<double>& tab, int W, int nmax, bool fp64) {
    if (fp64 || tab.empty()) return 36;
    const double thr = std::ldexp(1.0, -25);
    for (int c = 8; c <= 32; c += 4)
        if (factored_tail(tab, W, nmax, c) <= thr) return c;
    return 36;
}

// ------------------------------------------------------------------- FIR taps
// taps per distinct |k|, interleaved by level m: FP64 {p_m, q_m, pA_m, qA_m} (Eq. hggrid, dt folded
// in), or FP32 hi parts followed by lo parts ([kid][W][8]) on the mixed path
template <typename TT>
__global__ void k_taps(int64_t nk, const double* __restrict__ kap, double dt, int W, double lagshift, int ngt,
                       const double* __restrict__ sq, const double* __restrict__ wq, const double* __restrict__ f1,
                       const double* __restrict__ f2, TT* __restrict__ taps, double* __restrict__ rot, bool compact) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nk) return;
    if constexpr (sizeof(TT) == 4) {
        if (compact) {  // lag never active: p and q only
            mode_taps(kap[i], dt, W, lagshift, ngt, sq, wq, f1, f2, TapsCompact{taps + i * 4 * W}, rot + 3 * i);
            return;
        }
    }
    const int per = (sizeof(TT) == 8) ? 4 : 8;
    mode_taps(kap[i], dt, W, lagshift, ngt, sq, wq, f1, f2, TapsInterleaved<TT>{taps + i * per * W}, rot + 3 * i);
}

// v -> (hi, lo) float pair rows of length W, or double rows

// H[l][fk] *= f[l] (Hankel coefficients times the tail recurrence's input weight; see the far history)
__global__ void k_scale_terms(int nlam, int64_t nfk, const double* __restrict__ f, double* __restrict__ H) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (int64_t)nlam * nfk) H[i] *= f[i / nfk];
}

// head taps of the far recurrence: ffir[q][k] = sum_l H[l][k] coef[l][q]
__global__ void k_far_head(int nfk, int nlam, int Wh, const double* __restrict__ H, const double* __restrict__ coef,
                           double* __restrict__ ffir) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nfk * Wh) return;
    int64_t k = i / Wh;
    int qq = (int)(i - k * Wh);
    double acc = 0.0;
    for (int l = 0; l < nlam; l++) acc = fma(H[(int64_t)l * nfk + k], coef[(int64_t)l * Wh + qq], acc);
    ffir[(int64_t)qq * nfk + k] = acc;
}

// ------------------------------------------------------------------- Hankel coefficients (Eq. H)
// Tab[l][i] = q_l exp(-A lam_l) I0(lam_l r_i) phi_Delta(A - r_i) r_i w_i on composite GL nodes r_i in [0, A]
__global__ void k_hankel_tab(int nlam, int nr, const double* __restrict__ lam, const double* __restrict__ q,
                             const double* __restrict__ rn, const double* __restrict__ rw,
                             const double* __restrict__ phicoef, double A, double Delta, double* __restrict__ tab) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nlam * nr) return;
    int l = (int)(t / nr), i = (int)(t % nr);
    double r = rn[i];
    double x = A - r;  // phi_Delta(A - r)
    double ph = (x <= 0.0) ? 0.0 : (x >= Delta ? 1.0 : cheb_phi(phicoef, 2.0 * x / Delta - 1.0));
    // I0(lam r) exp(-A lam) = [I0(lam r) e^{-lam r}] e^{-lam (A - r)}
    double lr = lam[l] * r;
    tab[t] = q[l] * cyl_bessel_i0(lr) * exp(-lam[l] * A) * ph * r * rw[i];
}

// H[fk][l] = sum_i J0(kappa_fk r_i) Tab[l][i]
__global__ void k_hankel(int nfk, int nlam, int nr, const double* __restrict__ kap, const double* __restrict__ rn,
                         const double* __restrict__ tab, double* __restrict__ H) {
    extern __shared__ double s_j0[];
    int fk = blockIdx.x;
    double kp = kap[fk];
    for (int i = threadIdx.x; i < nr; i += blockDim.x) s_j0[i] = j0(kp * rn[i]);
    __syncthreads();
    for (int l = threadIdx.x; l < nlam; l += blockDim.x) {
        const double* tl = tab + (int64_t)l * nr;
        double s = 0.0;
        for (int i = 0; i < nr; i++) s = fma(s_j0[i], tl[i], s);
        H[(int64_t)l * nfk + fk] = s;  // [l][fk]: far modes of a warp read neighbouring |k|
    }
}

// ------------------------------------------------------------------- host helpers
template <typename T>
static cudaError_t upload(DevArena& mem, T** d, const std::vector<T>& h) {
    cudaError_t e = mem.alloc(d, h.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <typename T>
static cudaError_t upload_tmp(Tmp<T>& t, const std::vector<T>& h) {
    cudaError_t e = t.alloc(h.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(t.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// counting sort of points into nc x nc cells of side cs over [-1,1]^2; returns the order
static void cell_sort(const std::vector<double>& xy, int nc, double cs, std::vector<int>& order,
                      std::vector<int>& cell_start) {
    int64_t n = (int64_t)xy.size() / 2;
    std::vector<int> cid(n);
    cell_start.assign((size_t)nc * nc + 1, 0);
    for (int64_t i = 0; i < n; i++) {
        int cx = std::min(nc - 1, std::max(0, (int)std::floor((xy[2 * i] + 1.0) / cs)));
        int cy = std::min(nc - 1, std::max(0, (int)std::floor((xy[2 * i + 1] + 1.0) / cs)));
        cid[i] = cy * nc + cx;
        cell_start[cid[i] + 1]++;
    }
    for (size_t c = 0; c + 1 < cell_start.size(); c++) cell_start[c + 1] += cell_start[c];
    std::vector<int> fill(cell_start.begin(), cell_start.end() - 1);
    order.assign(n, 0);
    for (int64_t i = 0; i < n; i++) order[fill[cid[i]]++] = (int)i;
}

// footprint origin (band-relative) and kernel values of a point for the NUFFT
template <typename T>
static void point_kernel(const Params& P, double xs, double ys, int& off, T* ker) {
    double ux = (P.dk * xs + kPi) / P.h, uy = (P.dk * ys + kPi) / P.h;
    int lx = (int)std::ceil(ux - 0.5 * P.w), ly = (int)std::ceil(uy - 0.5 * P.w);
    for (int i = 0; i < P.w; i++) {
        ker[i] = (T)es_kernel((lx + i - ux) / (0.5 * P.w), P.beta);
        ker[P.w + i] = (T)es_kernel((ly + i - uy) / (0.5 * P.w), P.beta);
    }
    int ix0 = lx - P.lb0, iy0 = ly - P.lb0;
    off = (ix0 & 0xffff) | (iy0 << 16);
}

// ------------------------------------------------------------------- plan build
// Non-empty ts x ts tiles of the band and the sources whose footprint touches each, in ascending
// internal source order (tile coordinates packed tx | ty << 16).
struct TileLists {
    std::vector<int> txy, tptr, tsrc;
    bool made = false;
};

static int tile_slot(int ts) { return ts == 8 ? 0 : (ts == 16 ? 1 : 2); }

static TileLists build_tiles(const Params& P, const std::vector<int>& soff, int ts) {
    TileLists t;
    const int ntx = P.nb / ts;
    std::vector<std::pair<int, int>> pairs;
    pairs.reserve(soff.size() * 3);
    for (size_t k = 0; k < soff.size(); k++) {
        int ix0 = soff[k] & 0xffff, iy0 = soff[k] >> 16;
        for (int ty = iy0 / ts; ty <= (iy0 + P.w - 1) / ts; ty++)
            for (int tx = ix0 / ts; tx <= (ix0 + P.w - 1) / ts; tx++) pairs.push_back({ty * ntx + tx, (int)k});
    }
    std::sort(pairs.begin(), pairs.end());
    for (size_t i = 0; i < pairs.size(); i++) {
        if (i == 0 || pairs[i].first != pairs[i - 1].first) {
            int tt = pairs[i].first;
            t.txy.push_back((tt % ntx) | ((tt / ntx) << 16));
            t.tptr.push_back((int)i);
        }
        t.tsrc.push_back(pairs[i].second);
    }
    t.tptr.push_back((int)pairs.size());
    t.made = true;
    return t;
}

template <typename T>
static wfp_status build_t(Plan& pl, const std::vector<double>& sxy, const std::vector<double>& txy, std::string& err) {
    using C = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
    Params& P = pl.P;
    DevArena& mem = pl.mem;
    const int64_t M = P.M, Mt = P.Mt;
    pl.M = M;
    pl.Mt = Mt;
    pl.NW = (P.nmax <= 32) ? 32 : 64;

    CK(mem.alloc(&pl.d_step, 1));
    // ---- phi table
    std::vector<double> phic;
    build_phi_table(P.b, phic);
    CK(upload(mem, &pl.d_phicoef, phic));

    // ---- cell sort of sources and targets (cells of side >= delta)
    int nc = std::max(1, std::min(4096, (int)std::floor(2.0 / P.delta)));
    double cs = 2.0 / nc;
    std::vector<int> sorder, scs, torder, tcs;
    cell_sort(sxy, nc, cs, sorder, scs);
    cell_sort(txy, nc, cs, torder, tcs);
    std::vector<double> ss(2 * M), ts(2 * Mt);
    for (int64_t k = 0; k < M; k++) {
        ss[2 * k] = sxy[2 * (int64_t)sorder[k]];
        ss[2 * k + 1] = sxy[2 * (int64_t)sorder[k] + 1];
    }
    for (int64_t k = 0; k < Mt; k++) {
        ts[2 * k] = txy[2 * (int64_t)torder[k]];
        ts[2 * k + 1] = txy[2 * (int64_t)torder[k] + 1];
    }
    CK(upload(mem, &pl.d_src_perm, sorder));
    CK(upload(mem, &pl.d_tgt_perm, torder));

    // ---- neighbour search (Sec. 6: N_delta = {j : 0 < r_ij < delta})
    const int64_t bytes_before_local = mem.bytes;
    const int form = local_form_of(P, pl.opts);
    if (form < 0) {
        err = "local_form WFP_LOCAL_FACTORED needs nmax <= 32, W >= 2 and 8 (W - 1) M < 2^32";
        return WFP_EUNSUPPORTED;
    }
    pl.local_factored = form == WFP_LOCAL_FACTORED;
    {
        Tmp<double> d_s, d_t, d_r;
        Tmp<int> d_cs, d_cnt, d_self, d_ns;
        CK(upload_tmp(d_s, ss));
        CK(upload_tmp(d_t, ts));
        CK(upload_tmp(d_cs, scs));
        CK(d_cnt.alloc(Mt));
        CK(d_self.alloc(Mt));
        CK(d_ns.alloc(Mt));
        const double rc = 2e-12;  // coincident: distance <= 1e-12 of the domain side
        k_nbr<<<nblk(Mt, 128), 128>>>(0, Mt, (const double2*)d_t.p, (const double2*)d_s.p, d_cs.p, nc, cs, P.delta,
                                      rc, d_cnt.p, d_self.p, d_ns.p, nullptr, nullptr, nullptr);
        CK(cudaGetLastError());
        std::vector<int> cnt(Mt), selfj(Mt), ns(Mt);
        CK(cudaMemcpy(cnt.data(), d_cnt.p, Mt * sizeof(int), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(selfj.data(), d_self.p, Mt * sizeof(int), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(ns.data(), d_ns.p, Mt * sizeof(int), cudaMemcpyDeviceToHost));
        // stored form: rows padded to a multiple of 4 pair slots (zero-weight slots with r = 0, source
        // 0), so that every row starts 16-byte aligned in the index array for the bulk copies of the
        // local part; factored form: unpadded (the pairs are split by interval below)
        const bool fac = pl.local_factored;
        std::vector<int64_t> rowptr(Mt + 1, 0);
        pl.n_pairs = 0;
        for (int64_t i = 0; i < Mt; i++) {
            rowptr[i + 1] = rowptr[i] + (fac ? cnt[i] : ((cnt[i] + 3) & ~3));
            pl.n_pairs += cnt[i];
        }
        const int64_t nall = rowptr[Mt];
        std::vector<int> st, ssrc;
        for (int64_t i = 0; i < Mt; i++) {
            if (ns[i] > 1) {
                err = "a target coincides with more than one source";
                return WFP_EUNSUPPORTED;
            }
            if (selfj[i] >= 0) {
                st.push_back((int)i);
                ssrc.push_back(selfj[i]);
            }
        }
        pl.n_self = P.exclude_self ? (int64_t)st.size() : 0;
        if (pl.n_self > 0) {
            CK(upload(mem, &pl.d_self_tgt, st));
            CK(upload(mem, &pl.d_self_src, ssrc));
        }
        size_t freeb = 0, totb = 0;
        CK(cudaMemGetInfo(&freeb, &totb));
        size_t need = fac ? (size_t)nall * (sizeof(int) + sizeof(double) + sizeof(TabPair<T>)) +
                                (size_t)(P.W - 1) * M * 36 * sizeof(T)
                          : (size_t)nall * (sizeof(int) + sizeof(double) + pl.NW * sizeof(T));
        if (need + (size_t)(1ull << 30) > freeb) {
            err = "local part needs " + std::to_string(need >> 20) + " MiB of device memory";
            return WFP_ENOMEM;
        }
        Tmp<int64_t> d_rpall;
        Tmp<int> d_colall;
        int64_t* rp = nullptr;
        int* colp = nullptr;
        if (fac) {
            CK(upload_tmp(d_rpall, rowptr));
            CK(d_colall.alloc(nall));
            rp = d_rpall.p;
            colp = d_colall.p;
        } else {
            CK(upload(mem, &pl.d_rowptr, rowptr));
            CK(mem.alloc(&pl.d_col, nall));
            rp = pl.d_rowptr;
            colp = pl.d_col;
            pl.n_slots = nall;
        }
        CK(d_r.alloc(nall));
        CK(cudaMemset(d_r.p, 0, std::max<size_t>(nall, 1) * sizeof(double)));
        k_nbr<<<nblk(Mt, 128), 128>>>(1, Mt, (const double2*)d_t.p, (const double2*)d_s.p, d_cs.p, nc, cs, P.delta,
                                      rc, nullptr, nullptr, nullptr, rp, colp, d_r.p);
        CK(cudaGetLastError());
        // ---- local weights (Sec. 6)
        const int ng = 20;
        std::vector<double> gx(ng), gw(ng), wl(P.p);
        gauss_legendre(ng, gx.data(), gw.data());
        lagrange_ref_weights(P.p, wl.data());
        std::vector<double> bls;
        const double Omega = std::max(P.K0, 1e-3 / P.dt);
        build_ls_cheb(P.nmax, P.dt, Omega, kLsIntervals * P.dt, bls);
        Tmp<double> d_gx, d_gw, d_wl, d_bls;
        CK(upload_tmp(d_gx, gx));
        CK(upload_tmp(d_gw, gw));
        CK(upload_tmp(d_wl, wl));
        CK(upload_tmp(d_bls, bls));
        const double* Cls = pl.opts.local_interp == WFP_INTERP_LAGRANGE ? nullptr : d_bls.p;
        // Chebyshev table of the weights on the delay intervals k >= 1: direct weights at the nodes
        // (device), coefficients (host); pairs then evaluate the table instead of the quadrature
        Tmp<double> d_tab;
        std::vector<double> tab;
        if (P.W >= 2) {
            const int N = kEtaChebDeg + 1, nn = (P.W - 1) * N;
            std::vector<double> rn(nn), vals((size_t)nn * P.nmax);
            for (int k = 1; k < P.W; k++)
                for (int j = 0; j < N; j++) {
                    const double v = 0.5 * (std::cos(kPi * (j + 0.5) / N) + 1.0) * std::sqrt(P.dt);
                    rn[(size_t)(k - 1) * N + j] = (k + 1) * P.dt - v * v;
                }
            Tmp<double> d_rn, d_vals;
            CK(upload_tmp(d_rn, rn));
            CK(d_vals.alloc(vals.size()));
            k_eta_nodes<<<nblk(nn, 64), 64>>>(nn, d_rn.p, P.dt, P.W, P.p, P.nmax, pl.d_phicoef, d_gx.p, d_gw.p, ng,
                                             d_wl.p, Cls, d_vals.p);
            CK(cudaGetLastError());
            CK(cudaMemcpy(vals.data(), d_vals.p, vals.size() * sizeof(double), cudaMemcpyDeviceToHost));
            eta_table_coefficients(P.W, P.nmax, vals, tab);
            CK(upload_tmp(d_tab, tab));
        }
        Tmp<double> d_nr;  // factored form: distances of the near pairs
        const double* rslot = d_r.p;
        if (fac) {
            // split every row: r >= dt -> table pairs (factored weights), r < dt -> near pairs
            Tmp<int> d_nt, d_nn;
            CK(d_nt.alloc(Mt));
            CK(d_nn.alloc(Mt));
            k_split<T><<<nblk(Mt, 128), 128>>>(0, Mt, M, rp, colp, d_r.p, P.dt, P.W, d_nt.p, d_nn.p, nullptr, nullptr,
                                               nullptr, nullptr, nullptr);
            CK(cudaGetLastError());
            std::vector<int> nt(Mt), nnr(Mt);
            CK(cudaMemcpy(nt.data(), d_nt.p, Mt * sizeof(int), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(nnr.data(), d_nn.p, Mt * sizeof(int), cudaMemcpyDeviceToHost));
            std::vector<int64_t> trow(Mt + 1, 0), nrow(Mt + 1, 0);
            for (int64_t i = 0; i < Mt; i++) {
                trow[i + 1] = trow[i] + nt[i];
                nrow[i + 1] = nrow[i] + nnr[i];
            }
            pl.n_tab = trow[Mt];
            pl.n_near = nrow[Mt];
            pl.n_slots = pl.n_near;
            CK(upload(mem, &pl.d_trow, trow));
            CK(upload(mem, &pl.d_rowptr, nrow));
            TabPair<T>* tp = nullptr;
            CK(mem.alloc(&tp, (size_t)pl.n_tab));
            pl.d_tpair = tp;
            CK(mem.alloc(&pl.d_col, (size_t)pl.n_near));
            CK(d_nr.alloc(pl.n_near));
            k_split<T><<<nblk(Mt, 128), 128>>>(1, Mt, M, rp, colp, d_r.p, P.dt, P.W, nullptr, nullptr, pl.d_trow,
                                               pl.d_rowptr, tp, pl.d_col, d_nr.p);
            CK(cudaGetLastError());
            rslot = d_nr.p;
            // series coefficients by window position, cut after NC terms
            pl.NC = factored_nc_supported(factored_nc_choice(tab, P.W, P.nmax, sizeof(T) == 8), sizeof(T) == 8);
            // (FP32 blocks lane-interleaved by coefficient parity, see k_local_cheb2)
            std::vector<T> ctab((size_t)(P.W - 1) * 32 * pl.NC, (T)0);
            const int N = kEtaChebDeg + 1;
            for (int kk = 0; kk < P.W - 1; kk++)
                for (int l = 0; l < P.nmax; l++)
                    for (int c = 0; c < std::min(pl.NC, N); c++)
                        ctab[((size_t)kk * 32 + (32 - P.nmax + l)) * pl.NC + (sizeof(T) == 8 ? c : cheb2_position(c))] =
                            (T)tab[((size_t)kk * P.nmax + l) * N + c];
            T* dct = nullptr;
            CK(upload(mem, &dct, ctab));
            pl.d_ctab = dct;
            T* dy = nullptr;
            CK(mem.alloc(&dy, (size_t)(P.W - 1) * M * pl.NC));
            pl.d_ycoef = dy;
        }
        T* eta = nullptr;
        CK(mem.alloc(&eta, (size_t)pl.n_slots * pl.NW));
        pl.d_eta = eta;
        if (pl.n_slots > 0) {
            k_eta<T><<<nblk(pl.n_slots, 128), 128>>>(pl.n_slots, rslot, P.dt, P.W, P.p, P.nmax, pl.NW, pl.d_phicoef,
                                                     d_gx.p, d_gw.p, ng, d_wl.p, Cls, d_tab.p, eta);
            CK(cudaGetLastError());
        }
        CK(cudaStreamSynchronize(cudaStreamPerThread));
    }
    pl.bytes_local = mem.bytes - bytes_before_local;
    // step order: the two branches of a step compete for L2 and HBM once each fills the device alone
    if (pl.opts.step_order < WFP_ORDER_AUTO || pl.opts.step_order > WFP_ORDER_SERIAL) {
        err = "step_order must be WFP_ORDER_AUTO, WFP_ORDER_CONCURRENT or WFP_ORDER_SERIAL";
        return WFP_EINVAL;
    }
    pl.serial_step = pl.opts.step_order == WFP_ORDER_SERIAL ||
                     (pl.opts.step_order == WFP_ORDER_AUTO && pl.n_pairs >= (int64_t)200000000);

    // ---- near-history modes: half-plane disk |n| dk <= Km (n2 > 0, or n2 = 0 and n1 >= 0)
    const int Nh = P.Nh;
    const double R2 = (P.Km / P.dk) * (P.Km / P.dk), Rf2 = (P.Kf / P.dk) * (P.Kf / P.dk);
    const int64_t maxsq = (int64_t)std::floor(R2) + 1;
    std::vector<int2> modes;
    std::vector<int> sqidx(maxsq + 1, -1), fsqidx;
    modes.reserve((size_t)(1.6 * R2) + 16);
    for (int pass = 0; pass < 2; pass++) {
        for (int t = 0; t <= 2 * Nh; t++) {
            int n1 = (t <= Nh) ? t : t - 2 * Nh - 1;
            int n2max = (int)std::floor(std::sqrt(std::max(0.0, R2 - (double)n1 * n1)));
            for (int n2 = (n1 >= 0 ? 0 : 1); n2 <= n2max; n2++) {
                int64_t sq = (int64_t)n1 * n1 + (int64_t)n2 * n2;
                if ((double)sq > R2) continue;
                if (pass == 0)
                    sqidx[sq] = 1;
                else
                    modes.push_back(make_int2(n1, n2));
            }
        }
        if (pass == 0) {
            int nk = 0;
            for (auto& v : sqidx)
                if (v >= 0) v = nk++;
            pl.n_kappa = nk;
        }
    }
    // modes sorted by |n|^2: the 32 modes of a warp share a few distinct |k|, so the FIR taps (stored
    // once per |k|) are read by few transactions; the grid gather/scatter of k_modes is by index
    std::stable_sort(modes.begin(), modes.end(), [](const int2& a, const int2& b) {
        return (int64_t)a.x * a.x + (int64_t)a.y * a.y < (int64_t)b.x * b.x + (int64_t)b.y * b.y;
    });
    pl.n_modes = (int64_t)modes.size();
    std::vector<int> mk(pl.n_modes);
    std::vector<double> kap(pl.n_kappa);
    for (int64_t sq = 0; sq <= maxsq; sq++)
        if (sqidx[sq] >= 0) kap[sqidx[sq]] = P.dk * std::sqrt((double)sq);
    for (int64_t m = 0; m < pl.n_modes; m++)
        mk[m] = sqidx[(int64_t)modes[m].x * modes[m].x + (int64_t)modes[m].y * modes[m].y];
    CK(upload(mem, &pl.d_mode_n, modes));
    CK(upload(mem, &pl.d_mode_k, mk));

    // ---- FIR taps per distinct |k| (Eq. hggrid)
    {
        const int ngt = 24;
        std::vector<double> gx(ngt), gw(ngt), sq(ngt), wq(ngt), f1((size_t)P.W * ngt), f2((size_t)P.W * ngt);
        gauss_legendre(ngt, gx.data(), gw.data());
        for (int q = 0; q < ngt; q++) {
            sq[q] = 0.5 * P.dt * (gx[q] + 1.0);
            wq[q] = 0.5 * P.dt * gw[q];
        }
        for (int m = 0; m < P.W; m++)
            for (int q = 0; q < ngt; q++) {
                double d = sq[q] + m * P.dt;
                f1[(size_t)m * ngt + q] = dphi_host(d, P.delta, P.b);
                f2[(size_t)m * ngt + q] = d2phi_host(d, P.delta, P.b);
            }
        Tmp<double> d_kap, d_sq, d_wq, d_f1, d_f2;
        CK(upload_tmp(d_kap, kap));
        CK(upload_tmp(d_sq, sq));
        CK(upload_tmp(d_wq, wq));
        CK(upload_tmp(d_f1, f1));
        CK(upload_tmp(d_f2, f2));
        T* taps = nullptr;
        pl.compact_taps = (sizeof(T) == 4) && !P.lag_active;
        CK(mem.alloc(&taps, (size_t)pl.n_kappa * (sizeof(T) == 8 || pl.compact_taps ? 4 : 8) * P.W));
        pl.d_taps = taps;
        CK(mem.alloc(&pl.d_rot, (size_t)pl.n_kappa * 3));
        k_taps<T><<<nblk(pl.n_kappa, 128), 128>>>(pl.n_kappa, d_kap.p, P.dt, P.W, P.Aplus - P.delta, ngt, d_sq.p,
                                                  d_wq.p, d_f1.p, d_f2.p, taps, pl.d_rot, pl.compact_taps);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(cudaStreamPerThread));
    }

    // ---- far history (Sec. 5): far modes |k| <= Kf, SOE (Sec. 2.3), Hankel coefficients, taps
    if (P.far_active) {
        std::vector<int> fm, fk;
        fsqidx.assign((size_t)std::floor(Rf2) + 2, -1);
        int nfk = 0;
        for (int64_t m = 0; m < pl.n_modes; m++) {
            int64_t s2 = (int64_t)modes[m].x * modes[m].x + (int64_t)modes[m].y * modes[m].y;
            if ((double)s2 <= Rf2) {
                if (fsqidx[s2] < 0) fsqidx[s2] = -2;  // mark
                fm.push_back((int)m);
            }
        }
        std::vector<double> fkap;
        for (size_t s2 = 0; s2 < fsqidx.size(); s2++)
            if (fsqidx[s2] == -2) {
                fsqidx[s2] = nfk++;
                fkap.push_back(P.dk * std::sqrt((double)s2));
            }
        for (int m : fm) fk.push_back(fsqidx[(int64_t)modes[m].x * modes[m].x + (int64_t)modes[m].y * modes[m].y]);
        pl.n_far = (int64_t)fm.size();
        pl.n_fkappa = nfk;
        CK(upload(mem, &pl.d_far_mode, fm));
        CK(upload(mem, &pl.d_far_k, fk));
        std::vector<double> lam, q;
        soe_nodes(P.lam_max, P.soe_panels, P.soe_nodes, lam, q);
        // composite GL in r on [0, A]: 32 panels x 16 nodes
        const int npan = 32, ngr = 16, nr = npan * ngr;
        std::vector<double> gx(ngr), gw(ngr), rn(nr), rw(nr);
        gauss_legendre(ngr, gx.data(), gw.data());
        for (int k = 0; k < npan; k++)
            for (int i = 0; i < ngr; i++) {
                double a = P.A * k / npan, b = P.A * (k + 1) / npan;
                rn[k * ngr + i] = 0.5 * (b - a) * gx[i] + 0.5 * (b + a);
                rw[k * ngr + i] = 0.5 * (b - a) * gw[i];
            }
        Tmp<double> d_lam, d_q, d_rn, d_rw, d_tab, d_fkap;
        CK(upload_tmp(d_lam, lam));
        CK(upload_tmp(d_q, q));
        CK(upload_tmp(d_rn, rn));
        CK(upload_tmp(d_rw, rw));
        CK(upload_tmp(d_fkap, fkap));
        CK(d_tab.alloc((size_t)P.n_lambda * nr));
        k_hankel_tab<<<nblk((int64_t)P.n_lambda * nr, 256), 256>>>(P.n_lambda, nr, d_lam.p, d_q.p, d_rn.p, d_rw.p,
                                                                   pl.d_phicoef, P.A, P.Delta, d_tab.p);
        CK(cudaGetLastError());
        CK(mem.alloc(&pl.d_H, (size_t)nfk * P.n_lambda));
        k_hankel<<<nfk, 256, nr * sizeof(double)>>>(nfk, P.n_lambda, nr, d_fkap.p, d_rn.p, d_tab.p, pl.d_H);
        CK(cudaGetLastError());
        // The blended far kernel integrated against the trapezoid interpolant of the lagged S gives
        //   B_l(t_{n+1}) = r_l B_l(t_n) + sum_{m<W} a_l r_l^m d_m S_{n-L-m},
        //   r_l = exp(-lam_l dt), a_l = dt exp(-lam_l ((L+1) dt - A)), d_m = phi((W-m) dt) - phi((W-1-m) dt).
        // Unrolled, the partial sums of d_m telescope to P_q = 1 - phi((W-1-q) dt) (= 1 for q >= W-1), so
        //   alpha_F = sum_l H_l E_l + sum_{q<W-1} Phi_q(|k|) S_{n-L-q},
        //   E_l(t_{n+1}) = r_l E_l(t_n) + a_l r_l^(W-1) S_{n-L-W+1},
        //   Phi_q(|k|) = P_q sum_l H_l(|k|) a_l r_l^q
        // (the split of the far forcing into a one-tap tail recurrence and a FIR over the newest
        // lagged levels, Sec. 5): the same sums, with one tap per term instead of W.
        const int Wh = P.W - 1;
        std::vector<double> fdec(P.n_lambda), ffor(P.n_lambda), coef((size_t)P.n_lambda * std::max(Wh, 1));
        for (int l = 0; l < P.n_lambda; l++) {
            fdec[l] = std::exp(-lam[l] * P.dt);
            ffor[l] = P.dt * std::exp(-lam[l] * ((P.L + P.W) * P.dt - P.A));
            for (int qq = 0; qq < Wh; qq++)
                coef[(size_t)l * Wh + qq] = (1.0 - phi_host(phic.data(), (Wh - qq) * P.dt, P.delta)) * P.dt *
                                            std::exp(-lam[l] * ((P.L + 1 + qq) * P.dt - P.A));
        }
        Tmp<double> d_coef;
        CK(upload_tmp(d_coef, coef));
        CK(mem.alloc(&pl.d_ffir, (size_t)nfk * std::max(Wh, 1)));
        k_far_head<<<nblk((int64_t)nfk * Wh, 128), 128>>>(nfk, P.n_lambda, Wh, pl.d_H, d_coef.p, pl.d_ffir);
        CK(cudaGetLastError());
        CK(upload(mem, &pl.d_fdecay, fdec));
        CK(upload(mem, &pl.d_fforce, ffor));
        // the step keeps the tail state as Eh_l = E_l / f_l (f_l = a_l r_l^(W-1)), Eh_l <- r_l Eh_l +
        // S_{n-L-W+1}, and reads it with H_l f_l: two FP64 fused multiply-adds per term and component
        k_scale_terms<<<nblk((int64_t)nfk * P.n_lambda, 256), 256>>>(P.n_lambda, nfk, pl.d_fforce, pl.d_H);
        CK(cudaGetLastError());
        CK(mem.alloc(&pl.d_B, (size_t)P.n_lambda * pl.n_far));
        CK(mem.alloc(&pl.d_aF, (size_t)pl.n_far));
        pl.bytes_history += (int64_t)((size_t)P.n_lambda * pl.n_far + pl.n_far) * sizeof(double2);
        for (size_t f = 0; f < fm.size(); f++)
            if (fm[f] != (int)f) {  // modes are ordered by |k|, so the far modes are a prefix
                err = "far modes are not the first modes";
                return WFP_ECUDA;
            }
        CK(cudaStreamSynchronize(cudaStreamPerThread));
    }

    // ---- self term of coincident pairs: SOE of 1/d on [dt, T].  The trapezoid rule below evaluates
    // phi(d) sigma(t - d) / d only at grid delays d = m dt, m >= 1 (phi(0) = 0), so the sum of
    // exponentials has to represent 1/d there and nowhere closer to 0.
    if (pl.n_self > 0) {
        const double dlo = P.dt;
        double Tself = std::max(P.T, 2.0 * P.delta);
        std::vector<double> lam, q;
        const bool ok = self_soe(dlo, Tself, P.eps, lam, q);
        if (!ok) {
            err = "self-term sum of exponentials did not reach the tolerance";
            return WFP_EINVAL;
        }
        pl.n_soe_self = (int)lam.size();
        // Y_l(t_{n+1}) = r_l Y_l(t_n) + dt sum_{m<W} r_l^(m+1) [phi((m+1) dt) - phi(m dt)] sigma_{n-m}
        // (trapezoid on the grid); unrolled, the partial sums telescope to phi((q+1) dt), so
        //   u_self(t_n) = sum_{q<W-1} g_q sigma_{n-1-q} + sum_l (w_l dt / 2 pi) Z_l(t_n),
        //   Z_l(t_{n+1}) = r_l Z_l(t_n) + r_l^W sigma_{n+1-W},
        //   g_q = dt phi((q+1) dt) sum_l (w_l / 2 pi) r_l^(q+1):
        // one shared W-tap window and a one-tap recurrence per term.  The state is stored as
        // Zh_l = Z_l / r_l^W (Zh_l <- r_l Zh_l + sigma_{n+1-W}) and its weight as w_l dt r_l^W / 2 pi.
        const int Wh = P.W - 1;
        std::vector<double> sdec(pl.n_soe_self), sw(pl.n_soe_self), head(std::max(Wh, 1), 0.0);
        for (int l = 0; l < pl.n_soe_self; l++) {
            sdec[l] = std::exp(-lam[l] * P.dt);
            sw[l] = q[l] / (2.0 * kPi) * P.dt * std::exp(-lam[l] * P.W * P.dt);
        }
        for (int qq = 0; qq < Wh; qq++) {
            double acc = 0.0;
            for (int l = 0; l < pl.n_soe_self; l++) acc += q[l] / (2.0 * kPi) * std::exp(-lam[l] * (qq + 1) * P.dt);
            head[qq] = P.dt * phi_host(phic.data(), (qq + 1) * P.dt, P.delta) * acc;
        }
        CK(upload(mem, &pl.d_shead, head));
        CK(upload(mem, &pl.d_sdecay, sdec));
        CK(upload(mem, &pl.d_sw, sw));
        CK(mem.alloc(&pl.d_Y, (size_t)pl.n_soe_self * pl.n_self));
        pl.bytes_history += (int64_t)((size_t)pl.n_soe_self * pl.n_self * sizeof(double));
    }

    // ---- NUFFT tables: footprints, kernel values, deconvolution factors, spreading tiles
    TileLists tile_lists[3];  // tile side 8, 16, 32
    {
        if (P.nb >= 32768) {
            err = "NUFFT band too large for 16-bit footprint offsets";
            return WFP_EUNSUPPORTED;
        }
        std::vector<int> soff(M), toff(Mt);
        std::vector<T> sker((size_t)M * 2 * P.w), tker((size_t)Mt * 2 * P.w);
        for (int64_t k = 0; k < M; k++) point_kernel<T>(P, ss[2 * k], ss[2 * k + 1], soff[k], &sker[(size_t)k * 2 * P.w]);
        for (int64_t k = 0; k < Mt; k++)
            point_kernel<T>(P, ts[2 * k], ts[2 * k + 1], toff[k], &tker[(size_t)k * 2 * P.w]);
        CK(upload(mem, &pl.d_src_off, soff));
        CK(upload(mem, &pl.d_tgt_off, toff));
        T* dsk = nullptr;
        T* dtk = nullptr;
        CK(upload(mem, &dsk, sker));
        CK(upload(mem, &dtk, tker));
        pl.d_src_ker = dsk;
        pl.d_tgt_ker = dtk;
        std::vector<double> psihat;
        es_kernel_ft(P.w, P.beta, P.h, P.Nh, psihat);
        std::vector<double> fac(P.Nh + 1);
        for (int n = 0; n <= P.Nh; n++) fac[n] = ((n & 1) ? -1.0 : 1.0) * P.h / psihat[n];
        CK(upload(mem, &pl.d_fac, fac));
        std::vector<float> facf(fac.begin(), fac.end());
        CK(upload(mem, &pl.d_facf, facf));
        // tiles of the band touched by each source footprint, for each candidate tile side; the
        // autotuner below times them and keeps one
        const int opt_ts = pl.opts.spread_tile, opt_ch = pl.opts.spread_chunk;
        if ((opt_ts != 0 && opt_ts != 8 && opt_ts != 16 && opt_ts != 32) ||
            (opt_ch != 0 && opt_ch != 32 && opt_ch != 64)) {
            err = "spread_tile must be 0, 8, 16 or 32 and spread_chunk 0, 32 or 64";
            return WFP_EINVAL;
        }
        for (int ts : {8, 16, 32}) {
            if (opt_ts != 0 && ts != opt_ts) continue;
            tile_lists[tile_slot(ts)] = build_tiles(P, soff, ts);
        }

    }

    // ---- lagged S: stored history (L + W levels per mode) or a lagged type-1 NUFFT (Sec. 4.3)
    {
        size_t hist = (size_t)(P.L + P.W) * pl.n_modes * sizeof(C);
        size_t freeb = 0, totb = 0;
        CK(cudaMemGetInfo(&freeb, &totb));
        int mode = pl.opts.lag_mode;
        if (mode != WFP_LAG_AUTO && mode != WFP_LAG_RECOMPUTE && mode != WFP_LAG_STORE) {
            err = "lag_mode must be WFP_LAG_AUTO, WFP_LAG_RECOMPUTE or WFP_LAG_STORE";
            return WFP_EINVAL;
        }
        pl.lag_store = P.lag_active && (mode == WFP_LAG_STORE || (mode == WFP_LAG_AUTO && hist <= 0.4 * freeb));
        if (pl.lag_store) {
            pl.R_cur = P.L + P.W;
            pl.R_lag = pl.R_cur;
            pl.lag_off = 0;
        } else {
            pl.R_cur = P.W;
            pl.R_lag = P.W;
            pl.lag_off = P.L;
        }
    }

    // ---- grids and cuFFT plans (two-stage pruned transforms)
    const int64_t bytes_before_grid = mem.bytes;
    {
        const int64_t nf = P.nf, nh2 = P.nf / 2 + 1, nc1 = P.Nh + 1;
        T* sp = nullptr;
        C *tb = nullptr, *tc = nullptr, *td = nullptr, *te = nullptr;
        T* tf = nullptr;
        CK(mem.alloc(&sp, (size_t)P.nb * nf));
        pl.d_sp_cur = sp;
        CK(mem.alloc(&tb, (size_t)nf * nh2));
        pl.d_tb_cur = tb;
        CK(mem.alloc(&tc, (size_t)nf * nc1));
        pl.d_tcol_cur = tc;
        CK(mem.alloc(&tc, (size_t)nf * nc1));
        pl.d_tc_cur = tc;
        if (P.lag_active && !pl.lag_store) {
            CK(mem.alloc(&sp, (size_t)P.nb * nf));
            pl.d_sp_lag = sp;
            CK(mem.alloc(&tb, (size_t)nf * nh2));
            pl.d_tb_lag = tb;
            CK(mem.alloc(&tc, (size_t)nf * nc1));
            pl.d_tcol_lag = tc;
            CK(mem.alloc(&tc, (size_t)nf * nc1));
            pl.d_tc_lag = tc;
        } else {
            pl.d_tc_lag = pl.d_tc_cur;  // never read while the lag is inactive
        }
        CK(mem.alloc(&td, (size_t)nf * nc1));
        pl.d_td = td;
        CK(mem.alloc(&td, (size_t)nf * nc1));
        pl.d_te2 = td;
        CK(mem.alloc(&te, (size_t)nf * nh2));
        pl.d_te = te;
        CK(mem.alloc(&tf, (size_t)P.nb * nf));
        pl.d_tf = tf;
        const bool dbl = sizeof(T) == 8;
        int n[1] = {(int)nf};
        int emb_r[1] = {(int)nf}, emb_c[1] = {(int)nh2};
        CKF(cufftPlanMany(&pl.fftA, 1, n, emb_r, 1, (int)nf, emb_c, 1, (int)nh2, dbl ? CUFFT_D2Z : CUFFT_R2C, P.nb));
        pl.fft_made[0] = true;
        // column transforms over the column-major [Nh+1][nf] layout: contiguous vectors
        CKF(cufftPlanMany(&pl.fftB, 1, n, emb_r, 1, (int)nf, emb_r, 1, (int)nf, dbl ? CUFFT_Z2Z : CUFFT_C2C, (int)nc1));
        pl.fft_made[1] = true;
        CKF(cufftPlanMany(&pl.fftBi, 1, n, emb_r, 1, (int)nf, emb_r, 1, (int)nf, dbl ? CUFFT_Z2Z : CUFFT_C2C, (int)nc1));
        pl.fft_made[2] = true;
        CKF(cufftPlanMany(&pl.fftAi, 1, n, emb_c, 1, (int)nh2, emb_r, 1, (int)nf, dbl ? CUFFT_Z2D : CUFFT_C2R, P.nb));
        pl.fft_made[3] = true;
        for (int i = 0; i < 4; i++) {
            cufftHandle h = (i == 0) ? pl.fftA : (i == 1) ? pl.fftB : (i == 2) ? pl.fftBi : pl.fftAi;
            CKF(cufftSetStream(h, pl.stream));
            size_t ws = 0;
            CKF(cufftGetSize(h, &ws));
            pl.bytes_fft_work += (int64_t)ws;
        }
    }
    pl.bytes_grid = mem.bytes - bytes_before_grid;

    // ---- state
    const int64_t bytes_before_state = mem.bytes;
    {
        T* w = nullptr;
        CK(mem.alloc(&w, (size_t)M * pl.NW));
        pl.d_sigwin = w;
        if (pl.NW == 32) {
            CK(mem.alloc(&w, (size_t)M * 32));
            pl.d_siglin = w;
        }
        pl.n_hist = (P.lag_active && !pl.lag_store) ? P.L + 1 : 1;
        CK(mem.alloc(&w, (size_t)pl.n_hist * M));
        pl.d_sighist = w;
        CK(mem.alloc(&pl.d_sig_in, M));
        CK(mem.alloc(&pl.d_alpha, pl.n_modes));
        CK(mem.alloc(&pl.d_alphad, pl.n_modes));
        C* r = nullptr;
        CK(mem.alloc(&r, (size_t)pl.R_cur * pl.n_modes));
        pl.d_ring = r;
        if (P.lag_active && !pl.lag_store) {
            CK(mem.alloc(&r, (size_t)pl.R_lag * pl.n_modes));
            pl.d_ring_lag = r;
        } else {
            pl.d_ring_lag = pl.d_ring;  // the stored history serves both FIRs (or the lag is inactive)
        }
        CK(mem.alloc(&pl.d_uloc, Mt));
        CK(mem.alloc(&pl.d_uh, 2 * Mt));
        CK(mem.alloc(&pl.d_uself, Mt));
        CK(mem.alloc(&pl.d_u_out, Mt));
    }
    pl.bytes_history += mem.bytes - bytes_before_state;
    CK(mem.alloc(&pl.d_sched, 2));
    CK(cudaStreamCreateWithFlags(&pl.stream2, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&pl.stream3, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&pl.ev_far, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&pl.ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&pl.ev_join, cudaEventDisableTiming));
    CK(cudaHostAlloc(&pl.h_err, sizeof(int), cudaHostAllocMapped));
    *(volatile int*)pl.h_err = 0;
    CK(cudaHostGetDevicePointer((void**)&pl.d_err, pl.h_err, 0));
    local_bulk_setup();
    CK(cudaGetLastError());
    CK(cudaMallocHost(&pl.h_sig, std::max<int64_t>(M, 1) * sizeof(double)));
    CK(cudaMallocHost(&pl.h_u, std::max<int64_t>(Mt, 1) * sizeof(double)));
    CK(cudaEventCreateWithFlags(&pl.ev_out, cudaEventDisableTiming));
    CK(cudaStreamSynchronize(cudaStreamPerThread));

    // ---- spreading autotuner: every candidate tiling gives the same bits (ascending source order
    // per grid point), so the fastest on this device and workload is kept
    {
        struct Cand {
            int ts, ch;
        };
        std::vector<Cand> cands;
        for (int ts : {8, 16, 32})
            if (tile_lists[tile_slot(ts)].made)
                for (int ch : {32, 64})
                    if (pl.opts.spread_chunk == 0 || ch == pl.opts.spread_chunk) cands.push_back({ts, ch});
        size_t best = 0;
        if (cands.size() > 1) {
            Tmp<int> txy[3], tptr[3], tsrc[3];
            for (int i = 0; i < 3; i++)
                if (tile_lists[i].made) {
                    CK(upload_tmp(txy[i], tile_lists[i].txy));
                    CK(upload_tmp(tptr[i], tile_lists[i].tptr));
                    CK(upload_tmp(tsrc[i], tile_lists[i].tsrc));
                }
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            float best_ms = 1e30f;
            for (size_t c = 0; c < cands.size(); c++) {
                const int i = tile_slot(cands[c].ts);
                const int nt = (int)tile_lists[i].txy.size();
                for (int r = 0; r < 7; r++) {
                    if (r == 2) cudaEventRecord(e0, pl.stream);
                    spread_launch(pl, cands[c].ts, cands[c].ch, 0, nt, txy[i].p, tptr[i].p, tsrc[i].p, pl.d_sp_cur,
                                  pl.stream);
                }
                cudaEventRecord(e1, pl.stream);
                CK(cudaEventSynchronize(e1));
                CK(cudaGetLastError());
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            CK(cudaMemsetAsync(pl.d_sp_cur, 0, (size_t)P.nb * P.nf * sizeof(T), pl.stream));
            CK(cudaStreamSynchronize(pl.stream));
        }
        pl.spread_ts = cands[best].ts;
        pl.spread_ch = cands[best].ch;
        const TileLists& tl = tile_lists[tile_slot(pl.spread_ts)];
        pl.n_tiles = (int)tl.txy.size();
        CK(upload(mem, &pl.d_tile_xy, tl.txy));
        CK(upload(mem, &pl.d_tile_ptr, tl.tptr));
        CK(upload(mem, &pl.d_tile_src, tl.tsrc));
        CK(cudaStreamSynchronize(cudaStreamPerThread));
    }

    // ---- local-part autotuner (stored form): all variants give the same bits; keep the fastest
    const int ov = pl.opts.local_variant;
    if (ov < 0 || ov > kLocalVariants) {
        err = "local_variant must be 0 (auto) or 1.." + std::to_string(kLocalVariants);
        return WFP_EINVAL;
    }
    if (pl.local_factored) pl.local_variant = 0;
    if (pl.NW == 32 && Mt > 0 && !pl.local_factored) {
        if (ov > 0) {
            pl.local_variant = ov;
        } else {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            float best_ms = 1e30f;
            for (int v = 1; v <= kLocalVariants; v++) {
                for (int r = 0; r < 6; r++) {
                    if (r == 2) cudaEventRecord(e0, pl.stream);
                    local_launch(pl, v, pl.stream);
                }
                cudaEventRecord(e1, pl.stream);
                CK(cudaEventSynchronize(e1));
                CK(cudaGetLastError());
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best_ms) {
                    best_ms = ms;
                    pl.local_variant = v;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (*(volatile int*)pl.h_err) {
                err = "a bounded device-side wait ran out while timing the local part";
                return WFP_ETIMEOUT;
            }
        }
    }
    return WFP_OK;
}

wfp_status plan_build(Plan& pl, const double* src_xy, const double* tgt_xy, std::string& err) {
    Params& P = pl.P;
    const int64_t M = P.M, Mt = P.Mt;
    // bounding square of all points
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    auto acc = [&](const double* xy, int64_t n) {
        for (int64_t i = 0; i < n; i++) {
            xmin = std::min(xmin, xy[2 * i]);
            xmax = std::max(xmax, xy[2 * i]);
            ymin = std::min(ymin, xy[2 * i + 1]);
            ymax = std::max(ymax, xy[2 * i + 1]);
        }
    };
    acc(src_xy, M);
    acc(tgt_xy, Mt);
    P.cx = 0.5 * (xmin + xmax);
    P.cy = 0.5 * (ymin + ymax);
    double half = 0.5 * std::max(xmax - xmin, ymax - ymin);
    double mag = std::max({std::fabs(xmin), std::fabs(xmax), std::fabs(ymin), std::fabs(ymax), 1e-300});
    half = (half > 1e-12 * mag) ? half * (1.0 + 1e-9) : 1.0;
    wfp_status st = select_params(half, P.dt_user, P.Nt, P.K0_user, P.tol, pl.opts, P, err);
    if (st != WFP_OK) return st;
    P.M = M;
    P.Mt = Mt;
    P.cx = 0.5 * (xmin + xmax);
    P.cy = 0.5 * (ymin + ymax);
    if (P.W > 59) {
        err = "W > 59 is not supported";
        return WFP_EUNSUPPORTED;
    }
    std::vector<double> sxy(2 * M), txy(2 * Mt);
    for (int64_t i = 0; i < M; i++) {
        sxy[2 * i] = (src_xy[2 * i] - P.cx) * P.scale;
        sxy[2 * i + 1] = (src_xy[2 * i + 1] - P.cy) * P.scale;
    }
    for (int64_t i = 0; i < Mt; i++) {
        txy[2 * i] = (tgt_xy[2 * i] - P.cx) * P.scale;
        txy[2 * i + 1] = (tgt_xy[2 * i + 1] - P.cy) * P.scale;
    }
    return P.precision == WFP_FP64 ? build_t<double>(pl, sxy, txy, err) : build_t<float>(pl, sxy, txy, err);
}

void plan_free(Plan& pl) {
    for (int i = 0; i < 4; i++)
        if (pl.graph_exec[i]) cudaGraphExecDestroy(pl.graph_exec[i]);
    prof_collect(pl);
    if (pl.fft_made[0]) cufftDestroy(pl.fftA);
    if (pl.fft_made[1]) cufftDestroy(pl.fftB);
    if (pl.fft_made[2]) cufftDestroy(pl.fftBi);
    if (pl.fft_made[3]) cufftDestroy(pl.fftAi);
    pl.mem.release();
    if (pl.h_sig) cudaFreeHost(pl.h_sig);
    if (pl.h_u) cudaFreeHost(pl.h_u);
    if (pl.h_err) cudaFreeHost(pl.h_err);
    if (pl.ev_out) cudaEventDestroy(pl.ev_out);
    if (pl.ev_fork) cudaEventDestroy(pl.ev_fork);
    if (pl.ev_join) cudaEventDestroy(pl.ev_join);
    if (pl.ev_far) cudaEventDestroy(pl.ev_far);
    if (pl.stream2) cudaStreamDestroy(pl.stream2);
    if (pl.stream3) cudaStreamDestroy(pl.stream3);
    if (pl.own_stream && pl.stream) cudaStreamDestroy(pl.stream);
}

}  // namespace wfp
