// Plan-free evaluation of the local part of the field for one step, without any allocation.
// The paper has no counterpart: this exists for callers of the library, not for the method.
//
// Who needs this: callers that cannot allocate device memory at the time they need the result
// -- code whose device memory all comes from a fixed arena or pool that another part of the
// application reserved up front and that it may not grow, and real-time loops where an
// allocation's latency and the device-wide synchronisation that cudaMalloc and cudaFree can
// cause are not allowed.  wfp_plan_create allocates the plan's tables and state, so such a
// caller cannot use a plan; wfp_local_noalloc gives it the local part of one step instead (the
// same quadrature weights as a plan's local part), for a source/target set that may change
// from call to call.
//
// Scratch: every intermediate (bounding box, per-target pair counts and offsets, the pair
// list, the quadrature weights and the quadrature tables) lives in one file-scope
// `static __device__` array, g_noalloc_scratch, of kScratchBytes bytes.  Every GPU that loads
// this library holds that array until the process exits.  In host code the array's name is
// only a host-side stand-in, so its device address is looked up with cudaGetSymbolAddress once
// per device, by the first call made with that device current, and passed to the kernels.  All
// calls share the array and it keeps the last call's contents: two calls whose work overlaps on
// the GPU (different streams, or different host threads) race on it.  The count of targets that
// coincide with more than one source is cleared by the first kernel of every call; every other
// region is fully written before it is read.
//
// No cudaMalloc / cudaFree / allocating library routine is called, on the device or on the
// host: host-side tables are built in fixed-size static buffers.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "wfp.h"
#include "wfp_internal.h"
#include "wfp_quad.h"

namespace wfp {
void set_error(const std::string& s);
}

using namespace wfp;

namespace {

constexpr int64_t kNaMaxSources = 65536;
constexpr int64_t kNaMaxTargets = 32768;
constexpr int64_t kNaMaxPairs = 65536;
constexpr int kNaLevels = 32;  // weight row length; nmax must not exceed it
constexpr int kNaGL = 20;      // Gauss-Legendre nodes per panel, as in the plan
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kTabDoubles = (size_t)kPhiPanels * (kPhiDeg + 1) + (size_t)kNaLevels * (kLsDeg + 1) + 2 * kNaGL + 32;
constexpr size_t kOffHdr = 0;  // 4 doubles (bounding box), pair total, multiply-coincident target count
constexpr size_t kOffRow = 256;
constexpr size_t kOffCnt = kOffRow + align256((kNaMaxTargets + 1) * sizeof(int64_t));
constexpr size_t kOffCol = kOffCnt + align256(kNaMaxTargets * sizeof(int));
constexpr size_t kOffR = kOffCol + align256(kNaMaxPairs * sizeof(int));
constexpr size_t kOffEta = kOffR + align256(kNaMaxPairs * sizeof(double));
constexpr size_t kOffTab = kOffEta + align256((size_t)kNaMaxPairs * kNaLevels * sizeof(double));
constexpr size_t kScratchBytes = kOffTab + align256(kTabDoubles * sizeof(double));  // ~17 MiB

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_mu;                      // guards the per-device address table and the host tables
void* g_dev_ptr[kMaxDevices] = {};    // device address of g_noalloc_scratch, per device
double g_tab[kTabDoubles];            // host copy of the quadrature tables of the last call
double g_tab_key[6] = {-1, -1, -1, -1, -1, -1};

// bounding box of sources and targets -> hdr[0..3] = xmin, xmax, ymin, ymax (one block); clears
// the count of targets that coincide with more than one source (read back with the pair total)
__global__ void k_na_bbox(int64_t M, const double* __restrict__ src, int64_t Mt, const double* __restrict__ tgt,
                          double* __restrict__ hdr, unsigned long long* __restrict__ n_multi) {
    if (threadIdx.x == 0) *n_multi = 0;
    __shared__ double s[4][256];
    double a = 1e300, b = -1e300, c = 1e300, d = -1e300;
    for (int64_t i = threadIdx.x; i < M + Mt; i += blockDim.x) {
        const double* p = (i < M) ? src + 2 * i : tgt + 2 * (i - M);
        a = fmin(a, p[0]);
        b = fmax(b, p[0]);
        c = fmin(c, p[1]);
        d = fmax(d, p[1]);
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    s[2][threadIdx.x] = c;
    s[3][threadIdx.x] = d;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s[0][threadIdx.x] = fmin(s[0][threadIdx.x], s[0][threadIdx.x + o]);
            s[1][threadIdx.x] = fmax(s[1][threadIdx.x], s[1][threadIdx.x + o]);
            s[2][threadIdx.x] = fmin(s[2][threadIdx.x], s[2][threadIdx.x + o]);
            s[3][threadIdx.x] = fmax(s[3][threadIdx.x], s[3][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) hdr[threadIdx.x] = s[threadIdx.x][0];
}

// pass 0: count pairs 0 < r < delta per target (brute force) and the targets that coincide with
// more than one source (a plan rejects those too); pass 1: write the pairs in source order.  A pair
// is coincident (excluded, as a plan excludes it) when r <= 1e-12 of the bounding square's side.
__global__ void k_na_pairs(int pass, int64_t M, const double* __restrict__ src, int64_t Mt,
                           const double* __restrict__ tgt, double delta, const double* __restrict__ hdr,
                           int* __restrict__ cnt, const int64_t* __restrict__ rowptr, int* __restrict__ col,
                           double* __restrict__ rr, unsigned long long* __restrict__ n_multi) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Mt) return;
    double side = fmax(hdr[1] - hdr[0], hdr[3] - hdr[2]);
    double rc = 1e-12 * side;
    double x = tgt[2 * i], y = tgt[2 * i + 1];
    int64_t o = pass ? rowptr[i] : 0;
    int c = 0, coincident = 0;
    for (int64_t j = 0; j < M; j++) {
        double dx = x - src[2 * j], dy = y - src[2 * j + 1];
        double d2 = dx * dx + dy * dy;
        if (d2 <= rc * rc) coincident++;
        if (d2 <= rc * rc || !(d2 < delta * delta)) continue;
        if (pass) {
            col[o + c] = (int)j;
            rr[o + c] = sqrt(d2);
        }
        c++;
    }
    if (!pass) {
        cnt[i] = c;
        if (coincident > 1) atomicAdd(n_multi, 1ull);
    }
}

// exclusive scan of the per-target counts (one block) -> rowptr[0..Mt], and the pair total
__global__ void k_na_scan(int64_t Mt, const int* __restrict__ cnt, int64_t* __restrict__ rowptr,
                          int64_t* __restrict__ total) {
    __shared__ int64_t part[1024];
    int64_t per = (Mt + blockDim.x - 1) / blockDim.x;
    int64_t a = threadIdx.x * per, b = min(Mt, a + per);
    int64_t s = 0;
    for (int64_t i = a; i < b; i++) s += cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int t = 0; t < (int)blockDim.x; t++) {
            int64_t v = part[t];
            part[t] = run;
            run += v;
        }
        rowptr[Mt] = run;
        *total = run;
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int64_t i = a; i < b; i++) {
        rowptr[i] = run;
        run += cnt[i];
    }
}

__global__ void __launch_bounds__(128) k_na_eta(int64_t npairs, const double* __restrict__ rr, double dt, int W, int p,
                                               int nmax, const double* __restrict__ tab, double* __restrict__ eta) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npairs) return;
    const double* phic = tab;
    const double* cls = phic + (size_t)kPhiPanels * (kPhiDeg + 1);
    const double* gx = cls + (size_t)kNaLevels * (kLsDeg + 1);
    const double* gw = gx + kNaGL;
    const double* wl = gw + kNaGL;
    double e[kMaxLevels];
    eta_weights(rr[k], dt, W, p, nmax, phic, gx, gw, kNaGL, wl, cls, e);
    for (int l = 0; l < kNaLevels; l++) eta[k * kNaLevels + l] = (l < nmax) ? e[l] : 0.0;
}

// u_l(x_i) = sum over pairs of sum_l eta_l sigma_j(level l); one warp per target, lane = level.
// sigma_win is level-major [nmax][M], oldest level first.
__global__ void __launch_bounds__(256) k_na_local(int64_t M, int64_t Mt, int nmax, const int64_t* __restrict__ rowptr,
                                                  const int* __restrict__ col, const double* __restrict__ eta,
                                                  const double* __restrict__ sig, double* __restrict__ u) {
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= Mt) return;
    double acc = 0.0;
    if (lane < nmax)
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) acc = fma(eta[k * kNaLevels + lane], sig[(int64_t)lane * M + col[k]], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) u[i] = acc;
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

wfp_status na_fail(wfp_status s, const char* msg) {
    set_error(msg);
    return s;
}

}  // namespace

extern "C" wfp_status wfp_local_noalloc(int64_t M, const double* src_xy, int64_t Mt, const double* tgt_xy,
                                        const double* sigma_win, int nmax, double dt, double band_limit, double tol,
                                        double* u_local, void* stream) {
    if (M < 1 || Mt < 1) return na_fail(WFP_EINVAL, "wfp_local_noalloc: need M >= 1 and Mt >= 1");
    if (M > kNaMaxSources || Mt > kNaMaxTargets)
        return na_fail(WFP_EINVAL, "wfp_local_noalloc: at most 65536 sources and 32768 targets (fixed scratch)");
    if (!src_xy || !tgt_xy || !sigma_win || !u_local)
        return na_fail(WFP_EINVAL, "wfp_local_noalloc: NULL pointer");
    if (!on_device(src_xy) || !on_device(tgt_xy) || !on_device(sigma_win) || !on_device(u_local))
        return na_fail(WFP_EINVAL, "wfp_local_noalloc: src_xy, tgt_xy, sigma_win and u_local must be device memory");
    wfp_opts o;
    wfp_opts_default(&o);
    double eps;
    int W, p, nm;
    const char* why = "";
    wfp_status st = local_params(dt, band_limit, tol, o, &eps, &W, &p, &nm, &why);
    if (st != WFP_OK) return na_fail(st, why);
    if (nm > kNaLevels) return na_fail(WFP_EUNSUPPORTED, "wfp_local_noalloc: more than 32 stored levels needed");
    if (nmax != nm) return na_fail(WFP_EINVAL, "wfp_local_noalloc: nmax does not match W + 1 + p/2 for dt, band_limit, tol");
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return na_fail(WFP_ECUDA, "wfp_local_noalloc: cudaGetDevice failed");
    if (!g_dev_ptr[dev]) {  // once per device, with that device current
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return na_fail(WFP_ECUDA, "wfp_local_noalloc: cudaGetSymbolAddress of the scratch array failed");
        }
        g_dev_ptr[dev] = ptr;
    }
    unsigned char* base = (unsigned char*)g_dev_ptr[dev];
    double* hdr = (double*)(base + kOffHdr);
    int64_t* d_total = (int64_t*)(base + kOffHdr + 4 * sizeof(double));
    unsigned long long* d_multi = (unsigned long long*)(d_total + 1);  // read back with d_total
    int64_t* rowptr = (int64_t*)(base + kOffRow);
    int* cnt = (int*)(base + kOffCnt);
    int* col = (int*)(base + kOffCol);
    double* rr = (double*)(base + kOffR);
    double* eta = (double*)(base + kOffEta);
    double* tab = (double*)(base + kOffTab);
    // quadrature tables (host, fixed-size buffers), rebuilt when the parameters change
    double key[6] = {eps, (double)W, (double)p, dt, band_limit, (double)nm};
    if (std::memcmp(key, g_tab_key, sizeof(key)) != 0) {
        double* phic = g_tab;
        double* cls = phic + (size_t)kPhiPanels * (kPhiDeg + 1);
        double* gx = cls + (size_t)kNaLevels * (kLsDeg + 1);
        double* gw = gx + kNaGL;
        double* wl = gw + kNaGL;
        build_phi_table_into(std::log(1.0 / eps), phic);
        build_ls_cheb_into(nm, dt, std::max(band_limit, 1e-3 / dt), kLsIntervals * dt, cls);
        gauss_legendre(kNaGL, gx, gw);
        lagrange_ref_weights(p, wl);
        std::memcpy(g_tab_key, key, sizeof(key));
    }
    const double delta = W * dt;
    cudaError_t e = cudaMemcpyAsync(tab, g_tab, sizeof(g_tab), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return na_fail(WFP_ECUDA, "wfp_local_noalloc: table upload failed");
    k_na_bbox<<<1, 256, 0, s>>>(M, src_xy, Mt, tgt_xy, hdr, d_multi);
    k_na_pairs<<<(unsigned)((Mt + 127) / 128), 128, 0, s>>>(0, M, src_xy, Mt, tgt_xy, delta, hdr, cnt, nullptr,
                                                            nullptr, nullptr, d_multi);
    k_na_scan<<<1, 1024, 0, s>>>(Mt, cnt, rowptr, d_total);
    int64_t counts[2] = {-1, -1};  // pair total, targets coinciding with more than one source
    e = cudaMemcpyAsync(counts, d_total, sizeof(counts), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return na_fail(WFP_ECUDA, "wfp_local_noalloc: pair count failed");
    const int64_t total = counts[0];
    if (counts[1] != 0)
        return na_fail(WFP_EUNSUPPORTED, "wfp_local_noalloc: a target coincides with more than one source");
    if (total > kNaMaxPairs)
        return na_fail(WFP_EINVAL, "wfp_local_noalloc: more than 65536 local pairs (fixed scratch); split the targets");
    k_na_pairs<<<(unsigned)((Mt + 127) / 128), 128, 0, s>>>(1, M, src_xy, Mt, tgt_xy, delta, hdr, cnt, rowptr, col,
                                                            rr, d_multi);
    if (total > 0) k_na_eta<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(total, rr, dt, W, p, nm, tab, eta);
    k_na_local<<<(unsigned)((Mt * 32 + 255) / 256), 256, 0, s>>>(M, Mt, nm, rowptr, col, eta, sigma_win, u_local);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(WFP_ECUDA, "wfp_local_noalloc: kernel launch failed");
    return WFP_OK;
}
