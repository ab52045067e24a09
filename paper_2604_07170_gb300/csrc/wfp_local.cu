// Local part of the 2D TK-WFP step (Sec. 6, Eq. ul) on sm_103a:
//   u_l(x_i, t_n) = sum_{j in N_delta(i)} sum_{l=1}^{nmax} eta_l(r_ij) sigma_j(t_{n-nmax+l}),
// a CSR stream of per-pair weight rows against per-source windows of the newest signal levels.
// Launchers of the kernels in wfp_local_kernels.cuh (variants, persistent grid sizing, the
// autotuner's entry point) and the bounded-wait probe.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <string>

#include "wfp_debug.h"
#include "wfp_dev.h"
#include "wfp_local_factored.cuh"
#include "wfp_local_kernels.cuh"
#include "wfp_plan.h"
#include "wfp_ptx.h"

namespace wfp {

static inline unsigned nblk_u(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Local-part variants: 1 = k_local_vec; 2.. = staged configurations (CH slots per stage, S stages,
// WARPS warps per CTA), chosen per precision so that a stage is 2-4 KB of weights.
template <typename T, int CH, int S, int WARPS>
static void bulk_one(const Plan& pl, cudaStream_t st) {
    using G = LocalBulk<T, CH, S, WARPS>;
    // persistent grid: the CTAs that fit on the device at once (found once per kernel instance;
    // plans are built on several threads, so the cached value is atomic)
    static std::atomic<int> fit_cache{0};
    int fit = fit_cache.load(std::memory_order_relaxed);
    if (fit == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_local_bulk<T, CH, S, WARPS>, WARPS * 32, G::SMEM);
        fit = std::max(1, sms * std::max(per - 1, 1));  // one CTA slot per SM left to the advance stream
        fit_cache.store(fit, std::memory_order_relaxed);
    }
    const int64_t need = (pl.Mt + WARPS - 1) / WARPS;
    k_local_bulk<T, CH, S, WARPS><<<(unsigned)std::min<int64_t>(need, fit), WARPS * 32, G::SMEM, st>>>(
        pl.Mt, pl.d_rowptr, pl.d_col, (const T*)pl.d_eta, (const T*)pl.d_siglin, pl.d_uloc, pl.d_err, pl.d_sched);
}
template <typename T, int CH, int S, int WARPS>
static void bulk_attr() {
    cudaFuncSetAttribute(k_local_bulk<T, CH, S, WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         LocalBulk<T, CH, S, WARPS>::SMEM);
}

template <typename T>
static void local_variant_t(const Plan& pl, int v, cudaStream_t st) {
    constexpr bool D = sizeof(T) == 8;
    switch (v) {
        case 1:
            k_local_vec<T><<<nblk_u(pl.Mt * 32, 256), 256, 0, st>>>(pl.Mt, pl.d_rowptr, pl.d_col, (const T*)pl.d_eta,
                                                                    (const T*)pl.d_siglin, pl.d_uloc);
            break;
        case 2: bulk_one<T, D ? 16 : 32, 4, 4>(pl, st); break;
        case 3: bulk_one<T, D ? 8 : 16, 4, 8>(pl, st); break;
        case 4: bulk_one<T, D ? 8 : 16, 8, 4>(pl, st); break;
        default: bulk_one<T, D ? 8 : 16, 2, 16>(pl, st); break;
    }
}

template <typename T>
static void local_attrs_t() {
    constexpr bool D = sizeof(T) == 8;
    bulk_attr<T, D ? 16 : 32, 4, 4>();
    bulk_attr<T, D ? 8 : 16, 4, 8>();
    bulk_attr<T, D ? 8 : 16, 8, 4>();
    bulk_attr<T, D ? 8 : 16, 2, 16>();
}

// the resident-coefficient contraction takes up to this much dynamic shared memory (two CTAs per SM
// or more; above it, the interval-split contraction, which gives the same bits)
constexpr int kY5MaxSmem = 100 * 1024;

void local_bulk_setup() {
    local_attrs_t<double>();
    local_attrs_t<float>();
    cudaFuncSetAttribute(k_ycoef5<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kY5MaxSmem);
    cudaFuncSetAttribute(k_ycoef5<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kY5MaxSmem);
}

void local_launch(const Plan& pl, int variant, cudaStream_t st) {
    if (pl.P.precision == WFP_FP64)
        local_variant_t<double>(pl, variant, st);
    else
        local_variant_t<float>(pl, variant, st);
}

// Factored form: the per-step contraction of the windows, then the pair sums.
template <typename T, int NC>
static void factored_nc(const Plan& pl, cudaStream_t st) {
    const int nk = pl.P.W - 1;
    if constexpr (sizeof(T) == 8) {
        k_ycoef<T, NC><<<dim3(nblk_u(pl.M, 128), (unsigned)nk), 128, 0, st>>>(pl.M, (const T*)pl.d_siglin,
                                                                            (const T*)pl.d_ctab, (T*)pl.d_ycoef);
        k_local_cheb<T, NC><<<nblk_u(pl.Mt * 32, 256), 256, 0, st>>>(
            pl.Mt, pl.d_trow, (const TabPair<T>*)pl.d_tpair, (const T*)pl.d_ycoef, pl.d_rowptr, pl.d_col,
            (const T*)pl.d_eta, (const T*)pl.d_siglin, pl.d_uloc);
    } else {
        // k_ycoef5 gives every block 256 sources: below one block per SM (10^4 points: 40 blocks) the
        // interval-split k_ycoef4 fills the device better; both give the same bits
        static std::atomic<int> sm_count{0};
        int sms = sm_count.load(std::memory_order_relaxed);
        if (sms == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            sm_count.store(sms, std::memory_order_relaxed);
        }
        const size_t smem = (size_t)nk * 32 * NC * sizeof(float);
        if (smem <= (size_t)kY5MaxSmem && (int64_t)nblk_u(pl.M, 2 * kY5Threads) >= sms) {
            // every interval's coefficients fit in shared memory, and the grid fills the device
            k_ycoef5<NC><<<nblk_u(pl.M, 2 * kY5Threads), kY5Threads, smem, st>>>(
                pl.M, nk, (const float*)pl.d_siglin, (const float*)pl.d_ctab, (float*)pl.d_ycoef);
        } else {
            constexpr int KC = 64 / NC;  // intervals per block of k_ycoef4
            k_ycoef4<NC><<<nblk_u(pl.M, 32) * (unsigned)((nk + KC - 1) / KC), 128, 0, st>>>(
                pl.M, nk, (const float*)pl.d_siglin, (const float*)pl.d_ctab, (float*)pl.d_ycoef);
        }
        k_local_cheb2<NC><<<nblk_u(pl.Mt * 32, 256), 256, 0, st>>>(
            pl.Mt, pl.d_trow, (const TabPair<float>*)pl.d_tpair, (const float*)pl.d_ycoef, pl.d_rowptr,
            pl.d_col, (const float*)pl.d_eta, (const float*)pl.d_siglin, pl.d_uloc);
    }
}

static void factored_run(const Plan& pl, cudaStream_t st) {
    if (pl.P.precision == WFP_FP64)
        factored_nc<double, 36>(pl, st);
    else if (pl.NC == 16)
        factored_nc<float, 16>(pl, st);
    else
        factored_nc<float, 32>(pl, st);
}

// coefficient counts the factored kernels are built for: all 33 (padded to 36) in FP64; blocks of
// 16 or 32 in FP32
int factored_nc_supported(int nc, bool fp64) {
    if (fp64) return 36;
    return nc <= 16 ? 16 : 32;
}

// Local part of the current step into pl.d_uloc (the factored form; or, with stored weight rows,
// k_local for 64-level windows and otherwise the variant chosen at plan time).
void local_run(const Plan& pl, cudaStream_t st) {
    if (pl.local_factored) {
        factored_run(pl, st);
    } else if (pl.NW == 32) {
        local_launch(pl, pl.local_variant, st);
    } else if (pl.P.precision == WFP_FP64) {
        k_local<double><<<nblk_u(pl.Mt * 32, 256), 256, 0, st>>>(pl.d_step, pl.Mt, pl.d_rowptr, pl.d_col,
                                                                 (const double*)pl.d_eta, (const double*)pl.d_sigwin,
                                                                 pl.NW, pl.P.nmax, pl.d_uloc);
    } else {
        k_local<float><<<nblk_u(pl.Mt * 32, 256), 256, 0, st>>>(pl.d_step, pl.Mt, pl.d_rowptr, pl.d_col,
                                                                (const float*)pl.d_eta, (const float*)pl.d_sigwin,
                                                                pl.NW, pl.P.nmax, pl.d_uloc);
    }
}


// one warp: wait on an mbarrier of its own shared memory with the bounded wait (see wfp_debug.h)
__global__ void k_wait_probe(uint64_t limit_ns, int arrive, int* timed_out, unsigned long long* waited_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (arrive && threadIdx.x == 0) mbar_arrive(&bar);
    __syncwarp();
    const uint64_t t0 = global_ns();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    const uint64_t t1 = global_ns();
    if (threadIdx.x == 0) {
        *timed_out = ok ? 0 : 1;
        *waited_ns = (unsigned long long)(t1 - t0);
    }
}

}  // namespace wfp

extern "C" wfp_status wfp_debug_bounded_wait(double limit_s, int arrive, int* timed_out, double* waited_s) {
    if (!timed_out || !waited_s || !(limit_s >= 1e-3 && limit_s <= 1.0)) {
        wfp::set_error("limit_s must be in [0.001, 1] and the outputs non-NULL");
        return WFP_EINVAL;
    }
    int* d_to = nullptr;
    unsigned long long* d_w = nullptr;
    if (cudaMalloc(&d_to, sizeof(int)) != cudaSuccess || cudaMalloc(&d_w, sizeof(unsigned long long)) != cudaSuccess) {
        cudaFree(d_to);
        cudaGetLastError();
        wfp::set_error("device allocation failed");
        return WFP_ECUDA;
    }
    wfp::k_wait_probe<<<1, 32>>>((uint64_t)(limit_s * 1e9), arrive ? 1 : 0, d_to, d_w);
    unsigned long long w = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(timed_out, d_to, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&w, d_w, sizeof(w), cudaMemcpyDeviceToHost);
    cudaFree(d_to);
    cudaFree(d_w);
    if (e != cudaSuccess) {
        wfp::set_error(std::string("bounded-wait probe: ") + cudaGetErrorString(e));
        return WFP_ECUDA;
    }
    *waited_s = (double)w * 1e-9;
    return WFP_OK;
}
