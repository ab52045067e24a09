// Kernels of the local part of the 2D TK-WFP step (Sec. 6, Eq. ul) on sm_103a; launched from
// wfp_local.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "wfp_dev.h"
#include "wfp_ptx.h"

namespace wfp {

// ------------------------------------------------------------------------------- local part
// u_l(x_i, t_n) = sum_{j in N_delta(i)} sum_{l=1}^{nmax} eta_l(r_ij) sigma_j(t_{n-nmax+l})  (Sec. 6)
// One warp per target row; lane = time level, so each pair's weight row and each source's
// sigma window are read as contiguous 32-element segments.  eta carries the 1/(2 pi).  This form
// serves windows of 64 levels (nmax > 32); k_local_vec below serves nmax <= 32.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

template <typename T>
__global__ void __launch_bounds__(256) k_local(const int64_t* __restrict__ d_step, int64_t Mt,
                                               const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                                               const T* __restrict__ eta, const T* __restrict__ sigwin, int NW,
                                               int nmax, double* __restrict__ uloc) {
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= Mt) return;
    int64_t n = *d_step + 1;
    int64_t p0 = rowptr[row], p1 = rowptr[row + 1];
    int s0 = (int)((n - nmax + 1 + lane) & (NW - 1));
    int s1 = (int)((n - nmax + 1 + lane + 32) & (NW - 1));
    double tot;
    if constexpr (sizeof(T) == 8) {
        double acc = 0.0;
        int64_t p = p0;
        for (; p + 1 < p1; p += 2) {
            int j0 = col[p], j1 = col[p + 1];
            double e0 = eta[p * NW + lane], e1 = eta[(p + 1) * NW + lane];
            double x0 = sigwin[(int64_t)j0 * NW + s0], x1 = sigwin[(int64_t)j1 * NW + s0];
            acc = fma(e0, x0, acc);
            acc = fma(e1, x1, acc);
            if (NW == 64) {
                acc = fma(eta[p * NW + lane + 32], sigwin[(int64_t)j0 * NW + s1], acc);
                acc = fma(eta[(p + 1) * NW + lane + 32], sigwin[(int64_t)j1 * NW + s1], acc);
            }
        }
        if (p < p1) {
            int j0 = col[p];
            acc = fma(eta[p * NW + lane], sigwin[(int64_t)j0 * NW + s0], acc);
            if (NW == 64) acc = fma(eta[p * NW + lane + 32], sigwin[(int64_t)j0 * NW + s1], acc);
        }
        tot = acc;
    } else {
        // FP32 products, compensated FP32 accumulation per lane, FP64 across lanes
        float s = 0.f, c = 0.f;
        int64_t p = p0;
        for (; p + 1 < p1; p += 2) {
            int j0 = col[p], j1 = col[p + 1];
            float e0 = eta[p * NW + lane], e1 = eta[(p + 1) * NW + lane];
            float x0 = sigwin[(int64_t)j0 * NW + s0], x1 = sigwin[(int64_t)j1 * NW + s0];
            kahan_add(s, c, e0 * x0);
            kahan_add(s, c, e1 * x1);
            if (NW == 64) {
                kahan_add(s, c, eta[p * NW + lane + 32] * sigwin[(int64_t)j0 * NW + s1]);
                kahan_add(s, c, eta[(p + 1) * NW + lane + 32] * sigwin[(int64_t)j1 * NW + s1]);
            }
        }
        if (p < p1) {
            int j0 = col[p];
            kahan_add(s, c, eta[p * NW + lane] * sigwin[(int64_t)j0 * NW + s0]);
            if (NW == 64) kahan_add(s, c, eta[p * NW + lane + 32] * sigwin[(int64_t)j0 * NW + s1]);
        }
        tot = (double)s - (double)c;
    }
    tot = warp_sum(tot);
    if (lane == 0) uloc[row] = tot;
}

// Vectorised local part (NW = 32): eta rows are aligned with the linear window, so a pair is a dot
// product of two 32-level rows read as 16-byte vectors: LP lanes per pair (8 in FP32, 16 in FP64),
// 32/LP pairs per warp load, four such groups in flight per iteration.  Weights are streamed
// (read once); the windows are gathered from L2.
template <typename T>
__global__ void __launch_bounds__(256) k_local_vec(int64_t Mt, const int64_t* __restrict__ rowptr,
                                                   const int* __restrict__ col, const T* __restrict__ eta,
                                                   const T* __restrict__ siglin, double* __restrict__ uloc) {
    using V = typename Vec16<T>::type;
    constexpr int LP = 32 * sizeof(T) / 16;  // lanes per pair
    constexpr int PW = 32 / LP;              // pairs per warp load
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= Mt) return;
    const int c = lane % LP, g = lane / LP;
    const int64_t p0 = rowptr[row], p1 = rowptr[row + 1];
    const V* E = (const V*)eta;
    const V* X = (const V*)siglin;
    double tot;
    if constexpr (sizeof(T) == 8) {
        double a0 = 0.0, a1 = 0.0;
        int64_t p = p0 + g;
        for (; p + 3 * PW < p1; p += 4 * PW) {
            const int j0 = col[p], j1 = col[p + PW], j2 = col[p + 2 * PW], j3 = col[p + 3 * PW];
            const V e0 = __ldcs(E + p * LP + c), e1 = __ldcs(E + (p + PW) * LP + c);
            const V e2 = __ldcs(E + (p + 2 * PW) * LP + c), e3 = __ldcs(E + (p + 3 * PW) * LP + c);
            const V x0 = __ldg(X + (int64_t)j0 * LP + c), x1 = __ldg(X + (int64_t)j1 * LP + c);
            const V x2 = __ldg(X + (int64_t)j2 * LP + c), x3 = __ldg(X + (int64_t)j3 * LP + c);
            a0 = fma(e0.x, x0.x, a0);
            a1 = fma(e0.y, x0.y, a1);
            a0 = fma(e1.x, x1.x, a0);
            a1 = fma(e1.y, x1.y, a1);
            a0 = fma(e2.x, x2.x, a0);
            a1 = fma(e2.y, x2.y, a1);
            a0 = fma(e3.x, x3.x, a0);
            a1 = fma(e3.y, x3.y, a1);
        }
        for (; p < p1; p += PW) {
            const V e = __ldcs(E + p * LP + c), x = __ldg(X + (int64_t)col[p] * LP + c);
            a0 = fma(e.x, x.x, a0);
            a1 = fma(e.y, x.y, a1);
        }
        tot = a0 + a1;
    } else {
        // FP32 products, compensated FP32 accumulation per lane, FP64 across lanes
        float sm = 0.f, cm = 0.f;
        int64_t p = p0 + g;
        for (; p + 3 * PW < p1; p += 4 * PW) {
            const int j0 = col[p], j1 = col[p + PW], j2 = col[p + 2 * PW], j3 = col[p + 3 * PW];
            const V e0 = __ldcs(E + p * LP + c), e1 = __ldcs(E + (p + PW) * LP + c);
            const V e2 = __ldcs(E + (p + 2 * PW) * LP + c), e3 = __ldcs(E + (p + 3 * PW) * LP + c);
            const V x0 = __ldg(X + (int64_t)j0 * LP + c), x1 = __ldg(X + (int64_t)j1 * LP + c);
            const V x2 = __ldg(X + (int64_t)j2 * LP + c), x3 = __ldg(X + (int64_t)j3 * LP + c);
            kahan_add(sm, cm, fmaf(e0.w, x0.w, fmaf(e0.z, x0.z, fmaf(e0.y, x0.y, e0.x * x0.x))));
            kahan_add(sm, cm, fmaf(e1.w, x1.w, fmaf(e1.z, x1.z, fmaf(e1.y, x1.y, e1.x * x1.x))));
            kahan_add(sm, cm, fmaf(e2.w, x2.w, fmaf(e2.z, x2.z, fmaf(e2.y, x2.y, e2.x * x2.x))));
            kahan_add(sm, cm, fmaf(e3.w, x3.w, fmaf(e3.z, x3.z, fmaf(e3.y, x3.y, e3.x * x3.x))));
        }
        for (; p < p1; p += PW) {
            const V e = __ldcs(E + p * LP + c), x = __ldg(X + (int64_t)col[p] * LP + c);
            kahan_add(sm, cm, fmaf(e.w, x.w, fmaf(e.z, x.z, fmaf(e.y, x.y, e.x * x.x))));
        }
        tot = (double)sm - (double)cm;
    }
    tot = warp_sum(tot);
    if (lane == 0) uloc[row] = tot;
}

// Local part with the weight stream staged by bulk asynchronous copies (the form used on sm_103a
// for nmax <= 32).  A persistent grid (as many CTAs as fit at once) whose warps take target rows
// from a counter: lane 0 keeps S stages of CH pair slots of the row (their weight rows and source
// indices, contiguous in HBM) in flight into a per-warp shared-memory ring, each stage completed on
// its own mbarrier; the lanes consume a stage as in k_local_vec (weights from shared memory,
// windows gathered from L2) and lane 0 refills the buffer with the stage S ahead.  Rows are padded
// to multiples of 4 slots, so every copy is 16-byte aligned and sized.  The last warp to finish
// resets the counter for the next launch.  A wait that runs out sets *err (host-mapped); the warp
// drains its copies and stops.
constexpr uint64_t kBulkWaitNs = 2000000000ull;  // 2 s

template <typename T, int CH, int S, int WARPS_>
struct LocalBulk {
    static constexpr uint32_t ROWB = 32 * sizeof(T);          // bytes of one weight row
    static constexpr uint32_t STAGE = CH * ROWB + CH * 4;     // weights + indices
    static constexpr uint32_t WARPB = S * STAGE + S * 8;      // stages + mbarriers
    static constexpr int WARPS = WARPS_;
    static constexpr uint32_t SMEM = WARPS * WARPB;
};

// Every variant (k_local_vec and each staged configuration) gives lane (c, g) the pairs g, g + PW,
// g + 2 PW, ... of its row in that order with the same per-pair arithmetic, and each row is summed
// by one warp, so all produce the same bits and the plan-time autotuner may pick any of them.
template <typename T, int CH, int S, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_local_bulk(int64_t Mt, const int64_t* __restrict__ rowptr,
                                                    const int* __restrict__ col, const T* __restrict__ eta,
                                                    const T* __restrict__ siglin, double* __restrict__ uloc,
                                                    int* err, int* sched) {
    using V = typename Vec16<T>::type;
    using G = LocalBulk<T, CH, S, WARPS>;
    constexpr int LP = 32 * sizeof(T) / 16;  // lanes per pair
    constexpr int PW = 32 / LP;              // pairs per warp load
    static_assert(CH % 4 == 0 && CH % PW == 0, "stage must hold whole 4-slot groups");
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* base = smem + warp * G::WARPB;
    uint64_t* bar = (uint64_t*)(base + S * G::STAGE);
    if (lane == 0) {
        for (int s = 0; s < S; s++) mbar_init(bar + s, 1);
        fence_mbar_init();
    }
    __syncwarp();
    const int c = lane % LP, g = lane / LP;
    const V* X = (const V*)siglin;
    uint32_t kk = 0;  // stages this warp has consumed: stage kk goes to buffer kk % S, phase (kk / S) & 1
    for (;;) {
        int row = 0;
        if (lane == 0) row = atomicAdd(sched, 1);
        row = __shfl_sync(0xffffffffu, row, 0);
        if ((int64_t)row >= Mt) break;
        const int64_t p0 = rowptr[row], p1 = rowptr[row + 1];
        const int nst = (int)((p1 - p0 + CH - 1) / CH);
        auto issue = [&](int k) {  // stage k of the row (lane 0)
            const int b = (int)((kk + k) % S);
            const int64_t q0 = p0 + (int64_t)k * CH;
            const uint32_t np = (uint32_t)min((int64_t)CH, p1 - q0);
            unsigned char* dst = base + b * G::STAGE;
            mbar_expect_tx(bar + b, np * G::ROWB + np * 4);
            bulk_g2s(dst, eta + q0 * 32, np * G::ROWB, bar + b);
            bulk_g2s(dst + CH * G::ROWB, col + q0, np * 4, bar + b);
        };
        if (lane == 0)
            for (int k = 0; k < min(S, nst); k++) issue(k);
        double d0 = 0.0, d1 = 0.0;  // FP64 path (as k_local_vec)
        float sm = 0.f, cm = 0.f;   // FP32 path: compensated sum
        int k = 0;
        for (; k < nst; k++) {
            const uint32_t idx = kk + k;
            const int b = (int)(idx % S);
            const bool ok = mbar_wait_bounded(bar + b, (idx / S) & 1, kBulkWaitNs);
            if (!__all_sync(0xffffffffu, ok)) break;
            const int np = (int)min((int64_t)CH, p1 - p0 - (int64_t)k * CH);
            const V* E = (const V*)(base + b * G::STAGE);
            const int* C = (const int*)(base + b * G::STAGE + CH * G::ROWB);
#pragma unroll 4
            for (int q = g; q < np; q += PW) {
                const V e = E[q * LP + c];
                const V x = __ldg(X + (int64_t)C[q] * LP + c);
                if constexpr (sizeof(T) == 8) {
                    d0 = fma(e.x, x.x, d0);
                    d1 = fma(e.y, x.y, d1);
                } else {
                    kahan_add(sm, cm, fmaf(e.w, x.w, fmaf(e.z, x.z, fmaf(e.y, x.y, e.x * x.x))));
                }
            }
            __syncwarp();
            if (lane == 0 && k + S < nst) {
                fence_proxy_async_smem();
                issue(k + S);
            }
        }
        if (k < nst) {  // a wait ran out: record it, let the copies in flight land, leave the row unset
            if (lane == 0) *(volatile int*)err = 1;
            for (int j = k; j < min(nst, k + S); j++)
                mbar_wait_bounded(bar + (kk + j) % S, ((kk + j) / S) & 1, kBulkWaitNs);
            __syncwarp();
            break;
        }
        kk += nst;
        double tot;
        if constexpr (sizeof(T) == 8)
            tot = d0 + d1;
        else
            tot = (double)sm - (double)cm;
        tot = warp_sum(tot);
        if (lane == 0) uloc[row] = tot;
    }
    // every warp counts itself out; the last one resets the row counter for the next launch
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(sched + 1, 1) == (int)(gridDim.x * WARPS) - 1) {
            sched[0] = 0;
            sched[1] = 0;
            __threadfence();
        }
    }
}

}  // namespace wfp
