// Factored local part of the 2D TK-WFP step (Sec. 6, Eq. ul) on sm_103a; launched from
// wfp_local.cu.  The pair records are also written at plan time (wfp_plan.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "wfp_dev.h"
#include "wfp_local_kernels.cuh"

namespace wfp {

// One pair of the factored local part: the index (k - 1) M + j of its source's coefficient block
// for delay interval k, and the interval's Chebyshev variable x = 2 sqrt(((k+1) dt - r) / dt) - 1.
template <typename T>
struct TabPair;
template <>
struct __align__(8) TabPair<float> {
    unsigned blk;
    float x;
};
template <>
struct __align__(16) TabPair<double> {
    unsigned blk, pad;
    double x;
};

// ------------------------------------------------------------------ factored local part
// On a delay interval [k dt, (k+1) dt], k >= 1, each weight is a Chebyshev series in the interval's
// variable x(r): eta_l(r) = sum_c C[k][l][c] T_c(x(r)).  Summing over the levels first,
//   sum_l eta_l(r_ij) sigma_j,l = sum_c T_c(x_ij) y[k][j][c],   y[k][j][c] = sum_l C[k][l][c] sigma_j,l,
// so one contraction per source and interval per step (k_ycoef5 or k_ycoef4; k_ycoef in FP64) replaces a weight
// row per pair, and a pair needs only its block index and x: 8 bytes instead of 32 weights.  y holds
// sources x intervals x NC values; the pairs of neighbouring targets gather the same blocks, mostly
// from L2.

template <typename T>
__device__ __forceinline__ void unpack16(const typename Vec16<T>::type& q, T* out);
template <>
__device__ __forceinline__ void unpack16<float>(const float4& q, float* out) {
    out[0] = q.x;
    out[1] = q.y;
    out[2] = q.z;
    out[3] = q.w;
}
template <>
__device__ __forceinline__ void unpack16<double>(const double2& q, double* out) {
    out[0] = q.x;
    out[1] = q.y;
}

// y[kk][j][c] = sum_i ctab[kk][i][c] siglin[j][i] (window position i = 32 - nmax + l holds level l;
// the coefficients of the unused positions are zero).  The FP64 form (all 33 coefficients, used to
// check the factoring against the stored rows): thread = source, blockIdx.y = interval; the
// interval's coefficients are staged in shared memory and read as warp-uniform broadcasts.
template <typename T, int NC>
__global__ void __launch_bounds__(128) k_ycoef(int64_t M, const T* __restrict__ siglin, const T* __restrict__ ctab,
                                               T* __restrict__ y) {
    using V = typename Vec16<T>::type;
    constexpr int EV = 16 / (int)sizeof(T);
    __shared__ __align__(16) T sc[32 * NC];
    const int kk = blockIdx.y;
    for (int t = threadIdx.x; t < 32 * NC; t += blockDim.x) sc[t] = ctab[(int64_t)kk * 32 * NC + t];
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    T s[32];
    const V* sp = (const V*)(siglin + j * 32);
#pragma unroll
    for (int v = 0; v < 32 / EV; v++) unpack16<T>(__ldg(sp + v), s + v * EV);
    V* out = (V*)(y + ((int64_t)kk * M + j) * NC);
#pragma unroll
    for (int c0 = 0; c0 < NC; c0 += 4) {
        T a[4] = {0, 0, 0, 0};
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const T* cr = sc + i * NC + c0;
#pragma unroll
            for (int q = 0; q < 4; q++) a[q] = fma(cr[q], s[i], a[q]);
        }
        if constexpr (sizeof(T) == 4) {
            out[c0 / 4] = make_float4(a[0], a[1], a[2], a[3]);
        } else {
            out[c0 / 2] = make_double2(a[0], a[1]);
            out[c0 / 2 + 1] = make_double2(a[2], a[3]);
        }
    }
}

// sum_c T_c(x) yy[c], with T_c by the three-term recurrence T_{c+1} = 2x T_c - T_{c-1} (even and odd
// terms in two partial sums)
template <typename T, int NC>
__device__ __forceinline__ T cheb_dot(T x, const T* yy) {
    const T x2 = x + x;
    T tm = 1, tc = x;
    T s0 = yy[0], s1 = yy[1] * x;
#pragma unroll
    for (int c = 2; c < NC; c++) {
        const T tn = fma(x2, tc, -tm);
        if (c & 1)
            s1 = fma(tn, yy[c], s1);
        else
            s0 = fma(tn, yy[c], s0);
        tm = tc;
        tc = tn;
    }
    return s0 + s1;
}

// streamed (read-once) load of a pair record
__device__ __forceinline__ TabPair<float> load_pair(const TabPair<float>* p) {
    const uint2 q = __ldcs((const uint2*)p);
    return TabPair<float>{q.x, __uint_as_float(q.y)};
}
__device__ __forceinline__ TabPair<double> load_pair(const TabPair<double>* p) {
    const double2 q = __ldcs((const double2*)p);
    return TabPair<double>{(unsigned)(unsigned long long)__double_as_longlong(q.x), 0u, q.y};
}

template <typename T, int NC>
__device__ __forceinline__ T tab_pair_value(const TabPair<T>& e, const T* __restrict__ y) {
    using V = typename Vec16<T>::type;
    constexpr int EV = 16 / (int)sizeof(T);
    const V* yb = (const V*)(y + (int64_t)e.blk * NC);
    T yy[NC];
#pragma unroll
    for (int v = 0; v < NC / EV; v++) unpack16<T>(__ldg(yb + v), yy + v * EV);
    return cheb_dot<T, NC>(e.x, yy);
}

// FP64 form (coefficients in natural order): one warp per target row, one lane per pair (the row's
// table pairs 32 apart), then its near pairs (r < dt, stored 32-level rows against the source's
// window), one lane each.
template <typename T, int NC>
__global__ void __launch_bounds__(256) k_local_cheb(int64_t Mt, const int64_t* __restrict__ trow,
                                                    const TabPair<T>* __restrict__ tp, const T* __restrict__ y,
                                                    const int64_t* __restrict__ nrow, const int* __restrict__ ncol,
                                                    const T* __restrict__ neta, const T* __restrict__ siglin,
                                                    double* __restrict__ uloc) {
    using V = typename Vec16<T>::type;
    constexpr int EV = 16 / (int)sizeof(T);
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= Mt) return;
    static_assert(sizeof(T) == 8, "the FP32 form is k_local_cheb2");
    double d = 0.0;
    const int64_t p1 = trow[row + 1];
    for (int64_t p = trow[row] + lane; p < p1; p += 32) d += tab_pair_value<T, NC>(load_pair(tp + p), y);
    for (int64_t q = nrow[row] + lane; q < nrow[row + 1]; q += 32) {
        const V* E = (const V*)(neta + q * 32);
        const V* X = (const V*)(siglin + (int64_t)ncol[q] * 32);
        T a0 = 0, a1 = 0;
#pragma unroll
        for (int v = 0; v < 32 / EV; v++) {
            T e[EV], x[EV];
            unpack16<T>(__ldcs(E + v), e);
            unpack16<T>(__ldg(X + v), x);
#pragma unroll
            for (int u = 0; u < EV; u += 2) {
                a0 = fma(e[u], x[u], a0);
                a1 = fma(e[u + 1], x[u + 1], a1);
            }
        }
        d += a0 + a1;
    }
    const double tot = warp_sum(d);
    if (lane == 0) uloc[row] = tot;
}


// FP32 form.  A pair's y block (NC = 16 or 32 floats, 64 or 128 contiguous bytes) is read by two
// lanes with 32-byte loads, so a warp load gathers sixteen whole 64-byte blocks (sixteen L1
// wavefronts for sixteen pairs).  The block is stored lane-interleaved by coefficient parity:
// position 16 v + 8 q + e holds c = q + 2 (8 v + e), so lane q holds T_q, T_{q+2}, ... and runs the
// stride-2 recurrence T_{c+2} = 2 T_2 T_c - T_{c-2} (with T_{q-2} = T_{2-q}).
__device__ __forceinline__ void ldg_v8(const float* p, float* o) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]), "=f"(o[7])
        : "l"(p));
}

template <int NH>
__device__ __forceinline__ float cheb_half(float x, const float* yy, int q) {
    const float x2 = x + x;
    const float t2 = fmaf(x2, x, -1.f);
    float a = q ? x : 1.f;   // T_q
    float b = q ? x : t2;    // T_{q-2} = T_{2-q}
    const float w2 = t2 + t2;
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int m = 0; m < NH; m++) {
        if (m & 1)
            s1 = fmaf(a, yy[m], s1);
        else
            s0 = fmaf(a, yy[m], s0);
        const float n = fmaf(w2, a, -b);
        b = a;
        a = n;
    }
    return s0 + s1;
}

// One warp per target row; lanes (g, q) = (lane / 2, lane % 2) take the row's table pairs 16 apart,
// four per lane per round: the round's blocks are gathered while the next round's records load,
// and the four values are added and the round's sum accumulated in the lane's FP64 sum.  Near pairs
// (r < dt, a few per row): eight lanes per stored row, one 16-byte vector each, summed per lane in
// FP32 and added to the FP64 sum once.  The 32 lanes' sums are added in FP64 at the end.  (An FP64
// accumulator measured slightly faster than the compensated FP32 one it replaced, with the same error.)
template <int NC>
__global__ void __launch_bounds__(256) k_local_cheb2(int64_t Mt, const int64_t* __restrict__ trow,
                                                     const TabPair<float>* __restrict__ tp, const float* __restrict__ y,
                                                     const int64_t* __restrict__ nrow, const int* __restrict__ ncol,
                                                     const float* __restrict__ neta, const float* __restrict__ siglin,
                                                     double* __restrict__ uloc) {
    static_assert(NC == 16 || NC == 32, "blocks of 16 or 32 coefficients");
    constexpr int NL = NC / 16;  // 32-byte loads per lane per pair
    constexpr int U = 4;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= Mt) return;
    const int q = lane & 1, g = lane >> 1;
    double dsum = 0.0;
    const int64_t p1 = trow[row + 1];
    // software pipeline: the records of the next U pairs are loaded while this group's blocks are
    // gathered and summed; past the row's end a record reads as block 0 with its value masked
    const TabPair<float> none{0u, 0.f};
    int64_t p = trow[row] + g;
    TabPair<float> en[U];
#pragma unroll
    for (int u = 0; u < U; u++) en[u] = (p + 16 * u < p1) ? load_pair(tp + p + 16 * u) : none;
    for (; p < p1; p += 16 * U) {
        TabPair<float> e[U];
        float yy[U][NC / 2];
#pragma unroll
        for (int u = 0; u < U; u++) {
            e[u] = en[u];
#pragma unroll
            for (int v = 0; v < NL; v++) ldg_v8(y + (size_t)e[u].blk * NC + 16 * v + 8 * q, yy[u] + 8 * v);
        }
        const int64_t pn = p + 16 * U;
#pragma unroll
        for (int u = 0; u < U; u++) en[u] = (pn + 16 * u < p1) ? load_pair(tp + pn + 16 * u) : none;
        float acc = 0.f;
#pragma unroll
        for (int u = 0; u < U; u++) {
            const float v = cheb_half<NC / 2>(e[u].x, yy[u], q);
            if (p + 16 * u < p1) acc += v;
        }
        dsum += (double)acc;
    }
    const int c8 = lane & 7, g8 = lane >> 3;
    const float4* E = (const float4*)neta;
    const float4* X = (const float4*)siglin;
    float near = 0.f;
    for (int64_t r = nrow[row] + g8; r < nrow[row + 1]; r += 4) {
        const float4 ev = __ldcs(E + r * 8 + c8), xv = __ldg(X + (int64_t)ncol[r] * 8 + c8);
        near += fmaf(ev.w, xv.w, fmaf(ev.z, xv.z, fmaf(ev.y, xv.y, ev.x * xv.x)));
    }
    const double tot = warp_sum(dsum + (double)near);
    if (lane == 0) uloc[row] = tot;
}

// FP32 contraction as a register-blocked product of two shared-memory tiles: the windows of 32
// sources (transposed, [level][source]) times the coefficients of KC = 64 / NC intervals
// ([level][interval, position]).  Thread (a, b) accumulates sources 4a..4a+3 x positions
// 4b..4b+3: per level two 16-byte shared loads feed 16 FMAs.  Tiles are filled by coalesced loads.
// One-dimensional grid, interval groups fastest: the blocks that read one group of source windows
// run back to back, so the windows come from L2 rather than once per interval group from HBM.
template <int NC>
__global__ void __launch_bounds__(128) k_ycoef4(int64_t M, int nk, const float* __restrict__ siglin,
                                                const float* __restrict__ ctab, float* __restrict__ y) {
    constexpr int KC = 64 / NC, QN = NC / 4;
    __shared__ __align__(16) float sT[32][36];  // [level][source], rows padded
    __shared__ __align__(16) float sc[32][64];  // [level][(interval - k0) * NC + position]
    const int nkg = (nk + KC - 1) / KC;
    const int64_t j0 = (int64_t)(blockIdx.x / nkg) * 32;
    const int k0 = (int)(blockIdx.x % nkg) * KC, nkc = min(nk - k0, KC);
    for (int t = threadIdx.x; t < 32 * 8; t += 128) {  // 32 windows of 8 vectors
        const int s = t >> 3, v = t & 7;
        const float4 z = (j0 + s < M) ? __ldg((const float4*)(siglin + (j0 + s) * 32) + v) : make_float4(0.f, 0.f, 0.f, 0.f);
        sT[4 * v][s] = z.x;
        sT[4 * v + 1][s] = z.y;
        sT[4 * v + 2][s] = z.z;
        sT[4 * v + 3][s] = z.w;
    }
    const float4* C4 = (const float4*)(ctab + (int64_t)k0 * 32 * NC);
    for (int t = threadIdx.x; t < KC * 32 * QN; t += 128) {  // [interval][level][position / 4]
        const int kl = t / (32 * QN), i = (t / QN) % 32, qq = t % QN;
        *(float4*)&sc[i][kl * NC + 4 * qq] = (kl < nkc) ? __ldg(C4 + t) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const int b = threadIdx.x & 15, a = threadIdx.x >> 4;
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int e = 0; e < 4; e++) acc[r][e] = 0.f;
#pragma unroll 8
    for (int i = 0; i < 32; i++) {
        const float4 sa = *(const float4*)&sT[i][4 * a];
        const float4 cb = *(const float4*)&sc[i][4 * b];
        const float sv[4] = {sa.x, sa.y, sa.z, sa.w}, cv[4] = {cb.x, cb.y, cb.z, cb.w};
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int e = 0; e < 4; e++) acc[r][e] = fmaf(sv[r], cv[e], acc[r][e]);
    }
    const int kk = k0 + (4 * b) / NC, qq = ((4 * b) % NC) / 4;
    if (kk >= nk) return;
    float4* Y4 = (float4*)y;
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int64_t j = j0 + 4 * a + r;
        if (j < M) Y4[((int64_t)kk * M + j) * QN + qq] = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    }
}

// FP32 contraction with the coefficients of every interval resident in shared memory (nk x 32 x
// NC floats, dynamic) and each thread's two source windows in registers: per interval and group of
// 16 positions, a level's 16 coefficients are four broadcast 16-byte shared loads feeding 32 FMAs,
// issued as 16 packed two-lane FMAs (fma.rn.f32x2: each lane an IEEE fused multiply-add), and each
// source's 16 results leave as two 32-byte stores (a warp writes 32 consecutive blocks of one
// interval).  Every output is the FP32 fused multiply-add chain over the levels in ascending order,
// as in k_ycoef4, so both give the same bits.
constexpr int kY5Threads = 128;
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ void stg_v4b64(float* p, const unsigned long long* o) {
    asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(o[0]), "l"(o[1]), "l"(o[2]), "l"(o[3])
                 : "memory");
}
template <int NC>
__global__ void __launch_bounds__(kY5Threads, 4) k_ycoef5(int64_t M, int nk, const float* __restrict__ siglin,
                                                            const float* __restrict__ ctab, float* __restrict__ y) {
    extern __shared__ __align__(16) float sc5[];  // [interval][level][position]
    const int nc4 = nk * 32 * NC / 4;
    for (int t = threadIdx.x; t < nc4; t += kY5Threads) ((float4*)sc5)[t] = __ldg((const float4*)ctab + t);
    __syncthreads();
    const int64_t j0 = (int64_t)blockIdx.x * (2 * kY5Threads) + threadIdx.x;
    const int64_t jj[2] = {j0, j0 + kY5Threads};
    float w[2][32];
#pragma unroll
    for (int s = 0; s < 2; s++) {
        const float4* src = (const float4*)(siglin + jj[s] * 32);
#pragma unroll
        for (int v = 0; v < 8; v++) {
            const float4 z = (jj[s] < M) ? __ldg(src + v) : make_float4(0.f, 0.f, 0.f, 0.f);
            w[s][4 * v] = z.x;
            w[s][4 * v + 1] = z.y;
            w[s][4 * v + 2] = z.z;
            w[s][4 * v + 3] = z.w;
        }
    }
    for (int k = 0; k < nk; k++) {
#pragma unroll 1
        for (int h = 0; h < NC; h += 16) {
            unsigned long long acc[2][8];
#pragma unroll
            for (int s = 0; s < 2; s++)
#pragma unroll
                for (int e = 0; e < 8; e++) acc[s][e] = 0ull;
            const float* ck = sc5 + (size_t)k * 32 * NC + h;
#pragma unroll
            for (int i = 0; i < 32; i++) {
                unsigned long long c[8];
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    const ulonglong2 q = *(const ulonglong2*)(ck + i * NC + 4 * v);
                    c[2 * v] = q.x;
                    c[2 * v + 1] = q.y;
                }
#pragma unroll
                for (int s = 0; s < 2; s++) {
                    const unsigned long long ww = pk2(w[s][i], w[s][i]);
#pragma unroll
                    for (int e = 0; e < 8; e++) acc[s][e] = ffma2(ww, c[e], acc[s][e]);
                }
            }
#pragma unroll
            for (int s = 0; s < 2; s++)
                if (jj[s] < M) {
                    float* out = y + ((int64_t)k * M + jj[s]) * NC + h;
                    stg_v4b64(out, acc[s]);
                    stg_v4b64(out + 8, acc[s] + 4);
                }
        }
    }
}

// position of coefficient c in an FP32 block of NC (16 or 32): the inverse of c = q + 2 (8 v + e)
// at position 16 v + 8 q + e
__host__ __device__ inline int cheb2_position(int c) {
    const int q = c & 1, m = c >> 1;
    return 16 * (m >> 3) + 8 * q + (m & 7);
}

}  // namespace wfp
