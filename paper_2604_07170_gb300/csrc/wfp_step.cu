// Per-step kernels of the 2D TK-WFP evaluator (sm_103a).
//
// One call of wfp_step at level n (t_n = n dt) runs two phases on the plan's stream:
//   output : ingest sigma(t_n); local part u_l(t_n) (Sec. 6); coincident-pair self term;
//            combine u = u_l + u_h - u_self, with u_h(t_n) left by the previous advance.
//   advance: type-1 NUFFTs of sigma(t_n) and sigma(t_{n-L}) (Sec. 4.3); Duhamel update of
//            every near-history mode to t_{n+1} (Lemma 4.2, Eq. hggrid); far-history
//            recurrences (Sec. 5, Eqs. alphaFApprox, beta0); type-2 NUFFT giving u_h(t_{n+1}).
// Kernels read the level from a device counter so that both phases can be replayed from
// CUDA graphs.  T is the reduced precision (double on the FP64 path, float on the mixed path);
// mode state alpha, its rotation, the recurrences and all sums across sources are FP64.
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>

#include "wfp_dev.h"
#include "wfp_plan.h"

namespace wfp {

// ------------------------------------------------------------------------------------ ingest
// sigma(t_n) in caller order -> the window [M][NW] (slot n & (NW-1)), the linear window [M][32]
// (shifted by one level, newest last; NW = 32 only) and the level-major history [n_hist][M] in
// the grid precision (slot n % n_hist) read by both spreads.
// LP = 32 sizeof(T) / 16 lanes per source (8 in FP32, 16 in FP64), each holding one 16-byte vector of
// the source's linear window: the shift by one level takes the next lane's first element by a shuffle.
template <typename T>
__global__ void __launch_bounds__(256) k_ingest(const int64_t* __restrict__ d_step, int64_t M,
                                                const double* __restrict__ sig_in, const int* __restrict__ perm,
                                                T* __restrict__ sigwin, int NW, T* __restrict__ siglin,
                                                T* __restrict__ sighist, int n_hist) {
    using V = typename Vec16<T>::type;
    constexpr int LP = 32 * sizeof(T) / 16;  // 16-byte vectors per 32-level row = lanes per source
    constexpr int E = 16 / sizeof(T);        // elements per vector
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t k = tid / LP;
    const int c = (int)(tid % LP);
    const bool valid = k < M;
    const int64_t n = *d_step + 1;
    double s = 0.0;
    if (valid) {
        s = sig_in[perm[k]];
        if (c == 0) {
            sigwin[k * NW + (n & (NW - 1))] = (T)s;
            sighist[(n % n_hist) * M + k] = (T)s;
        }
    }
    if (siglin) {  // uniform: the whole grid takes this branch or none of it
        V v = {};
        if (valid) v = ((const V*)(siglin + k * 32))[c];
        const T* t = (const T*)&v;
        const T next = __shfl_down_sync(0xffffffffu, t[0], 1, LP);  // the next vector's first element
        if (valid) {
            T out[E];
#pragma unroll
            for (int i = 0; i + 1 < E; i++) out[i] = t[i + 1];
            out[E - 1] = (c == LP - 1) ? (T)s : next;
            ((V*)(siglin + k * 32))[c] = *(const V*)out;
        }
    }
}

// -------------------------------------------------------------------------------- self term
// u_self,i(t_n) = (1/2pi) int_0^t phi(d) sigma_i(t_n - d)/d dd, with 1/d ~ sum_l w_l exp(-mu_l d) on
// [d_lo, T] and the trapezoid rule on the grid, arranged as a shared window plus one-tap recurrences:
//   u_self(t_n) = sum_{q<W-1} g_q sigma_{n-1-q} + sum_l w'_l Z_l(t_n),
//   Z_l(t_{n+1}) = r_l Z_l(t_n) + r_l^W sigma_{n+1-W}.
// The state is kept as Zh_l = Z_l / r_l^W, so that a term costs two FP64 fused multiply-adds:
//   Zh_l(t_{n+1}) = r_l Zh_l(t_n) + sigma_{n+1-W},   u_self += (w'_l r_l^W) Zh_l(t_n).
constexpr int kMaxWFar = 64;  // W <= 59

constexpr int kSelfGroups = 8;

template <typename T>
__global__ void __launch_bounds__(32 * kSelfGroups) k_self(const int64_t* __restrict__ d_step, int64_t n_self,
                                                           const int* __restrict__ self_tgt,
                                                           const int* __restrict__ self_src,
                                                           const T* __restrict__ sigwin, int NW, int W, int nsoe,
                                                           const double* __restrict__ shead,
                                                           const double* __restrict__ sdecay,
                                                           const double* __restrict__ sw, double* __restrict__ Y,
                                                           double* __restrict__ uself) {
    // block (32, G): 32 coincident targets x G interleaved groups of SOE terms
    constexpr int G = kSelfGroups;
    __shared__ double s_red[G][32];
    int64_t s = (int64_t)blockIdx.x * 32 + threadIdx.x;
    int g = threadIdx.y;
    double u = 0.0;
    if (s < n_self) {
        const int64_t n = *d_step + 1;
        const T* win = sigwin + (int64_t)self_src[s] * NW;
        for (int q = g; q < W - 1; q += G) u = fma(shead[q], (double)win[(n - 1 - q) & (NW - 1)], u);
        const double x = (double)win[(n + 1 - W) & (NW - 1)];
        // terms l = g, g + G, ... in batches of 8 with every load of a batch issued first
        for (int l0 = g; l0 < nsoe; l0 += 8 * G) {
            double z[8];
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int l = l0 + k * G;
                if (l < nsoe) z[k] = Y[(int64_t)l * n_self + s];
            }
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int l = l0 + k * G;
                if (l < nsoe) {
                    u = fma(sw[l], z[k], u);
                    Y[(int64_t)l * n_self + s] = fma(sdecay[l], z[k], x);
                }
            }
        }
    }
    s_red[g][threadIdx.x] = u;
    __syncthreads();
    if (g == 0 && s < n_self) {
        for (int k = 1; k < G; k++) u += s_red[k][threadIdx.x];
        uself[self_tgt[s]] = u;
    }
}

// u(t_n) = u_l + u_h - u_self; u_h(t_n) was written by the advance of step n - 1 into slot n & 1
__global__ void k_combine(const int64_t* __restrict__ d_step, int64_t Mt, const int* __restrict__ tgt_perm,
                          const double* __restrict__ uloc, const double* __restrict__ uh,
                          const double* __restrict__ uself, double* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Mt) return;
    const int64_t n = *d_step + 1;
    out[tgt_perm[i]] = uloc[i] + uh[(n & 1) * Mt + i] - uself[i];
}

__global__ void k_tick(int64_t* d_step) { *d_step += 1; }

// ------------------------------------------------------------------------------- spreading
// Type-1 spreading onto the fine-grid band, one CTA per non-empty TS x TS tile.  The tile's source
// list (every source whose w x w footprint meets the tile, ascending internal index) is shared out by
// the residue of the source index modulo kSpreadWarps: warp c takes the sources j = c (mod
// kSpreadWarps), in list order, and adds each one's footprint, clipped to the tile, into its own
// partial tile in shared memory (lanes over footprint columns and rows, kernel values staged in
// shared memory SM sources at a time).  The tile is then the sum of the partials in warp order.  So
// every grid point gets
//     sum_{c < kSpreadWarps} ( sum over the sources j = c (mod kSpreadWarps) that cover it, ascending j )
// whatever TS or CH: no atomics, results independent of the tiling, and the current and lagged
// transforms of a level bit-identical.  CH is the number of list entries a warp scans per round.
constexpr int kSpreadWarps = 4;  // residue classes of the source index (fixed: the sums depend on it)
constexpr int kSpreadStage = 8;  // sources whose kernel values a warp stages at once
constexpr int kSpreadKer = 48;   // 2 w values per staged source (w <= 24)

template <typename T, int TS, int CH>
__global__ void __launch_bounds__(32 * kSpreadWarps) k_spread(const int64_t* __restrict__ d_step, int lag, int L,
                                                             int64_t M, const T* __restrict__ sighist, int n_hist,
                                                             const int* __restrict__ tile_xy,
                                                             const int* __restrict__ tile_ptr,
                                                             const int* __restrict__ tile_src,
                                                             const int* __restrict__ src_off,
                                                             const T* __restrict__ src_ker, int w, T* __restrict__ sp,
                                                             int nf, int lb0) {
    constexpr int P = TS + 1;  // padded row of a partial tile
    constexpr int SM = kSpreadStage;
    const int64_t n = *d_step + 1;
    const int64_t lev = lag ? n - L : n;
    if (lev < 1) return;
    const T* sig = sighist + (lev % n_hist) * M;
    __shared__ T part[kSpreadWarps][TS * P];
    __shared__ T stage[kSpreadWarps][SM][kSpreadKer];
    __shared__ T s_val[kSpreadWarps][SM];
    __shared__ int s_src[kSpreadWarps][SM], s_off[kSpreadWarps][SM];
    for (int i = threadIdx.x; i < kSpreadWarps * TS * P; i += blockDim.x) (&part[0][0])[i] = (T)0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;  // lanes below this one
    const int txy = tile_xy[blockIdx.x];
    const int tx0 = (txy & 0xffff) * TS, ty0 = (txy >> 16) * TS;
    const int a0 = tile_ptr[blockIdx.x], a1 = tile_ptr[blockIdx.x + 1];
    const int w2 = 2 * w;
    // lanes over a footprint: CL columns (a power of two >= w, at most 32) x 32 / CL rows per pass
    const int lcl = w <= 8 ? 3 : (w <= 16 ? 4 : 5);
    const int cx = lane & ((1 << lcl) - 1), ry = lane >> lcl, rpp = 32 >> lcl;
    T* my = part[warp];
    for (int c0 = a0; c0 < a1; c0 += CH) {
#pragma unroll
        for (int h = 0; h < CH; h += 32) {
            const int i = c0 + h + lane;
            const int sidx = (i < a1) ? tile_src[i] : -1;
            const bool member = sidx >= 0 && (sidx & (kSpreadWarps - 1)) == warp;
            unsigned mine = __ballot_sync(0xffffffffu, member);
            while (mine) {  // uniform across the warp
                // stage the next (up to SM) of this warp's sources, in list order: a member lane whose
                // rank among the remaining members is below SM writes its source to slot rank
                const int rank = __popc(mine & lt);
                const bool take = ((mine >> lane) & 1u) && rank < SM;
                const int k = min(__popc(mine), SM);
                if (take) {
                    s_src[warp][rank] = sidx;
                    s_off[warp][rank] = src_off[sidx];
                    s_val[warp][rank] = sig[sidx];
                }
                __syncwarp();
                T kvv[SM], kvw[SM];
#pragma unroll
                for (int j = 0; j < SM; j++) {
                    kvv[j] = (j < k && lane < w2) ? src_ker[(int64_t)s_src[warp][j] * w2 + lane] : (T)0;
                    kvw[j] = (j < k && lane + 32 < w2) ? src_ker[(int64_t)s_src[warp][j] * w2 + lane + 32] : (T)0;
                }
#pragma unroll
                for (int j = 0; j < SM; j++) {
                    stage[warp][j][lane] = kvv[j];
                    if (lane + 32 < kSpreadKer) stage[warp][j][lane + 32] = kvw[j];
                }
                __syncwarp();
                for (int j = 0; j < k; j++) {
                    const int off = s_off[warp][j];
                    const int ox = (off & 0xffff) - tx0, oy = (off >> 16) - ty0;  // footprint origin in the tile
                    const int xx = ox + cx;
                    if (cx < w && xx >= 0 && xx < TS) {
                        const T* kv = stage[warp][j];
                        const T kxs = s_val[warp][j] * kv[cx];  // x-kernel value times the strength
                        for (int dy = ry; dy < w; dy += rpp) {  // footprint rows dy = ry (mod rpp)
                            const int yy = oy + dy;
                            if ((unsigned)yy < (unsigned)TS) {
                                T* cell = my + yy * P + xx;
                                *cell = fma(kxs, kv[w + dy], *cell);
                            }
                        }
                    }
                    __syncwarp();
                }
                mine &= ~__ballot_sync(0xffffffffu, take);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < TS * TS; i += blockDim.x) {
        const int r = i / TS, c = i - r * TS;
        T v = part[0][r * P + c];
#pragma unroll
        for (int q = 1; q < kSpreadWarps; q++) v += part[q][r * P + c];
        sp[(int64_t)(ty0 + r) * nf + lb0 + tx0 + c] = v;
    }
}

template <typename T, int TS, int CH>
static void spread_one(const Plan& pl, int lag, int n_tiles, const int* txy, const int* tptr, const int* tsrc, T* sp,
                       cudaStream_t st) {
    const Params& P = pl.P;
    k_spread<T, TS, CH><<<n_tiles, 32 * kSpreadWarps, 0, st>>>(pl.d_step, lag, P.L, pl.M, (const T*)pl.d_sighist, pl.n_hist,
                                                       txy, tptr, tsrc, pl.d_src_off, (const T*)pl.d_src_ker, P.w, sp,
                                                       P.nf, P.lb0);
}

template <typename T>
static void spread_t(const Plan& pl, int ts, int ch, int lag, int n_tiles, const int* txy, const int* tptr,
                     const int* tsrc, T* sp, cudaStream_t st) {
    if (ts == 8)
        (ch == 32 ? spread_one<T, 8, 32> : spread_one<T, 8, 64>)(pl, lag, n_tiles, txy, tptr, tsrc, sp, st);
    else if (ts == 16)
        (ch == 32 ? spread_one<T, 16, 32> : spread_one<T, 16, 64>)(pl, lag, n_tiles, txy, tptr, tsrc, sp, st);
    else
        (ch == 32 ? spread_one<T, 32, 32> : spread_one<T, 32, 64>)(pl, lag, n_tiles, txy, tptr, tsrc, sp, st);
}

void spread_launch(const Plan& pl, int ts, int ch, int lag, int n_tiles, const int* txy, const int* tptr,
                   const int* tsrc, void* sp, cudaStream_t st) {
    if (n_tiles <= 0) return;
    if (pl.P.precision == WFP_FP64)
        spread_t<double>(pl, ts, ch, lag, n_tiles, txy, tptr, tsrc, (double*)sp, st);
    else
        spread_t<float>(pl, ts, ch, lag, n_tiles, txy, tptr, tsrc, (float*)sp, st);
}

// ------------------------------------------------------------------------------ mode update
// For each half-plane mode k = (n1, n2) dk:
//   S_n = conj(T1[k]) fac(n1) fac(n2)   (type-1 result, deconvolved, shifted by pi)
//   h = sum_{m<W} p_m S_{n-m} - pA_m S_{n-m-L},  g likewise with q, qA    (Eq. hggrid)
//   alpha(t+dt)  =  cos(k dt) alpha + sin(k dt)/k alphadot + h            (Eq. alphakEvolution)
//   alphad(t+dt) = -k sin(k dt) alpha + cos(k dt) alphadot + g
// and writes the type-2 coefficient (dk/2pi)^2 alpha fac(n1) fac(n2) (conjugated) for the C2C pass.
template <typename T>
__global__ void __launch_bounds__(256) k_modes(
    const int64_t* __restrict__ d_step, int64_t n_modes, int W, int L, int Nh, int nf, const int2* __restrict__ mode_n,
    const int* __restrict__ mode_k, const double* __restrict__ fac, double coef2,
    const typename Cplx<T>::type* __restrict__ tc_cur, const typename Cplx<T>::type* __restrict__ tc_lag,
    typename Cplx<T>::type* __restrict__ ring, typename Cplx<T>::type* __restrict__ ring_lag, int R_cur, int R_lag,
    int lag_off, int write_lag,
    const T* __restrict__ taps, const double* __restrict__ rot, double2* __restrict__ alpha,
    double2* __restrict__ alphad, typename Cplx<T>::type* __restrict__ td, int64_t near_sq,
    const double2* __restrict__ aF, int64_t n_far_now) {
    using C = typename Cplx<T>::type;
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_modes) return;
    int64_t n = *d_step + 1;
    bool lag = (n - L >= 1);
    int2 nn = mode_n[m];
    int kid = mode_k[m];
    int row = nn.x < 0 ? nn.x + nf : nn.x;
    int64_t gi = (int64_t)nn.y * nf + row;  // column-major pruned spectrum [Nh+1][nf]
    double f = fac[nn.x < 0 ? -nn.x : nn.x] * fac[nn.y];
    const int slot = (int)(n % R_cur);
    {
        C t = tc_cur[gi];
        C s;
        s.x = (T)((double)t.x * f);
        s.y = (T)(-(double)t.y * f);
        ring[(int64_t)slot * n_modes + m] = s;
    }
    if (lag && write_lag) {  // lagged NUFFT result: level n - L goes to slot (n - L + lag_off) mod R_lag
        C t = tc_lag[gi];
        C s;
        s.x = (T)((double)t.x * f);
        s.y = (T)(-(double)t.y * f);
        ring_lag[(int64_t)((n - L + lag_off) % R_lag) * n_modes + m] = s;
    }
    // the near history is truncated at |k| <= K (Eq. uhtraptrunc); modes between K and the far
    // cut-off carry only S (for the far forcing) and the far coefficient alpha_F
    const double2 af = (m < n_far_now) ? aF[m] : make_double2(0.0, 0.0);
    if ((int64_t)nn.x * nn.x + (int64_t)nn.y * nn.y > near_sq) {
        const double cf = coef2 * f;
        C o;
        o.x = (T)(af.x * cf);
        o.y = (T)(-af.y * cf);
        td[gi] = o;
        if (nn.y == 0 && nn.x > 0) {
            o.y = (T)(af.y * cf);
            td[nf - nn.x] = o;  // column 0, row nf - n1
        }
        return;
    }
    // levels n - j (ring slot sl) and n - L - j (ring_lag slot sll), j = 0..W-1, taken U at a time
    // with all loads issued before the arithmetic (the order of the sums is j ascending)
    int sl = slot;
    int sll = (int)((((n - L + lag_off) % R_lag) + R_lag) % R_lag);
    double hxd, hyd, gxd, gyd;
    constexpr int U = sizeof(T) == 8 ? 2 : 4;  // the FP64 form is bound by FP64 issue, not latency
    if constexpr (sizeof(T) == 8) {
        const double2* tp = (const double2*)(taps + (int64_t)kid * 4 * W);  // {p, q}, {pA, qA} per level
        double hx = 0, hy = 0, gx = 0, gy = 0;
        for (int j0 = 0; j0 < W; j0 += U) {
            double2 a[U], b[U], pq[U], pqA[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int j = j0 + u;
                if (j < W) {
                    const int s1 = sl - u < 0 ? sl - u + R_cur : sl - u;
                    a[u] = ring[(int64_t)s1 * n_modes + m];
                    pq[u] = tp[2 * j];
                    if (lag) {
                        const int s2 = sll - u < 0 ? sll - u + R_lag : sll - u;
                        b[u] = ring_lag[(int64_t)s2 * n_modes + m];
                        pqA[u] = tp[2 * j + 1];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (j0 + u < W) {
                    hx = fma(pq[u].x, a[u].x, hx);
                    hy = fma(pq[u].x, a[u].y, hy);
                    gx = fma(pq[u].y, a[u].x, gx);
                    gy = fma(pq[u].y, a[u].y, gy);
                    if (lag) {
                        hx = fma(-pqA[u].x, b[u].x, hx);
                        hy = fma(-pqA[u].x, b[u].y, hy);
                        gx = fma(-pqA[u].y, b[u].x, gx);
                        gy = fma(-pqA[u].y, b[u].y, gy);
                    }
                }
            }
            sl = sl - U < 0 ? sl - U + R_cur : sl - U;
            sll = sll - U < 0 ? sll - U + R_lag : sll - U;
        }
        hxd = hx, hyd = hy, gxd = gx, gyd = gy;
    } else {
        static_assert(sizeof(T) == 8, "the FP32 mode update is k_modes_one");
    }
    double c = rot[3 * kid], sk = rot[3 * kid + 1], ks = rot[3 * kid + 2];
    double2 a = alpha[m], ad = alphad[m];
    double2 an, adn;
    an.x = fma(c, a.x, fma(sk, ad.x, hxd));
    an.y = fma(c, a.y, fma(sk, ad.y, hyd));
    adn.x = fma(-ks, a.x, fma(c, ad.x, gxd));
    adn.y = fma(-ks, a.y, fma(c, ad.y, gyd));
    alpha[m] = an;
    alphad[m] = adn;
    double cf = coef2 * f;
    C o;  // type-2 coefficient of the near plus far history
    o.x = (T)((an.x + af.x) * cf);
    o.y = (T)(-(an.y + af.y) * cf);
    td[gi] = o;
    if (nn.y == 0 && nn.x > 0) {
        o.y = (T)((an.y + af.y) * cf);
        td[nf - nn.x] = o;  // column 0, row nf - n1
    }
}

// Mixed-path mode update, one thread per mode.  Both FIRs of Eq. hggrid -- h with the taps {p, pA},
// g with {q, qA}, hi/lo pairs -- are formed from one set of ring loads with error-free products
// summed in double-float, so that the FIR adding a level and the one removing it L steps later
// round alike and nothing persists in alpha.  The newest current and lagged levels come from
// registers; a level's taps for both FIRs are one 32-byte load.  Then alpha and alpha-dot advance
// (Eq. alphakEvolution, FP64) and the type-2 coefficient is written.  (Two threads per mode, one
// per FIR, gave the same bits with every ring value loaded twice: 6% slower at 10^4 points and 33%
// at 10^6.)
// A plan whose run ends before the lag switches on (COMPACT: N_t dt < A+ - delta) never removes a
// level, so there is nothing to round alike: its FIRs are plain FP32 fused multiply-add sums with the
// taps' high parts, four levels in flight.  Their rounding (a relative ~1e-7 perturbation of h each
// step, the size of the FP32 rounding of the S levels themselves) enters alpha once and is carried
// with it, and the kernel reads its ring at the memory rate instead of being bound by the
// double-float arithmetic.
__device__ __forceinline__ void ldg_v8f(const float* p, float4& a, float4& b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

template <bool COMPACT>
__global__ void __launch_bounds__(256) k_modes_one(
    const int64_t* __restrict__ d_step, int64_t n_modes, int W, int L, int Nh, int nf, const int2* __restrict__ mode_n,
    const int* __restrict__ mode_k, const float* __restrict__ facf, float coef2, const float2* __restrict__ tc_cur,
    const float2* __restrict__ tc_lag, float2* __restrict__ ring, float2* __restrict__ ring_lag, int R_cur, int R_lag,
    int lag_off, int write_lag, const float* __restrict__ taps, const double* __restrict__ rot,
    double2* __restrict__ alpha, double2* __restrict__ alphad, float2* __restrict__ td, int64_t near_sq,
    const double2* __restrict__ aF, int64_t n_far_now) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_modes) return;
    const int64_t n = *d_step + 1;
    const bool lag = (n - L >= 1);
    const int slot = (int)(n % R_cur);
    const int slot_lag = (int)((((n - L + lag_off) % R_lag) + R_lag) % R_lag);  // level n - L
    const int2 nn = mode_n[m];
    const int kid = mode_k[m];
    const int row = nn.x < 0 ? nn.x + nf : nn.x;
    const int64_t gi = (int64_t)nn.y * nf + row;  // column-major pruned spectrum [Nh+1][nf]
    const float f = facf[nn.x < 0 ? -nn.x : nn.x] * facf[nn.y];  // deconvolution, FP32 like the transform
    float2 s_cur, s_lag = make_float2(0.f, 0.f);
    {
        const float2 t = tc_cur[gi];
        s_cur.x = t.x * f;
        s_cur.y = -t.y * f;
    }
    ring[(int64_t)slot * n_modes + m] = s_cur;
    if (lag) {
        if (write_lag) {  // lagged NUFFT result: level n - L
            const float2 u = tc_lag[gi];
            s_lag.x = u.x * f;
            s_lag.y = -u.y * f;
            ring_lag[(int64_t)slot_lag * n_modes + m] = s_lag;
        } else {
            s_lag = ring_lag[(int64_t)slot_lag * n_modes + m];
        }
    }
    const float cf = coef2 * f;
    if ((int64_t)nn.x * nn.x + (int64_t)nn.y * nn.y > near_sq) {  // only the far coefficient, if any
        const double2 af = (m < n_far_now) ? aF[m] : make_double2(0.0, 0.0);
        float2 o;
        o.x = (float)af.x * cf;
        o.y = -(float)af.y * cf;
        td[gi] = o;
        if (nn.y == 0 && nn.x > 0) {
            o.y = (float)af.y * cf;
            td[nf - nn.x] = o;  // column 0, row nf - n1
        }
        return;
    }
    // h: (hxh, hxl, hyh, hyl); g: (gxh, gxl, gyh, gyl)
    float hxh = 0.f, hxl = 0.f, hyh = 0.f, hyl = 0.f, gxh = 0.f, gxl = 0.f, gyh = 0.f, gyl = 0.f;
    const float* tk = taps + (int64_t)kid * (COMPACT ? 4 : 8) * W;
    if constexpr (COMPACT) {
        constexpr int U4 = 4;  // levels whose loads are in flight together
        int sc = slot;
        for (int j0 = 0; j0 < W; j0 += U4) {
            float2 a[U4];
            float4 t[U4];
#pragma unroll
            for (int u = 0; u < U4; u++) {
                const int j = j0 + u;
                if (j < W) {
                    t[u] = *(const float4*)(tk + 4 * j);  // {p hi, p lo, q hi, q lo}
                    if (j == 0) {
                        a[u] = s_cur;
                    } else {
                        const int s1 = sc - u < 0 ? sc - u + R_cur : sc - u;
                        a[u] = ring[(int64_t)s1 * n_modes + m];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U4; u++) {
                if (j0 + u < W) {
                    hxh = fmaf(t[u].x, a[u].x, hxh);
                    hyh = fmaf(t[u].x, a[u].y, hyh);
                    gxh = fmaf(t[u].z, a[u].x, gxh);
                    gyh = fmaf(t[u].z, a[u].y, gyh);
                }
            }
            sc = sc - U4 < 0 ? sc - U4 + R_cur : sc - U4;
        }
    } else {
        constexpr int U = 2;  // levels whose loads are in flight together
        int sl = slot, sll = slot_lag;
        for (int j0 = 0; j0 < W; j0 += U) {
            float2 a[U], b[U];
            float4 th[U], tg[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int j = j0 + u;
                if (j < W) {
                    ldg_v8f(tk + 8 * j, th[u], tg[u]);
                    if (j == 0) {
                        a[u] = s_cur;
                        b[u] = s_lag;
                    } else {
                        const int s1 = sl - u < 0 ? sl - u + R_cur : sl - u;
                        a[u] = ring[(int64_t)s1 * n_modes + m];
                        if (lag) {
                            const int s2 = sll - u < 0 ? sll - u + R_lag : sll - u;
                            b[u] = ring_lag[(int64_t)s2 * n_modes + m];
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (j0 + u < W) {
                    df_acc(hxh, hxl, th[u].x, th[u].z, a[u].x);
                    df_acc(hyh, hyl, th[u].x, th[u].z, a[u].y);
                    if (lag) {
                        df_acc(hxh, hxl, -th[u].y, -th[u].w, b[u].x);
                        df_acc(hyh, hyl, -th[u].y, -th[u].w, b[u].y);
                    }
                    df_acc(gxh, gxl, tg[u].x, tg[u].z, a[u].x);
                    df_acc(gyh, gyl, tg[u].x, tg[u].z, a[u].y);
                    if (lag) {
                        df_acc(gxh, gxl, -tg[u].y, -tg[u].w, b[u].x);
                        df_acc(gyh, gyl, -tg[u].y, -tg[u].w, b[u].y);
                    }
                }
            }
            sl = sl - U < 0 ? sl - U + R_cur : sl - U;
            sll = sll - U < 0 ? sll - U + R_lag : sll - U;
        }
    }
    double hx, hy, gx, gy;
    if constexpr (COMPACT) {  // plain FP32 sums: no low parts to add
        hx = (double)hxh;
        hy = (double)hyh;
        gx = (double)gxh;
        gy = (double)gyh;
    } else {
        hx = (double)hxh + (double)hxl;
        hy = (double)hyh + (double)hyl;
        gx = (double)gxh + (double)gxl;
        gy = (double)gyh + (double)gyl;
    }
    const double c = rot[3 * kid], sk = rot[3 * kid + 1], ks = rot[3 * kid + 2];
    const double2 a = alpha[m], ad = alphad[m];
    double2 an, adn;
    an.x = fma(c, a.x, fma(sk, ad.x, hx));
    an.y = fma(c, a.y, fma(sk, ad.y, hy));
    adn.x = fma(-ks, a.x, fma(c, ad.x, gx));
    adn.y = fma(-ks, a.y, fma(c, ad.y, gy));
    alpha[m] = an;
    alphad[m] = adn;
    if (m < n_far_now) {  // near plus far history
        const double2 af = aF[m];
        an.x += af.x;
        an.y += af.y;
    }
    float2 o;
    o.x = (float)an.x * cf;
    o.y = -(float)an.y * cf;
    td[gi] = o;
    if (nn.y == 0 && nn.x > 0) {
        o.y = (float)an.y * cf;
        td[nf - nn.x] = o;  // column 0, row nf - n1
    }
}

// ------------------------------------------------------------------------------ spectrum layout
// The pruned spectrum is kept column-major, [Nh+1][nf] (column = the half-spectrum frequency of the
// row transform, row = the full frequency of the column transform), so that the column transforms
// run over contiguous vectors.  These move the band rows lb0..lb0+nb of the row transforms'
// [nf][nf/2+1] layout into the kept columns of that layout and back, 32 x 32 tiles through shared
// memory (block (32, 8), grid (ceil((Nh+1)/32), ceil(nb/32))).  Rows outside the band are never
// written: the column transforms' input keeps its zeros there.
template <typename C>
__global__ void __launch_bounds__(256) k_band_to_cols(const C* __restrict__ src, C* __restrict__ dst, int nb, int nc1,
                                                      int nh2, int nf, int lb0) {
    __shared__ C tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
    for (int k = ty; k < 32; k += 8)
        if (r0 + k < nb && c0 + tx < nc1) tile[k][tx] = src[(int64_t)(lb0 + r0 + k) * nh2 + c0 + tx];
    __syncthreads();
    for (int k = ty; k < 32; k += 8)
        if (r0 + tx < nb && c0 + k < nc1) dst[(int64_t)(c0 + k) * nf + lb0 + r0 + tx] = tile[tx][k];
}

template <typename C>
__global__ void __launch_bounds__(256) k_cols_to_band(const C* __restrict__ src, C* __restrict__ dst, int nb, int nc1,
                                                      int nh2, int nf, int lb0) {
    __shared__ C tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
    for (int k = ty; k < 32; k += 8)
        if (r0 + tx < nb && c0 + k < nc1) tile[k][tx] = src[(int64_t)(c0 + k) * nf + lb0 + r0 + tx];
    __syncthreads();
    for (int k = ty; k < 32; k += 8)
        if (r0 + k < nb && c0 + tx < nc1) dst[(int64_t)(lb0 + r0 + k) * nh2 + c0 + tx] = tile[tx][k];
}

// ------------------------------------------------------------------------------ far history
// For each far mode (|k| <= Kf), Sec. 5 with the blended far kernel integrated against the
// trapezoid interpolant of the lagged S on the grid (exp(A lam) scaling carried in the state):
//   E_l(t_{n+1}) = r_l E_l(t_n) + f_l S_{n-L-W+1}                  (tail recurrence, one tap)
//   alpha_F = sum_l H_l(|k|) E_l + sum_{q<W-1} Phi_q(|k|) S_{n-L-q}   (Eq. alphaFApprox + newest levels)
// with the state kept as Eh_l = E_l / f_l and H_l f_l stored in H: Eh_l <- r_l Eh_l + S_{n-L-W+1},
// alpha_F = sum_l (H_l f_l) Eh_l + ..., two FP64 fused multiply-adds per term and component.
// alpha_F goes to aF_out; the mode update adds it to the type-2 coefficient.  With the S history
// stored every level read here is at least L steps old, so the kernel can run while this step's
// type-1 transform is computed; with the lag recomputed the newest lagged level n - L is taken from
// this step's lagged transform and deconvolved exactly as the mode update does.  Block (32, G): 32
// far modes x G groups of terms; the W newest lagged levels of the block's modes are staged in
// shared memory.  Far modes are the first n_far modes (modes are ordered by |k|); H and Phi are
// stored [term][|k|], so the 32 modes of a warp read neighbours.
constexpr int kFarGroups = 8;
constexpr int kFarBatch = 8;  // terms of a thread whose loads are issued together

template <typename T>
__global__ void __launch_bounds__(32 * kFarGroups) k_far(
    const int64_t* __restrict__ d_step, int64_t n_far, int64_t n_modes, int W, int L, int Nh, int nf, int nlam,
    int64_t n_fk, const int* __restrict__ far_k, const int2* __restrict__ mode_n, const double* __restrict__ fac,
    const float* __restrict__ facf, const typename Cplx<T>::type* __restrict__ tc_lag, int from_tc,
    const typename Cplx<T>::type* __restrict__ ring_lag, int R_lag, int lag_off, const double* __restrict__ H,
    const double* __restrict__ ffir, const double* __restrict__ fdecay, double2* __restrict__ B,
    double2* __restrict__ aF_out) {
    using C = typename Cplx<T>::type;
    constexpr int G = kFarGroups;
    int64_t n = *d_step + 1;
    if (n - L < 1) return;
    __shared__ double2 s_red[G][32];
    __shared__ C s_S[kMaxWFar][32];
    const int64_t f = (int64_t)blockIdx.x * 32 + threadIdx.x;  // far mode f is mode f
    const int g = threadIdx.y;
    const bool valid = f < n_far;
    for (int j = g; j < W; j += G) {
        C v;
        v.x = 0;
        v.y = 0;
        if (valid) {
            if (j == 0 && from_tc) {  // level n - L from this step's lagged transform
                const int2 nn = mode_n[f];
                const int row = nn.x < 0 ? nn.x + nf : nn.x;
                const C t = tc_lag[(int64_t)nn.y * nf + row];
                if constexpr (sizeof(T) == 8) {
                    const double fd = fac[nn.x < 0 ? -nn.x : nn.x] * fac[nn.y];
                    v.x = (T)((double)t.x * fd);
                    v.y = (T)(-(double)t.y * fd);
                } else {
                    const float ff = facf[nn.x < 0 ? -nn.x : nn.x] * facf[nn.y];
                    v.x = t.x * ff;
                    v.y = -t.y * ff;
                }
            } else {
                const int sl = (int)((((n - L - j + lag_off) % R_lag) + R_lag) % R_lag);  // level n - L - j
                v = ring_lag[(int64_t)sl * n_modes + f];
            }
        }
        s_S[j][threadIdx.x] = v;
    }
    __syncthreads();
    double2 aF = make_double2(0.0, 0.0);
    if (valid) {
        const int64_t fk = far_k[f];
        for (int q = g; q < W - 1; q += G) {
            const C sq = s_S[q][threadIdx.x];
            const double fq = ffir[(int64_t)q * n_fk + fk];
            aF.x = fma(fq, (double)sq.x, aF.x);
            aF.y = fma(fq, (double)sq.y, aF.y);
        }
        const C st = s_S[W - 1][threadIdx.x];
        const double sx = st.x, sy = st.y;
        // terms l = g, g + G, ... in batches with every load of a batch issued first
        constexpr int NB = kFarBatch;
        for (int l0 = g; l0 < nlam; l0 += NB * G) {
            double2 b[NB];
            double hl[NB];
#pragma unroll
            for (int u = 0; u < NB; u++) {
                const int l = l0 + u * G;
                if (l < nlam) {
                    b[u] = B[(int64_t)l * n_far + f];
                    hl[u] = H[(int64_t)l * n_fk + fk];
                }
            }
#pragma unroll
            for (int u = 0; u < NB; u++) {
                const int l = l0 + u * G;
                if (l < nlam) {
                    const double d = fdecay[l];
                    b[u].x = fma(d, b[u].x, sx);
                    b[u].y = fma(d, b[u].y, sy);
                    B[(int64_t)l * n_far + f] = b[u];
                    aF.x = fma(hl[u], b[u].x, aF.x);
                    aF.y = fma(hl[u], b[u].y, aF.y);
                }
            }
        }
    }
    s_red[g][threadIdx.x] = aF;
    __syncthreads();
    if (g == 0 && valid) {
        for (int k = 1; k < G; k++) {
            aF.x += s_red[k][threadIdx.x].x;
            aF.y += s_red[k][threadIdx.x].y;
        }
        aF_out[f] = aF;
    }
}

// --------------------------------------------------------------------------- interpolation
// Type-2 interpolation: u_h(x_i) = sum over the w x w footprint of grid * psi_x psi_y.
// G = 32 / H targets per warp, H = 16 lanes per target when w <= 16 (else 32), lane = column offset:
// a lane sums its column over the footprint's rows, weights it by its column's kernel value, and the
// H lanes are added by shuffles -- in the grid precision T (FP32 on the mixed path, whose
// interpolation is FP32; FP64 on the FP64 path), converted to FP64 for the output.
// u_h(t_{n+1}) goes to slot (n + 1) & 1 of uh, so that step n's output can still read slot n & 1.
template <typename T, int H>
__global__ void __launch_bounds__(256) k_interp(const int64_t* __restrict__ d_step, int64_t Mt,
                                                const int* __restrict__ tgt_off, const T* __restrict__ tgt_ker, int w,
                                                const T* __restrict__ tf, int nf, int lb0, double* __restrict__ uh) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / H;
    const int lane = threadIdx.x & (H - 1);
    if (((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / H >= Mt) return;  // whole warp past the end
    const bool valid = i < Mt;
    uh += ((*d_step + 2) & 1) * Mt;
    T v = 0;
    if (valid && lane < w) {
        const int off = tgt_off[i];
        const int ix0 = off & 0xffff, iy0 = off >> 16;
        const T* ker = tgt_ker + i * 2 * w;
        const T* base = tf + (int64_t)iy0 * nf + lb0 + ix0 + lane;
        for (int dy = 0; dy < w; dy++) v += base[(int64_t)dy * nf] * ker[w + dy];
        v *= ker[lane];
    }
#pragma unroll
    for (int o = H / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (valid && lane == 0) uh[i] = (double)v;
}

// ================================================================================ drivers
static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

#define CK(x)                                                                                   \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess) {                                                                \
            err = std::string(#x) + ": " + cudaGetErrorString(e_);                              \
            return WFP_ECUDA;                                                                   \
        }                                                                                       \
    } while (0)
#define CKF(x)                                                                                  \
    do {                                                                                        \
        cufftResult r_ = (x);                                                                   \
        if (r_ != CUFFT_SUCCESS) {                                                              \
            err = std::string(#x) + ": cufft error " + std::to_string((int)r_);                 \
            return WFP_ECUDA;                                                                   \
        }                                                                                       \
    } while (0)

const char* const kPartNames[PP_NPARTS] = {"ingest", "local", "self", "combine", "spread", "fft_type1",
                                           "modes",  "far",   "fft_type2", "interp", "copy"};

void prof_collect(Plan& pl) {
    if (pl.prof_ev.empty()) return;
    cudaStreamSynchronize(pl.stream);
    for (size_t i = 0; i < pl.prof_part.size(); i++) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pl.prof_ev[2 * i], pl.prof_ev[2 * i + 1]) == cudaSuccess) {
            pl.prof_ms[pl.prof_part[i]] += ms;
            pl.prof_n[pl.prof_part[i]] += 1;
        }
        cudaEventDestroy(pl.prof_ev[2 * i]);
        cudaEventDestroy(pl.prof_ev[2 * i + 1]);
    }
    pl.prof_ev.clear();
    pl.prof_part.clear();
}

template <typename T>
static wfp_status ingest_t(Plan& pl, std::string& err) {
    ProfScope ps0(pl, PP_INGEST);
    constexpr int LP = 32 * sizeof(T) / 16;  // lanes per source
    k_ingest<T><<<nblk(pl.M * LP, 256), 256, 0, pl.stream>>>(pl.d_step, pl.M, pl.d_sig_in, pl.d_src_perm,
                                                               (T*)pl.d_sigwin, pl.NW, (T*)pl.d_siglin,
                                                               (T*)pl.d_sighist, pl.n_hist);
    CK(cudaGetLastError());
    return WFP_OK;
}

// local part, self term and combine on stream st
template <typename T>
static wfp_status localpart_t(Plan& pl, cudaStream_t st, std::string& err) {
    const Params& P = pl.P;
    if (pl.Mt > 0) {
        ProfScope ps(pl, PP_LOCAL);
        local_run(pl, st);
        CK(cudaGetLastError());
    }
    if (pl.n_self > 0) {
        ProfScope ps(pl, PP_SELF);
        k_self<T><<<nblk(pl.n_self, 32), dim3(32, kSelfGroups), 0, st>>>(
            pl.d_step, pl.n_self, pl.d_self_tgt, pl.d_self_src, (const T*)pl.d_sigwin, pl.NW, P.W, pl.n_soe_self,
            pl.d_shead, pl.d_sdecay, pl.d_sw, pl.d_Y, pl.d_uself);
        CK(cudaGetLastError());
    }
    {
        ProfScope ps(pl, PP_COMBINE);
        k_combine<<<nblk(pl.Mt, 256), 256, 0, st>>>(pl.d_step, pl.Mt, pl.d_tgt_perm, pl.d_uloc, pl.d_uh,
                                                    pl.d_uself, pl.d_u_out);
        CK(cudaGetLastError());
    }
    return WFP_OK;
}

template <typename T>
static wfp_status output_t(Plan& pl, std::string& err) {
    wfp_status s = ingest_t<T>(pl, err);
    return s != WFP_OK ? s : localpart_t<T>(pl, pl.stream, err);
}

template <typename T>
static wfp_status exec_r2c(cufftHandle h, T* in, typename Cplx<T>::type* out);
template <>
wfp_status exec_r2c<double>(cufftHandle h, double* in, double2* out) {
    return cufftExecD2Z(h, in, (cufftDoubleComplex*)out) == CUFFT_SUCCESS ? WFP_OK : WFP_ECUDA;
}
template <>
wfp_status exec_r2c<float>(cufftHandle h, float* in, float2* out) {
    return cufftExecR2C(h, in, (cufftComplex*)out) == CUFFT_SUCCESS ? WFP_OK : WFP_ECUDA;
}
template <typename T>
static wfp_status exec_c2c(cufftHandle h, typename Cplx<T>::type* in, typename Cplx<T>::type* out, int dir);
template <>
wfp_status exec_c2c<double>(cufftHandle h, double2* in, double2* out, int dir) {
    return cufftExecZ2Z(h, (cufftDoubleComplex*)in, (cufftDoubleComplex*)out, dir) == CUFFT_SUCCESS ? WFP_OK
                                                                                                   : WFP_ECUDA;
}
template <>
wfp_status exec_c2c<float>(cufftHandle h, float2* in, float2* out, int dir) {
    return cufftExecC2C(h, (cufftComplex*)in, (cufftComplex*)out, dir) == CUFFT_SUCCESS ? WFP_OK : WFP_ECUDA;
}
template <typename T>
static wfp_status exec_c2r(cufftHandle h, typename Cplx<T>::type* in, T* out);
template <>
wfp_status exec_c2r<double>(cufftHandle h, double2* in, double* out) {
    return cufftExecZ2D(h, (cufftDoubleComplex*)in, out) == CUFFT_SUCCESS ? WFP_OK : WFP_ECUDA;
}
template <>
wfp_status exec_c2r<float>(cufftHandle h, float2* in, float* out) {
    return cufftExecC2R(h, (cufftComplex*)in, out) == CUFFT_SUCCESS ? WFP_OK : WFP_ECUDA;
}

template <typename T>
static wfp_status far_t(Plan& pl, cudaStream_t st, std::string& err) {
    using C = typename Cplx<T>::type;
    const Params& P = pl.P;
    ProfScope ps(pl, PP_FAR);
    dim3 blk(32, kFarGroups);
    k_far<T><<<nblk(pl.n_far, 32), blk, 0, st>>>(
        pl.d_step, pl.n_far, pl.n_modes, P.W, P.L, P.Nh, P.nf, P.n_lambda, pl.n_fkappa, pl.d_far_k, pl.d_mode_n,
        pl.d_fac, pl.d_facf, (const C*)pl.d_tc_lag, pl.lag_store ? 0 : 1, (const C*)pl.d_ring_lag, pl.R_lag,
        pl.lag_off, pl.d_H, pl.d_ffir, pl.d_fdecay, pl.d_B, pl.d_aF);
    CK(cudaGetLastError());
    return WFP_OK;
}

// far_elsewhere: the far history of this step was enqueued on another stream (it only reads stored
// levels) and the caller has made this stream wait for it before the mode update
template <typename T>
static wfp_status advance_t(Plan& pl, bool lag_now, std::string& err, cudaEvent_t far_done = nullptr) {
    using C = typename Cplx<T>::type;
    const Params& P = pl.P;
    cudaStream_t st = pl.stream;
    const int nh2 = P.nf / 2 + 1;
    // type-1 spreading: current level and (when active) the lagged level
    if (pl.n_tiles > 0) {
        ProfScope ps(pl, PP_SPREAD);
        spread_t<T>(pl, pl.spread_ts, pl.spread_ch, 0, pl.n_tiles, pl.d_tile_xy, pl.d_tile_ptr, pl.d_tile_src,
                    (T*)pl.d_sp_cur, st);
        CK(cudaGetLastError());
        if (lag_now && !pl.lag_store) {
            spread_t<T>(pl, pl.spread_ts, pl.spread_ch, 1, pl.n_tiles, pl.d_tile_xy, pl.d_tile_ptr, pl.d_tile_src,
                        (T*)pl.d_sp_lag, st);
            CK(cudaGetLastError());
        }
    }
    // two-stage pruned FFT: rows of the band (R2C), the kept columns into the column-major layout,
    // then the columns (C2C, forward, contiguous)
    ProfScope psf(pl, PP_FFT1);
    const dim3 tgrid((unsigned)((P.Nh + 1 + 31) / 32), (unsigned)((P.nb + 31) / 32)), tblk(32, 8);
    if (exec_r2c<T>(pl.fftA, (T*)pl.d_sp_cur, (C*)pl.d_tb_cur + (int64_t)P.lb0 * nh2) != WFP_OK) {
        err = "cufft type-1 row pass failed";
        return WFP_ECUDA;
    }
    k_band_to_cols<C><<<tgrid, tblk, 0, st>>>((const C*)pl.d_tb_cur, (C*)pl.d_tcol_cur, P.nb, P.Nh + 1, nh2, P.nf,
                                              P.lb0);
    CK(cudaGetLastError());
    if (exec_c2c<T>(pl.fftB, (C*)pl.d_tcol_cur, (C*)pl.d_tc_cur, CUFFT_FORWARD) != WFP_OK) {
        err = "cufft type-1 column pass failed";
        return WFP_ECUDA;
    }
    if (lag_now && !pl.lag_store) {
        if (exec_r2c<T>(pl.fftA, (T*)pl.d_sp_lag, (C*)pl.d_tb_lag + (int64_t)P.lb0 * nh2) != WFP_OK) {
            err = "cufft lagged type-1 failed";
            return WFP_ECUDA;
        }
        k_band_to_cols<C><<<tgrid, tblk, 0, st>>>((const C*)pl.d_tb_lag, (C*)pl.d_tcol_lag, P.nb, P.Nh + 1, nh2,
                                                  P.nf, P.lb0);
        CK(cudaGetLastError());
        if (exec_c2c<T>(pl.fftB, (C*)pl.d_tcol_lag, (C*)pl.d_tc_lag, CUFFT_FORWARD) != WFP_OK) {
            err = "cufft lagged type-1 failed";
            return WFP_ECUDA;
        }
    }
    psf.stop();
    const bool far_now = lag_now && P.far_active && pl.n_far > 0;
    if (far_now) {
        if (far_done) {
            CK(cudaStreamWaitEvent(st, far_done, 0));
        } else {
            wfp_status sf = far_t<T>(pl, st, err);
            if (sf != WFP_OK) return sf;
        }
    }
    const int64_t n_far_now = far_now ? pl.n_far : 0;
    double coef2 = (P.dk / (2 * kPi)) * (P.dk / (2 * kPi));
    ProfScope psm(pl, PP_MODES);
    const int64_t near_sq = (int64_t)std::floor((P.K / P.dk) * (P.K / P.dk));
    if constexpr (sizeof(T) == 8) {
        k_modes<T><<<nblk(pl.n_modes, 256), 256, 0, st>>>(
            pl.d_step, pl.n_modes, P.W, P.L, P.Nh, P.nf, pl.d_mode_n, pl.d_mode_k, pl.d_fac, coef2,
            (const C*)pl.d_tc_cur, (const C*)pl.d_tc_lag, (C*)pl.d_ring, (C*)pl.d_ring_lag, pl.R_cur, pl.R_lag,
            pl.lag_off, pl.lag_store ? 0 : 1, (const T*)pl.d_taps, pl.d_rot, pl.d_alpha, pl.d_alphad, (C*)pl.d_td,
            near_sq, pl.d_aF, n_far_now);
    } else {
        auto kern = pl.compact_taps ? k_modes_one<true> : k_modes_one<false>;
        kern<<<nblk(pl.n_modes, 256), 256, 0, st>>>(
            pl.d_step, pl.n_modes, P.W, P.L, P.Nh, P.nf, pl.d_mode_n, pl.d_mode_k, pl.d_facf, (float)coef2,
            (const float2*)pl.d_tc_cur, (const float2*)pl.d_tc_lag, (float2*)pl.d_ring, (float2*)pl.d_ring_lag,
            pl.R_cur, pl.R_lag, pl.lag_off, pl.lag_store ? 0 : 1, (const float*)pl.d_taps, pl.d_rot, pl.d_alpha,
            pl.d_alphad, (float2*)pl.d_td, near_sq, pl.d_aF, n_far_now);
    }
    CK(cudaGetLastError());
    psm.stop();
    // type-2: columns (C2C, inverse) then band rows (C2R); the C2R input beyond column Nh is re-zeroed
    ProfScope ps2(pl, PP_FFT2);
    if (exec_c2c<T>(pl.fftBi, (C*)pl.d_td, (C*)pl.d_te2, CUFFT_INVERSE) != WFP_OK) {
        err = "cufft type-2 column pass failed";
        return WFP_ECUDA;
    }
    k_cols_to_band<C><<<tgrid, tblk, 0, st>>>((const C*)pl.d_te2, (C*)pl.d_te, P.nb, P.Nh + 1, nh2, P.nf, P.lb0);
    CK(cudaGetLastError());
    if (nh2 > P.Nh + 1)
        CK(cudaMemset2DAsync((C*)pl.d_te + (int64_t)P.lb0 * nh2 + (P.Nh + 1), nh2 * sizeof(C), 0,
                             (nh2 - P.Nh - 1) * sizeof(C), P.nb, st));
    if (exec_c2r<T>(pl.fftAi, (C*)pl.d_te + (int64_t)P.lb0 * nh2, (T*)pl.d_tf) != WFP_OK) {
        err = "cufft type-2 row pass failed";
        return WFP_ECUDA;
    }
    ps2.stop();
    ProfScope psi(pl, PP_INTERP);
    if (P.w <= 16)
        k_interp<T, 16><<<nblk(pl.Mt * 16, 256), 256, 0, st>>>(pl.d_step, pl.Mt, pl.d_tgt_off,
                                                               (const T*)pl.d_tgt_ker, P.w, (const T*)pl.d_tf, P.nf,
                                                               P.lb0, pl.d_uh);
    else
        k_interp<T, 32><<<nblk(pl.Mt * 32, 256), 256, 0, st>>>(pl.d_step, pl.Mt, pl.d_tgt_off,
                                                               (const T*)pl.d_tgt_ker, P.w, (const T*)pl.d_tf, P.nf,
                                                               P.lb0, pl.d_uh);
    CK(cudaGetLastError());
    return WFP_OK;
}

wfp_status step_output(Plan& pl, std::string& err) {
    return pl.P.precision == WFP_FP64 ? output_t<double>(pl, err) : output_t<float>(pl, err);
}

wfp_status step_advance_body(Plan& pl, bool lag_now, std::string& err) {
    return pl.P.precision == WFP_FP64 ? advance_t<double>(pl, lag_now, err) : advance_t<float>(pl, lag_now, err);
}

wfp_status step_tick(Plan& pl, std::string& err) {
    k_tick<<<1, 1, 0, pl.stream>>>(pl.d_step);
    CK(cudaGetLastError());
    return WFP_OK;
}

// One whole step: ingest on the plan's stream, then the local part / self term / combine on the
// side stream concurrently with the advance (spreading, FFTs, modes, far history, interpolation) on
// the plan's stream; both join before the step counter moves.  The two branches share no written
// buffer: u_h is double-buffered by step parity.
template <typename T>
static wfp_status concurrent_t(Plan& pl, bool do_advance, bool lag_now, std::string& err) {
    wfp_status s = ingest_t<T>(pl, err);
    if (s != WFP_OK) return s;
    CK(cudaEventRecord(pl.ev_fork, pl.stream));
    CK(cudaStreamWaitEvent(pl.stream2, pl.ev_fork, 0));
    s = localpart_t<T>(pl, pl.stream2, err);
    if (s != WFP_OK) return s;
    CK(cudaEventRecord(pl.ev_join, pl.stream2));
    if (do_advance) {
        // with the S history stored the far history reads only old levels: a third branch
        cudaEvent_t far_done = nullptr;
        if (lag_now && pl.P.far_active && pl.n_far > 0 && pl.lag_store) {
            CK(cudaStreamWaitEvent(pl.stream3, pl.ev_fork, 0));
            s = far_t<T>(pl, pl.stream3, err);
            if (s != WFP_OK) return s;
            CK(cudaEventRecord(pl.ev_far, pl.stream3));
            far_done = pl.ev_far;
        }
        s = advance_t<T>(pl, lag_now, err, far_done);
        if (s != WFP_OK) return s;
    }
    CK(cudaStreamWaitEvent(pl.stream, pl.ev_join, 0));
    return step_tick(pl, err);
}

wfp_status step_concurrent(Plan& pl, bool do_advance, bool lag_now, std::string& err) {
    return pl.P.precision == WFP_FP64 ? concurrent_t<double>(pl, do_advance, lag_now, err)
                                      : concurrent_t<float>(pl, do_advance, lag_now, err);
}

}  // namespace wfp
