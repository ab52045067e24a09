// Device-side plan of the 2D TK-WFP evaluator: buffers, tables and state (CUDA path).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdint>
#include <string>
#include <vector>

#include "wfp_internal.h"

namespace wfp {

// Device memory owned by a plan; freed in reverse order of allocation.
struct DevArena {
    std::vector<void*> ptrs;
    int64_t bytes = 0;
    template <typename T>
    cudaError_t alloc(T** p, size_t count) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
        if (e != cudaSuccess) return e;
        ptrs.push_back(q);
        bytes += (int64_t)(count * sizeof(T));
        *p = (T*)q;
        return cudaMemsetAsync(q, 0, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    }
    void release() {
        for (auto it = ptrs.rbegin(); it != ptrs.rend(); ++it) cudaFree(*it);
        ptrs.clear();
        bytes = 0;
    }
};

struct Plan {
    Params P;
    wfp_opts opts;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // side stream of a step: the local part and self term run on it concurrently with the advance
    cudaStream_t stream2 = nullptr;
    cudaStream_t stream3 = nullptr;  // far history (stored S history only)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_far = nullptr;
    bool poisoned = false;
    int64_t step = 0;  // completed steps
    // device footprint by role: local part (pair lists, weights or factored records), fine grids and
    // spectra, carried state (signal windows and history, mode amplitudes, S levels, far and self
    // recurrences, outputs); cuFFT work areas (not in mem)
    int64_t bytes_local = 0, bytes_grid = 0, bytes_history = 0, bytes_fft_work = 0;
    uint64_t inputs_hash = 0;  // coordinates, dt, N_t, band limit, tol and result-changing options
    bool serial_step = false;  // the step's two branches one after the other on the plan's stream
    int device = 0;
    DevArena mem;

    // step counter on the device (kernels read it, so the step can be captured in a graph)
    int64_t* d_step = nullptr;

    // ------------------------------------------------------------ geometry (internal order)
    int64_t M = 0, Mt = 0;
    int* d_src_perm = nullptr;   // internal source k -> caller index
    int* d_tgt_perm = nullptr;   // internal target k -> caller index
    int NW = 32;                 // sigma window length (power of two >= nmax)

    // local part (Sec. 6): CSR by internal target, weights [pair][NW]
    int64_t n_pairs = 0;         // source-target pairs with 0 < r < delta
    int64_t n_slots = 0;         // pair slots: each row padded to a multiple of 4 (zero weights)
    int64_t* d_rowptr = nullptr;
    int* d_col = nullptr;
    void* d_eta = nullptr;       // NW = 32: row position 32 - nmax + l holds eta_l (aligned with d_siglin)
    // factored form (WFP_LOCAL_FACTORED): pairs with r >= dt as {source | (k - 1) << 26, x} with x the
    // Chebyshev variable of their delay interval k; the pairs with r < dt keep d_rowptr / d_col /
    // d_eta above (rows not padded)
    bool local_factored = false;
    int NC = 0;                  // Chebyshev coefficients kept per interval (multiple of 4)
    int64_t n_tab = 0, n_near = 0;
    int64_t* d_trow = nullptr;   // [Mt + 1] table-pair rows
    void* d_tpair = nullptr;     // [n_tab] TabPair<T>
    void* d_ctab = nullptr;      // [W - 1][32][NC] series coefficients by window position, reduced precision
    void* d_ycoef = nullptr;     // [W - 1][M][NC] per step: windows contracted with d_ctab

    // sigma storage
    void* d_sigwin = nullptr;    // [M][NW] window of the last NW levels (slot = level & (NW-1)), reduced precision
    void* d_siglin = nullptr;    // [M][32] the last 32 levels oldest first (NW = 32 only), reduced precision
    void* d_sighist = nullptr;   // [n_hist][M] in the grid precision (slot = level % n_hist)
    int n_hist = 1;
    double* d_sig_in = nullptr;  // caller-order sigma_n staged on the device

    // NUFFT (type-1 and type-2)
    int* d_src_off = nullptr;    // [M] packed (ix0, iy0) band-relative footprint origin
    void* d_src_ker = nullptr;   // [M][2w] kernel values (x then y), grid precision
    int* d_tgt_off = nullptr;    // [Mt]
    void* d_tgt_ker = nullptr;   // [Mt][2w]
    int local_variant = 1;       // local-part kernel variant (NW = 32), all bit-identical
    int spread_ts = 32;          // spreading tile side (16 or 32)
    int spread_ch = 64;          // sources staged per round (32 or 64)
    int n_tiles = 0;             // non-empty spreading tiles
    int* d_tile_xy = nullptr;    // [n_tiles] packed (tx, ty)
    int* d_tile_ptr = nullptr;   // [n_tiles + 1]
    int* d_tile_src = nullptr;   // sources per tile (internal index), fixed order
    void* d_sp_cur = nullptr;    // [nb][nf] real spread grid (current)
    void* d_sp_lag = nullptr;    // [nb][nf] real spread grid (lagged)
    void* d_tb_cur = nullptr;    // [nf][nf/2+1] complex: row transforms of the band (band rows only)
    void* d_tb_lag = nullptr;
    void* d_tcol_cur = nullptr;  // [Nh+1][nf] complex: their kept columns, column-major (rows outside the band stay zero)
    void* d_tcol_lag = nullptr;
    void* d_tc_cur = nullptr;    // [Nh+1][nf] complex: type-1 result before deconvolution, column-major
    void* d_tc_lag = nullptr;
    void* d_td = nullptr;        // [Nh+1][nf] complex: type-2 coefficients (conjugated), column-major
    void* d_te2 = nullptr;       // [Nh+1][nf] complex: their column transforms
    void* d_te = nullptr;        // [nf][nf/2+1] complex: band rows of those, for the row transforms
    void* d_tf = nullptr;        // [nb][nf] real: type-2 grid in the band
    double* d_fac = nullptr;     // [Nh+1] (-1)^n h / psihat(n)
    float* d_facf = nullptr;     // the same in FP32 (mixed-path deconvolution)
    cufftHandle fftA = 0, fftB = 0, fftBi = 0, fftAi = 0;
    bool fft_made[4] = {false, false, false, false};

    // near-history modes (Sec. 4): half-plane disk, ordered by |n|^2
    int64_t n_modes = 0, n_kappa = 0;
    int2* d_mode_n = nullptr;    // (n1, n2)
    int* d_mode_k = nullptr;     // distinct-|k| index
    bool compact_taps = false;   // mixed path without lag: taps hold p and q only (4 floats per level)
    void* d_taps = nullptr;      // [n_kappa][4W] p, q, pA, qA (Eq. hggrid), step dt folded in (mixed: FP32 hi/lo pairs, [8W]; [4W] of p and q when compact_taps)
    double* d_rot = nullptr;     // [n_kappa][3] cos(k dt), sin(k dt)/k, k sin(k dt)
    double2* d_alpha = nullptr;  // [n_modes]
    double2* d_alphad = nullptr; // [n_modes]
    void* d_ring = nullptr;      // [R_cur][n_modes] S by level: level l in slot l mod R_cur
    void* d_ring_lag = nullptr;  // [R_lag][n_modes] lagged S: level l in slot (l + lag_off) mod R_lag
    bool lag_store = false;      // S history kept (R_cur = L + W, ring_lag = ring) instead of a lagged NUFFT
    int R_cur = 0, R_lag = 0, lag_off = 0;

    // far history (Sec. 5)
    int64_t n_far = 0, n_fkappa = 0;
    int* d_far_mode = nullptr;   // [n_far] mode index
    int* d_far_k = nullptr;      // [n_far] far-|k| index
    double* d_H = nullptr;       // [n_lambda][n_fkappa] Hankel coefficients (Eq. H) times d_fforce[l]
    double* d_ffir = nullptr;    // [n_fkappa][W-1] taps of the newest lagged levels, Phi_q(|k|)
    double* d_fdecay = nullptr;  // [n_lambda] r_l = exp(-lambda_l dt)
    double* d_fforce = nullptr;  // [n_lambda] a_l r_l^(W-1): weight of S_{n-L-W+1} in the tail recurrence
    double2* d_B = nullptr;      // [n_lambda][n_far] tail state E_l / d_fforce[l] (E_l carries exp(A lambda_l), Eq. beta0)
    double2* d_aF = nullptr;     // [n_far] alpha_F of the current step, added by the mode update

    // self term of coincident pairs
    int64_t n_self = 0;
    int n_soe_self = 0;
    int* d_self_tgt = nullptr;   // internal target
    int* d_self_src = nullptr;   // internal source
    double* d_shead = nullptr;   // [W-1] shared window weights g_q
    double* d_sdecay = nullptr;  // [n_soe_self] r_l = exp(-mu_l dt)
    double* d_sw = nullptr;      // [n_soe_self] SOE weights * dt * r_l^W / (2 pi)
    double* d_Y = nullptr;       // [n_soe_self][n_self] tail state Z_l / r_l^W

    // outputs (internal target order)
    double* d_uloc = nullptr;
    double* d_uh = nullptr;      // [2][Mt] u_h by step parity: step n reads slot n & 1, its advance writes (n+1) & 1
    double* d_uself = nullptr;
    double* d_u_out = nullptr;   // caller order

    // device-side error flag (a bounded wait that ran out), host-mapped pinned memory
    int* h_err = nullptr;
    int* d_err = nullptr;
    int* d_sched = nullptr;      // row counter and finished-warp count of the persistent local kernel

    // host staging
    double* h_sig = nullptr;     // pinned
    double* h_u = nullptr;       // pinned
    cudaEvent_t ev_out = nullptr;

    // graphs: 0 output phase, 1 advance without lag, 2 advance with lag, 3 final tick
    bool use_graph = true;
    cudaGraphExec_t graph_exec[4] = {nullptr, nullptr, nullptr, nullptr};
    int graph_uses[4] = {0, 0, 0, 0};

    // phi table (device)
    double* d_phicoef = nullptr;

    // per-part timing with CUDA events on the plan's stream (graphs are bypassed while enabled)
    bool prof = false;
    std::vector<cudaEvent_t> prof_ev;      // pairs (start, stop)
    std::vector<int> prof_part;            // part id of each pair
    double prof_ms[16] = {0};
    int64_t prof_n[16] = {0};
};

enum ProfPart {
    PP_INGEST = 0, PP_LOCAL, PP_SELF, PP_COMBINE, PP_SPREAD, PP_FFT1, PP_MODES, PP_FAR, PP_FFT2, PP_INTERP,
    PP_COPY, PP_NPARTS
};
extern const char* const kPartNames[PP_NPARTS];

// Record an event pair around a part when profiling is on.
struct ProfScope {
    Plan& pl;
    int part;
    cudaEvent_t e1 = nullptr;
    ProfScope(Plan& p, int part_) : pl(p), part(part_) {
        if (!pl.prof) return;
        cudaEvent_t e0;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, pl.stream);
        pl.prof_ev.push_back(e0);
        pl.prof_ev.push_back(e1);
        pl.prof_part.push_back(part);
    }
    void stop() {
        if (pl.prof && e1) cudaEventRecord(e1, pl.stream);
        e1 = nullptr;
    }
    ~ProfScope() { stop(); }
};
void prof_collect(Plan& pl);  // synchronise and fold recorded pairs into prof_ms / prof_n
wfp_status plan_step_device(Plan& pl, double* u_dev, std::string& err);
void local_bulk_setup();  // raises the dynamic shared-memory limit of the staged local kernels
constexpr int kLocalVariants = 5;  // 1 = warp-vector loads, 2..5 = bulk-staged configurations
void local_launch(const Plan& pl, int variant, cudaStream_t st);
void local_run(const Plan& pl, cudaStream_t st);  // the plan's local-part kernel(s)
int factored_nc_supported(int nc, bool fp64);      // coefficient count the factored kernels use for nc
// one spreading launch with the given tiling (plan-time autotuner and step loop)
void spread_launch(const Plan& pl, int ts, int ch, int lag, int n_tiles, const int* txy, const int* tptr,
                   const int* tsrc, void* sp, cudaStream_t st);  // input already in d_sig_in
Plan& plan_of(wfp_plan h);

wfp_status plan_build(Plan& pl, const double* src_xy, const double* tgt_xy, std::string& err);
void plan_free(Plan& pl);
wfp_status step_output(Plan& pl, std::string& err);   // ingest, local, self, combine (device)
wfp_status step_advance_body(Plan& pl, bool lag_now, std::string& err);  // NUFFTs, modes, far, interp
wfp_status step_tick(Plan& pl, std::string& err);     // advance the device step counter
// the whole step with the local part and self term on stream2, concurrent with the advance
wfp_status step_concurrent(Plan& pl, bool do_advance, bool lag_now, std::string& err);

}  // namespace wfp
