/*
 * wfp.h -- C ABI of the GB300 (sm_103a) evaluator of the 2D free-space wave field of M
 * point sources, by the truncated-kernel windowed Fourier projection (2D TK-WFP) method of
 * Al Hassanieh, Greengard & Barnett, "A spectral method for the rapid evaluation of
 * hyperbolic potentials in two dimensions using windowed Fourier projection".
 *
 * Problem (Sec. 1, Eqs. wave2d, solnRep, Green, pointSources): with unit wave speed and
 * zero initial data, the field at target x_i and time t_n = n dt is
 *
 *     u(x_i, t_n) = sum_j int_0^{t_n} G(x_i - y_j, t_n - tau) sigma_j(tau) dtau,
 *     G(x, t)     = H(t - |x|) / (2 pi sqrt(t^2 - |x|^2)),
 *
 * where sigma_j(t) = 0 for t <= 0.  Pairs with coincident source and target are excluded
 * from the sum, as in the paper's reference formula (Sec. 7, Eq. exactSol).
 *
 * Each call of wfp_step takes the M samples sigma_j(t_n) of the current step and returns
 * u(x_i, t_n) at the Mt targets.  Internally the field is split (Sec. 3, Eq. split) into a
 * local part (direct quadrature, Sec. 6), a near history (Fourier modes advanced by a Duhamel
 * recurrence and fed by type-1/type-2 NUFFTs, Sec. 4) and a far history (sum-of-exponentials
 * recurrences, Sec. 5), all evaluated on the GPU.
 *
 * Conventions for every entry point:
 *   - Return codes only: no exceptions cross the ABI, nothing aborts or traps.
 *   - The caller owns every buffer it passes; the plan owns all memory it allocates.
 *   - Coordinates and times are in the caller's units; the library normalises them.
 *   - After WFP_ECUDA a plan is poisoned: every later call except wfp_destroy returns
 *     WFP_ESTATE.
 *   - One plan must not be used from two threads at once; distinct plans are independent.
 *   - A NULL stream means the calling thread's default stream (the library is built with
 *     per-thread default streams), so plans created on different threads do not serialise.
 *   - wfp_last_error() returns a thread-local message describing the last failure.
 */
#ifndef WFP_H
#define WFP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WFP_OK = 0,
    WFP_EINVAL = 1,        /* invalid argument (sizes, NaN/Inf coordinates, dt too coarse for the band limit) */
    WFP_ENOMEM = 2,        /* device or pinned-host allocation failed; nothing is left allocated */
    WFP_ECUDA = 3,         /* a CUDA or cuFFT call failed; the plan is poisoned */
    WFP_ESTATE = 4,        /* call not valid in the plan's state (e.g. step beyond Nt, poisoned plan) */
    WFP_ETIMEOUT = 5,      /* a bounded device-side wait ran out (server) */
    WFP_EUNSUPPORTED = 6   /* option combination not supported */
} wfp_status;

enum { WFP_FP64 = 0, WFP_MIXED = 1 };

/*
 * Options.  wfp_opts_default() fills every field; zero in a numeric field means "derive".
 *   precision     WFP_FP64: every step in FP64.  WFP_MIXED: spreading, interpolation, FFTs,
 *                 FIR taps and local weights in FP32; mode state, its per-step rotation, the
 *                 sum-of-exponentials recurrences and all accumulations across sources in FP64.
 *   eps           internal tolerance epsilon; 0 => tol/1000.  b = ln(1/eps) (Sec. 2.1).
 *   W             blending width in steps, delta = W dt (Eq. W); 0 => ceil(delta / dt) when delta > 0,
 *                 else ceil(2b/(pi - K0 dt)) (Eq. dt).  2 <= W <= 59 and Eq. dt must hold.
 *   p             interpolation order of the local part (Sec. 6); 0 => 20, lowered (even, >= 8) so
 *                 that nmax = W + 1 + p/2 fits a 32-level window, or else a 64-level one.
 *   delta         fixed blending width in the caller's time units (the fixed-delta variant of the
 *                 paper's remark on small time steps: delta stays put as dt shrinks and W grows);
 *                 0 => derived from W as above.
 *   Kf            far-history cut-off wavenumber in normalised units (Sec. 5); 0 => derived from eps.
 *   upsampfac     minimum NUFFT fine-grid upsampling factor; 0 => 1.25 on the FP64 path; on the MIXED path
 *                 2.0 while that keeps the grid at most 4096 points a side, else 1.25.  The grid
 *                 size n_f is the smallest 2^a, 3*2^a or 9*2^a at or above upsampfac * (2 Nh + 1).
 *   kernel_width  NUFFT spreading-kernel width in grid points; 0 => from eps and the effective
 *                 upsampling n_f / (2 Nh + 1).
 *   soe_nodes     Gauss-Legendre nodes per dyadic panel of the far sum of exponentials
 *                 (Sec. 2.3, Eq. LaplaceApprox); 0 => the smallest of 16..32 meeting eps.
 *   exclude_self  1 (default): for a target coincident with a source (distance <= 1e-12 of the
 *                 domain size) the self term is excluded, as in Eq. exactSol.
 *   stream        cudaStream_t to run on, or NULL for a plan-owned stream.
 *   use_graph     1 (default): the per-step device work is captured once into a CUDA graph.
 *   lag_mode      how S(k, t - A+ + delta) reaches the removal term of Eq. hggrid:
 *                 WFP_LAG_RECOMPUTE recomputes it each step by a second (lagged) type-1 NUFFT of
 *                 the stored signal history, as the paper does (Sec. 4.3); WFP_LAG_STORE keeps the
 *                 last L + W levels of S per mode in device memory; WFP_LAG_AUTO (0, default) stores
 *                 when that history takes at most 40% of the free device memory, else recomputes.
 *   spread_tile   side of the grid tile one CTA spreads onto (8, 16 or 32); 0 => chosen at plan time
 *                 by timing each.  spread_chunk: entries of a tile's source list each warp scans per
 *                 round (32 or 64); 0 => timed likewise.  Every grid point sums the sources that cover
 *                 it in one fixed order (by the residue of the source index modulo 4, ascending index
 *                 within a residue class, the four partial sums added in class order) whatever the
 *                 tiling, so these choices do not change any result bit.
 *   local_variant kernel of the local part when nmax <= 32: 1 = warp-vector loads, 2..5 = weight rows
 *                 staged into shared memory by bulk asynchronous copies (four stage/CTA shapes);
 *                 0 => the fastest, timed at plan time.  All variants give the same bits.
 *   local_interp  interpolant of the signal inside the local quadrature (Sec. 6): WFP_INTERP_HYBRID
 *                 (0, default) fits the newest four intervals by band-limited least squares and uses
 *                 p-point Lagrange elsewhere; WFP_INTERP_LAGRANGE uses p-point Lagrange on the p nearest
 *                 grid values everywhere, as the paper does (order-p convergence, Sec. 7).
 *   local_form    how the local weights eta_l(r_ij) of Sec. 6 reach the step.  WFP_LOCAL_STORED: one
 *                 row of nmax weights per pair, computed at plan time and streamed from device memory
 *                 every step.  WFP_LOCAL_FACTORED: on each delay interval [k dt, (k+1) dt], k >= 1, the
 *                 weights are a Chebyshev series in v = sqrt((k+1) dt - r); the step first contracts
 *                 each source's signal window with the series coefficients (y_{j,k,c}, per source,
 *                 interval and coefficient) and each pair then sums T_c(v_ij) y_{j,k,c} -- the same
 *                 weights, factored, with a pair costing 8 bytes (16 in FP64) instead of a weight row;
 *                 pairs with r < dt keep stored rows.  The series is cut after the first coefficient
 *                 count (a multiple of 4) whose dropped tail is below the path's rounding (below 2^-25
 *                 of the interval's weight scale on the MIXED path, rounded up to 16 or 32 for its
 *                 kernels; every coefficient on the FP64 path); wfp_plan_get_info reports the count
 *                 and wfp_debug_factored_table the table and the tail.  WFP_LOCAL_AUTO (0, default):
 *                 FACTORED on the MIXED path, STORED on the FP64 path (where the stored form needs
 *                 fewer FP64 operations per pair).  FACTORED needs nmax <= 32 and 8 (W - 1) M < 2^32.
 *   step_order    how a step's two independent branches (local part / self term / output, and the
 *                 advance: NUFFTs, modes, far history) are issued.  WFP_ORDER_CONCURRENT: on two
 *                 (three) streams joined at the end of the step, so small problems fill the device;
 *                 WFP_ORDER_SERIAL: one after the other on the plan's stream, so large problems do not
 *                 compete for L2 and HBM bandwidth; WFP_ORDER_AUTO (0, default): serial when the local
 *                 part has at least 2e8 source-target pairs, else concurrent.  The branches share no
 *                 written buffer, so both orders give the same bits.
 */
typedef struct {
    int precision;
    double eps;
    int W;
    int p;
    double Kf;
    double upsampfac;
    int kernel_width;
    int soe_nodes;
    int exclude_self;
    void* stream;
    int use_graph;
    int lag_mode;
    int spread_tile;
    int spread_chunk;
    int local_variant;
    int local_interp;
    double delta;
    int local_form;
    int step_order;
} wfp_opts;

enum { WFP_INTERP_HYBRID = 0, WFP_INTERP_LAGRANGE = 1 };

enum { WFP_LOCAL_AUTO = 0, WFP_LOCAL_STORED = 1, WFP_LOCAL_FACTORED = 2 };

enum { WFP_LAG_AUTO = 0, WFP_LAG_RECOMPUTE = 1, WFP_LAG_STORE = 2 };

enum { WFP_ORDER_AUTO = 0, WFP_ORDER_CONCURRENT = 1, WFP_ORDER_SERIAL = 2 };

/*
 * Derived parameters of a plan (normalised units: the bounding square of all points is
 * mapped onto B = [-1,1]^2 by x -> (x - c) * scale, t -> t * scale; the field is invariant).
 */
typedef struct {
    double scale, cx, cy;            /* normalisation */
    double dt, T, K0;                /* normalised step, end time, band limit */
    double eps, b;                   /* tolerance, KB shape parameter */
    int W, p, nmax;                  /* blending width (steps), interpolation order, local levels */
    double delta, K, A, Aplus, dk;   /* Eqs. W, K, A, Ap, dk */
    int L;                           /* lag in steps: A+ - delta = L dt */
    double Kf;                       /* far cut-off */
    int Nh;                          /* modes n in [-Nh, Nh]^2 */
    int64_t n_modes, n_far_modes;    /* half-plane disk modes (near), (far) */
    int64_t n_kappa;                 /* distinct |k| among near modes */
    int n_lambda, soe_panels, soe_nodes;  /* far sum of exponentials */
    int n_self_soe;                  /* self-term sum of exponentials */
    int nf, nb, kernel_width;        /* NUFFT fine grid, band, spreading width */
    double upsampfac;
    int64_t n_pairs;                 /* local source-target pairs */
    int64_t n_self;                  /* coincident targets */
    int lag_active, far_active;
    int precision;
    int64_t device_bytes;            /* device memory held by the plan */
    int lag_store;                   /* 1: S history stored (L + W levels), 0: lagged NUFFT */
    int64_t s_levels;                /* levels of S kept per mode */
    int spread_tile, spread_chunk;   /* spreading tile side and staging chunk in use */
    int local_variant;               /* local-part kernel variant in use (0: 64-level window form
                                        or the factored form) */
    int local_form;                  /* WFP_LOCAL_STORED or WFP_LOCAL_FACTORED, as built */
    int local_nc;                    /* Chebyshev coefficients per interval (factored form), else 0 */
    int64_t n_near_pairs;            /* pairs with r < dt (stored weight rows in the factored form) */
    int64_t n_spread_tiles;          /* non-empty spread_tile x spread_tile tiles of the fine-grid band
                                        (the part of the band that spreading writes and interpolation reads) */
    int64_t bytes_local;             /* device_bytes held by the local part (pair lists, weight rows or
                                        factored records, series table and the per-step contraction) */
    int64_t bytes_grid;              /* ... by the NUFFT fine-grid band and the pruned spectra */
    int64_t bytes_history;           /* ... by the carried state: signal windows and history, mode amplitudes
                                        alpha and alpha-dot, the S levels, far and self recurrence states */
    int64_t bytes_fft_work;          /* cuFFT work areas (held by the plan, not counted in device_bytes) */
    int step_order;                  /* WFP_ORDER_CONCURRENT or WFP_ORDER_SERIAL, as built */
} wfp_info;

typedef struct wfp_plan_s* wfp_plan;

/* Fill *opts with the defaults described above. */
void wfp_opts_default(wfp_opts* opts);

/*
 * Create a plan (Sec. 1 problem statement; parameters per Secs. 2-6).
 *   M, src_xy     number of sources (>= 1) and their coordinates, 2*M doubles interleaved (x, y),
 *                 host memory, read during the call only.
 *   Mt, tgt_xy    number of targets (>= 1) and coordinates (host, 2*Mt doubles); may alias src_xy.
 *   dt, Nt        time step (> 0) and the number of steps the plan will be stepped (>= 1).
 *   band_limit    K0, the epsilon-bandwidth of the signals in rad per unit time (Thm. 4.1);
 *                 K0 * dt must be below pi - 2b/W for some W <= 64 (Eq. dt), else WFP_EINVAL.
 *   tol           target accuracy of the field (e.g. 1e-6); 0 < tol < 1.
 *   opts          NULL for defaults.
 *   out           receives the plan handle (NULL on failure).
 * Errors: WFP_EINVAL (bad sizes / NaN / Inf / dt too coarse), WFP_ENOMEM, WFP_ECUDA.
 * The call runs the plan-time precomputation (neighbour lists, local weights, FIR taps,
 * Hankel coefficients, NUFFT set-up) on the current CUDA device and synchronises.
 */
wfp_status wfp_plan_create(int64_t M, const double* src_xy, int64_t Mt, const double* tgt_xy, double dt,
                           int64_t Nt, double band_limit, double tol, const wfp_opts* opts, wfp_plan* out);

/*
 * Advance one step (Secs. 4.3, 5.1, 6): ingest sigma_j(t_n), n = 1, 2, ..., Nt, and write
 * u(x_i, t_n).
 *   sigma_n   M doubles (host or device pointer; detected with cudaPointerGetAttributes).
 *   u_n       Mt doubles (host or device pointer).
 * With host pointers the call returns when u_n is written.  With device pointers the work
 * is ordered on the plan's stream and the call returns after enqueueing it.  Page-locked host
 * buffers (cudaHostAlloc, cudaMallocHost, cudaHostRegister) are copied to and from the device
 * directly; pageable ones go through the plan's own page-locked stage (one host memcpy each way).
 * Errors: WFP_EINVAL (NULL pointer), WFP_ESTATE (more than Nt steps, poisoned plan), WFP_ECUDA.
 */
wfp_status wfp_step(wfp_plan plan, const double* sigma_n, double* u_n);

/* Free everything the plan holds.  NULL is accepted. */
wfp_status wfp_destroy(wfp_plan plan);

/* Derived parameters and memory footprint of a plan. */
wfp_status wfp_plan_get_info(wfp_plan plan, wfp_info* info);

/*
 * Per-part outputs of the last completed step, for diagnostics (host arrays of Mt doubles,
 * any may be NULL): u_local (Sec. 6, Eq. ul), u_hist (near + far history, Eqs. unh + ufh,
 * including the self contribution of coincident pairs), u_self (the coincident-pair term
 * subtracted when exclude_self is set).  u = u_local + u_hist - u_self.
 */
wfp_status wfp_step_components(wfp_plan plan, double* u_local, double* u_hist, double* u_self);

/*
 * Per-part timing with CUDA events recorded on the plan's stream around each part of a step
 * (ingest, local, self, combine, spread, fft_type1, modes, far, fft_type2, interp, copy).
 * wfp_profile(plan, 1) resets the totals and starts recording (CUDA graphs are bypassed while
 * recording); wfp_profile(plan, 0) stops.  wfp_profile_read synchronises the stream and returns,
 * for up to max_parts parts, the part names (static strings), the total milliseconds and the
 * number of timed launches; *n_parts receives the number of parts.  Any output array may be NULL.
 */
wfp_status wfp_profile(wfp_plan plan, int enable);
wfp_status wfp_profile_read(wfp_plan plan, int max_parts, const char** names, double* total_ms, int64_t* launches,
                            int* n_parts);

/*
 * Derived parameters without creating a plan or touching a GPU (host-only):
 * same arguments as wfp_plan_create except the coordinates, replaced by the half-side
 * `halfside` of the bounding square.  Fills the normalisation-independent fields of *info.
 */
wfp_status wfp_select_params(double halfside, double dt, int64_t Nt, double band_limit, double tol,
                             const wfp_opts* opts, wfp_info* info);

/*
 * Checkpoint and resume.  The state a plan carries from step to step -- the step count, the
 * signal windows and history, the stored S levels, the mode amplitudes alpha and alpha-dot
 * (Sec. 4), the far-history and self-term recurrence states (Sec. 5) and the near-history field
 * u_h left for the next step -- is written to, or read from, a caller-owned host buffer.
 *   wfp_checkpoint_size: *bytes receives the buffer size the plan needs.
 *   wfp_checkpoint_save: synchronises the plan's stream and copies the state into buf (bytes >= size).
 *   wfp_checkpoint_load: copies a saved state into a plan created from the same inputs and options
 *                        (checked against the derived parameters and sizes and a 64-bit hash of the
 *                        coordinates, dt, N_t, band limit, tolerance and the options that change
 *                        results; a mismatch returns WFP_EINVAL and leaves the plan unchanged).  Stepping then
 *                        continues from the saved step and gives the same bits as the plan that was
 *                        saved.
 * Errors: WFP_EINVAL (NULL, short buffer, mismatch), WFP_ESTATE (poisoned plan), WFP_ECUDA.
 */
wfp_status wfp_checkpoint_size(wfp_plan plan, int64_t* bytes);
wfp_status wfp_checkpoint_save(wfp_plan plan, void* buf, int64_t bytes);
wfp_status wfp_checkpoint_load(wfp_plan plan, const void* buf, int64_t bytes);

/*
 * Local part of one step without any allocation.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need the result -- code whose
 * device memory all comes from a fixed arena or pool that the application reserved up front and
 * that it may not grow, and real-time loops where an allocation's latency, and the device-wide
 * synchronisation that cudaMalloc and cudaFree can cause, are not allowed.  A plan allocates its
 * tables and state in wfp_plan_create; this call instead evaluates, from scratch for the given
 * points,
 *     u_l(x_i, t_n) = sum_{j: 0 < r_ij < delta} sum_l eta_l(r_ij) sigma_j(t_{n-nmax+1+l})
 * with the same quadrature weights eta_l as a plan's local part (delta = W dt).
 *   M, src_xy      sources, 2*M doubles (x, y), device memory; M <= 65536.
 *   Mt, tgt_xy     targets, 2*Mt doubles, device memory; Mt <= 32768 (may alias src_xy).  A target
 *                  whose distance to a source is at most 1e-12 times the side of the points'
 *                  bounding square coincides with it and that pair is left out; a target that
 *                  coincides with two or more sources returns WFP_EUNSUPPORTED, as
 *                  wfp_plan_create does.
 *   sigma_win      device, [nmax][M] doubles, level-major, oldest level first: row l holds
 *                  sigma_j(t_{n-nmax+1+l}) (zero for levels <= 0).
 *   nmax           W + 1 + p/2 for (dt, band_limit, tol) as wfp_select_params reports; must match.
 *   dt, band_limit, tol   as in wfp_plan_create (caller units).
 *   u_local        device, Mt doubles (output).
 *   stream         cudaStream_t or NULL.
 * Scratch: one file-scope device array of about 17 MiB, held by every GPU that loads the
 * library until exit, holds the pair list (at most 65536 pairs with 0 < r < delta), the weights
 * and the tables; more sources or targets than the limits above, or more pairs, return
 * WFP_EINVAL with a message.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  All calls share the array and it keeps the
 * last call's contents: calls whose work overlaps on the GPU (other streams, other threads) race
 * on it.  The call synchronises the stream once (to read the pair count back) and returns with
 * the last kernels enqueued on it.  No cudaMalloc, cudaFree or allocating library routine is
 * called.
 */
wfp_status wfp_local_noalloc(int64_t M, const double* src_xy, int64_t Mt, const double* tgt_xy,
                             const double* sigma_win, int nmax, double dt, double band_limit, double tol,
                             double* u_local, void* stream);

/* ------------------------------------------------------------------------------------------
 * Request server: many independent evaluations (each a full problem of Sec. 1 over its own
 * N_t steps) share one GPU by continuous batching.  The paper evaluates one problem at a time;
 * the server only schedules plans and adds no arithmetic of its own.
 *
 * Each request carries its geometry and its signal parameters; signals are generated on the
 * device each step, so a request needs no host traffic until its result is read.
 * wfp_server_tick():
 *   1. admits pending requests, in arrival order, whose estimated device footprint fits the
 *      free part of hbm_budget_bytes (a request that does not fit waits; later, smaller ones may
 *      pass it); a request is admitted with its S history stored (WFP_LAG_STORE) when that
 *      footprint fits, else with the lagged NUFFT (WFP_LAG_RECOMPUTE); at most max_active
 *      requests are admitted at once; a request larger than the whole budget fails.  An admitted
 *      request's plan is built on a worker thread (WFP_REQ_BUILDING) while the active requests
 *      keep stepping; it joins the active set on the first tick after its build completes;
 *   2. enqueues steps of every active request, each on its own stream, so that kernels of
 *      different requests overlap on the device; a request may have up to four steps in flight
 *      (step n is enqueued once step n - 4 has completed, asked without blocking), so each
 *      request advances at its own pace;
 *   3. retires requests whose last step has completed (copies the result to host memory and frees
 *      the request's device memory).
 * A request's outputs are bitwise the same whether it runs alone or among others.
 * Not thread-safe: one thread drives a server.
 * ------------------------------------------------------------------------------------------ */
typedef struct wfp_server_s* wfp_server;

/* Signal families generated on the device.
 * WFP_SIGNAL_GAUSS3: 8 doubles per source [a1 a2 a3 c1 c2 c3 s w],
 *   sigma_j(t) = sum_q a_q exp(-(t - c_q)^2 / (2 s^2)) sin(w (t - c_q)) for t > 0, 0 for t <= 0
 *   (Gaussian-modulated pulses).
 * WFP_SIGNAL_ERF: 2 doubles per source [t0 w],
 *   sigma_j(t) = 0.5 (erf(5 (t - t0)) + 1) sin(w (t - t0)) for t > 0, 0 for t <= 0
 *   (the switched sines of the paper's examples, Sec. 7, Eq. exampleDensities). */
enum { WFP_SIGNAL_GAUSS3 = 0, WFP_SIGNAL_ERF = 1 };

typedef struct {
    int64_t M;                    /* sources (>= 1) */
    const double* src_xy;         /* host, 2*M doubles; copied by wfp_server_submit */
    int64_t Mt;                   /* targets (>= 1) */
    const double* tgt_xy;         /* host, 2*Mt doubles, or NULL for targets = sources (then Mt = M) */
    double dt;                    /* as wfp_plan_create */
    int64_t Nt;
    double band_limit;
    double tol;
    int signal_family;            /* WFP_SIGNAL_GAUSS3 or WFP_SIGNAL_ERF */
    const double* signal_params;  /* host, 8*M (GAUSS3) or 2*M (ERF) doubles; copied */
    int n_out;                    /* number of output steps; 0 => the final step N_t only */
    const int64_t* out_steps;     /* host, n_out step indices in 1..N_t (any order; kept sorted) */
} wfp_request;

enum { WFP_REQ_PENDING = 0, WFP_REQ_ACTIVE = 1, WFP_REQ_DONE = 2, WFP_REQ_FAILED = 3, WFP_REQ_BUILDING = 4 };

typedef struct {
    int state;                    /* WFP_REQ_* */
    int64_t steps_done, Nt, Mt;
    int n_out;                    /* outputs kept: the result holds n_out * Mt doubles */
    double t_submit, t_admit, t_done;  /* host steady-clock seconds (same clock for all requests) */
    int64_t device_bytes;         /* footprint used for admission (estimate) */
    int64_t plan_bytes;           /* device memory the plan actually held (0 before admission) */
    double t_active;              /* when its plan was built and it started stepping (0 before) */
} wfp_request_status;

/* Create a server.  opts (NULL for defaults) apply to every request, except lag_mode and stream,
 * which the server chooses.  Errors: WFP_EINVAL, WFP_ENOMEM. */
wfp_status wfp_server_create(int64_t hbm_budget_bytes, int max_active, const wfp_opts* opts, wfp_server* out);

/* Queue a request; *id receives its id (> 0).  Copies everything it needs from *req.
 * Errors: WFP_EINVAL (bad sizes, output step outside 1..Nt), WFP_EUNSUPPORTED (signal family). */
wfp_status wfp_server_submit(wfp_server server, const wfp_request* req, int64_t* id);

/* One round of admission, stepping and retirement (see above).  *n_active and *n_pending
 * (either may be NULL) receive the counts after the round.  A request whose plan cannot be
 * built or whose step fails is marked WFP_REQ_FAILED; the server carries on. */
wfp_status wfp_server_tick(wfp_server server, int* n_active, int* n_pending);

/* Tick until no request is pending or active.  WFP_ENOMEM if pending requests remain that can
 * not be admitted with nothing active. */
wfp_status wfp_server_run(wfp_server server);

/* State and timestamps of a request. */
wfp_status wfp_server_query(wfp_server server, int64_t id, wfp_request_status* status);

/* Copy a finished request's outputs, n_out * Mt doubles (row r = step out_steps[r] in ascending
 * order), into host memory u_out.  WFP_ESTATE if the request is not done or failed. */
wfp_status wfp_server_result(wfp_server server, int64_t id, double* u_out);

/* Free every plan and buffer of the server (active requests are abandoned).  NULL is accepted. */
wfp_status wfp_server_destroy(wfp_server server);

/* Human-readable name of a status code, and the thread-local message of the last failure. */
const char* wfp_status_string(wfp_status s);
const char* wfp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* WFP_H */
