// C ABI of the 2D TK-WFP evaluator: plan creation, stepping, diagnostics.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <string>

#include "wfp.h"
#include "wfp_debug.h"
#include "wfp_plan.h"
#include "wfp_quad.h"

struct wfp_plan_s {
    wfp::Plan pl;
};

namespace wfp {
const char* last_error_cstr();
}

using namespace wfp;

static wfp_status fail(wfp_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

extern "C" {

void wfp_opts_default(wfp_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = WFP_FP64;
    o->exclude_self = 1;
    o->use_graph = 1;
}

const char* wfp_status_string(wfp_status s) {
    switch (s) {
        case WFP_OK: return "WFP_OK";
        case WFP_EINVAL: return "WFP_EINVAL";
        case WFP_ENOMEM: return "WFP_ENOMEM";
        case WFP_ECUDA: return "WFP_ECUDA";
        case WFP_ESTATE: return "WFP_ESTATE";
        case WFP_ETIMEOUT: return "WFP_ETIMEOUT";
        case WFP_EUNSUPPORTED: return "WFP_EUNSUPPORTED";
    }
    return "WFP_UNKNOWN";
}

const char* wfp_last_error(void) { return last_error_cstr(); }

wfp_status wfp_select_params(double halfside, double dt, int64_t Nt, double band_limit, double tol,
                             const wfp_opts* opts, wfp_info* info) {
    if (!info) return fail(WFP_EINVAL, "info is NULL");
    wfp_opts o;
    if (opts)
        o = *opts;
    else
        wfp_opts_default(&o);
    Params P;
    std::string err;
    wfp_status st = select_params(halfside, dt, Nt, band_limit, tol, o, P, err);
    if (st != WFP_OK) return fail(st, err);
    fill_info(P, *info);
    return WFP_OK;
}

wfp_status wfp_plan_create(int64_t M, const double* src_xy, int64_t Mt, const double* tgt_xy, double dt, int64_t Nt,
                           double band_limit, double tol, const wfp_opts* opts, wfp_plan* out) {
    if (!out) return fail(WFP_EINVAL, "out is NULL");
    *out = nullptr;
    if (M < 1 || Mt < 1 || !src_xy || !tgt_xy) return fail(WFP_EINVAL, "need M >= 1, Mt >= 1 and coordinates");
    if (M >= (1ll << 31) || Mt >= (1ll << 31)) return fail(WFP_EINVAL, "M and Mt must be below 2^31");
    for (int64_t i = 0; i < 2 * M; i++)
        if (!std::isfinite(src_xy[i])) return fail(WFP_EINVAL, "non-finite source coordinate");
    for (int64_t i = 0; i < 2 * Mt; i++)
        if (!std::isfinite(tgt_xy[i])) return fail(WFP_EINVAL, "non-finite target coordinate");
    wfp_plan_s* h = new (std::nothrow) wfp_plan_s();
    if (!h) return fail(WFP_ENOMEM, "host allocation failed");
    Plan& pl = h->pl;
    if (opts)
        pl.opts = *opts;
    else
        wfp_opts_default(&pl.opts);
    pl.P.M = M;
    pl.P.Mt = Mt;
    pl.P.Nt = Nt;
    pl.P.dt_user = dt;
    pl.P.K0_user = band_limit;
    pl.P.tol = tol;
    pl.P.precision = pl.opts.precision;
    pl.P.exclude_self = pl.opts.exclude_self != 0;
    pl.use_graph = pl.opts.use_graph != 0;
    {  // fingerprint of the inputs and of the options that change results (checkpoints carry it)
        uint64_t hsh = 1469598103934665603ull;  // FNV-1a, 64 bit
        auto mix = [&hsh](const void* p, size_t n) {
            const unsigned char* c = (const unsigned char*)p;
            for (size_t i = 0; i < n; i++) hsh = (hsh ^ c[i]) * 1099511628211ull;
        };
        mix(src_xy, sizeof(double) * 2 * M);
        mix(tgt_xy, sizeof(double) * 2 * Mt);
        const wfp_opts& o = pl.opts;
        const double dv[6] = {dt, band_limit, tol, o.eps, o.Kf, o.delta};
        const double dv2[1] = {o.upsampfac};
        const int iv[10] = {o.precision, o.W, o.p, o.kernel_width, o.soe_nodes, o.exclude_self,
                            o.lag_mode, o.local_interp, o.local_form, 0};
        mix(dv, sizeof(dv));
        mix(dv2, sizeof(dv2));
        mix(iv, sizeof(iv));
        mix(&Nt, sizeof(Nt));
        pl.inputs_hash = hsh;
    }
    std::string err;
    // validate the scalar arguments before touching the GPU
    {
        Params tmp;
        wfp_status st = select_params(1.0, dt, Nt, band_limit, tol, pl.opts, tmp, err);
        if (st != WFP_OK) {
            delete h;
            return fail(st, err);
        }
    }
    cudaGetDevice(&pl.device);
    if (pl.opts.stream) {
        pl.stream = (cudaStream_t)pl.opts.stream;
    } else {
        if (cudaStreamCreateWithFlags(&pl.stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return fail(WFP_ECUDA, "cudaStreamCreate failed");
        }
        pl.own_stream = true;
    }
    wfp_status st = plan_build(pl, src_xy, tgt_xy, err);
    if (st != WFP_OK) {
        plan_free(pl);
        delete h;
        cudaGetLastError();
        return fail(st, err);
    }
    *out = h;
    return WFP_OK;
}

}  // extern "C"

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// page-locked host memory (cudaHostAlloc / cudaMallocHost / cudaHostRegister): copied by the GPU's
// DMA engines directly, with no staging copy on the host
static bool is_pinned_host(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

static wfp_status poison(Plan& pl, const std::string& msg) {
    pl.poisoned = true;
    return fail(WFP_ECUDA, msg);
}

// a kernel whose bounded wait ran out has set the host-mapped flag: the step's output is not valid
static bool device_timed_out(const Plan& pl) { return pl.h_err && *(volatile int*)pl.h_err != 0; }

static wfp_status poison_timeout(Plan& pl) {
    pl.poisoned = true;
    return fail(WFP_ETIMEOUT, "a bounded device-side wait ran out (bulk copy not completed)");
}

// Run one phase of a step on the plan's stream: directly, or replayed from a CUDA graph that is
// captured on the phase's second use (the first use initialises cuFFT outside any capture).
template <typename F>
static wfp_status run_phase(Plan& pl, int which, F body, std::string& err) {
    int& uses = pl.graph_uses[which];
    cudaGraphExec_t& ge = pl.graph_exec[which];
    if (!pl.use_graph || pl.prof || uses < 1) {
        uses++;
        return body();
    }
    if (!ge) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(pl.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            pl.use_graph = false;  // e.g. the legacy default stream cannot be captured
            return body();
        }
        wfp_status st = body();
        cudaError_t e = cudaStreamEndCapture(pl.stream, &g);
        if (st != WFP_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            err = std::string("graph capture failed: ") + cudaGetErrorString(e);
            return WFP_ECUDA;
        }
        cudaGraphDestroy(g);
    }
    if (cudaGraphLaunch(ge, pl.stream) != cudaSuccess) {
        err = "cudaGraphLaunch failed";
        return WFP_ECUDA;
    }
    return WFP_OK;
}

// The step's output to the caller's device buffer or the pinned host stage, on the plan's stream.
static wfp_status copy_output(Plan& pl, cudaEvent_t after_output, double* u_dev_dst, double* u_host_stage,
                              std::string& err) {
    cudaError_t e = cudaSuccess;
    {
        ProfScope ps(pl, PP_COPY);
        if (u_dev_dst)
            e = cudaMemcpyAsync(u_dev_dst, pl.d_u_out, pl.Mt * sizeof(double), cudaMemcpyDeviceToDevice, pl.stream);
        else if (u_host_stage)
            e = cudaMemcpyAsync(u_host_stage, pl.d_u_out, pl.Mt * sizeof(double), cudaMemcpyDeviceToHost,
                                pl.stream);
    }
    if (e != cudaSuccess) {
        err = std::string("output copy: ") + cudaGetErrorString(e);
        return WFP_ECUDA;
    }
    if (after_output && cudaEventRecord(after_output, pl.stream) != cudaSuccess) {
        err = "cudaEventRecord failed";
        return WFP_ECUDA;
    }
    return WFP_OK;
}

// Enqueue the device work of one step on the plan's stream.
static wfp_status enqueue_step(Plan& pl, bool do_advance, bool lag_now, cudaEvent_t after_output,
                               double* u_dev_dst, double* u_host_stage, std::string& err) {
    const int which = do_advance ? (lag_now ? 2 : 1) : 3;
    if (!pl.prof && !pl.serial_step) {  // the whole step as one (graph-captured) fork/join of two streams
        wfp_status st = run_phase(pl, which, [&]() { return step_concurrent(pl, do_advance, lag_now, err); }, err);
        if (st != WFP_OK) return st;
        return copy_output(pl, after_output, u_dev_dst, u_host_stage, err);
    }
    if (!pl.prof) {  // the whole step (graph-captured) with its branches in sequence on the plan's stream
        wfp_status st = run_phase(pl, which, [&]() {
            wfp_status s2 = step_output(pl, err);
            if (s2 == WFP_OK && do_advance) s2 = step_advance_body(pl, lag_now, err);
            return s2 == WFP_OK ? step_tick(pl, err) : s2;
        }, err);
        if (st != WFP_OK) return st;
        return copy_output(pl, after_output, u_dev_dst, u_host_stage, err);
    }
    // profiling: every part in sequence on the plan's stream, each bracketed by events
    wfp_status st = step_output(pl, err);
    if (st != WFP_OK) return st;
    st = copy_output(pl, after_output, u_dev_dst, u_host_stage, err);
    if (st != WFP_OK) return st;
    if (do_advance) {
        st = step_advance_body(pl, lag_now, err);
        if (st != WFP_OK) return st;
    }
    return step_tick(pl, err);
}

namespace wfp {
// One step whose input sigma_n is already in pl.d_sig_in (caller order), enqueued on pl.stream; the
// output is copied to u_dev (device) when non-NULL.  Used by the server's device-side signal source.
wfp_status plan_step_device(Plan& pl, double* u_dev, std::string& err) {
    if (pl.poisoned) {
        err = "plan is poisoned";
        return WFP_ESTATE;
    }
    if (pl.step >= pl.P.Nt) {
        err = "all Nt steps have been taken";
        return WFP_ESTATE;
    }
    if (device_timed_out(pl)) {
        pl.poisoned = true;
        err = "a bounded device-side wait ran out (bulk copy not completed)";
        return WFP_ETIMEOUT;
    }
    const int64_t n = pl.step + 1;
    bool adv = n < pl.P.Nt;
    bool lag_now = pl.P.lag_active && (n - pl.P.L >= 1);
    wfp_status st = enqueue_step(pl, adv, lag_now, nullptr, u_dev, nullptr, err);
    if (st != WFP_OK) {
        pl.poisoned = true;
        return st;
    }
    pl.step = n;
    return WFP_OK;
}
Plan& plan_of(wfp_plan h) { return h->pl; }
}  // namespace wfp

extern "C" {

wfp_status wfp_step(wfp_plan plan, const double* sigma_n, double* u_n) {
    if (!plan) return fail(WFP_EINVAL, "plan is NULL");
    Plan& pl = plan->pl;
    if (pl.poisoned) return fail(WFP_ESTATE, "plan is poisoned by an earlier CUDA error");
    if (!sigma_n || !u_n) return fail(WFP_EINVAL, "sigma_n and u_n must not be NULL");
    if (pl.step >= pl.P.Nt) return fail(WFP_ESTATE, "all Nt steps have been taken");
    if (device_timed_out(pl)) return poison_timeout(pl);
    const int64_t n = pl.step + 1;
    const bool dev_in = is_device_ptr(sigma_n), dev_out = is_device_ptr(u_n);
    // with a host output the call returns after the whole step, so a pinned input is copied from the
    // caller's buffer directly; with a device output it returns early and the input goes through the
    // plan's own stage, which the caller cannot overwrite
    const bool pin_in = !dev_in && !dev_out && is_pinned_host(sigma_n);
    const bool pin_out = !dev_out && is_pinned_host(u_n);
    cudaError_t e;
    if (dev_in) {
        e = cudaMemcpyAsync(pl.d_sig_in, sigma_n, pl.M * sizeof(double), cudaMemcpyDeviceToDevice, pl.stream);
    } else if (pin_in) {
        e = cudaMemcpyAsync(pl.d_sig_in, sigma_n, pl.M * sizeof(double), cudaMemcpyHostToDevice, pl.stream);
    } else {
        // the pinned staging buffer may still feed the previous step's copy
        cudaStreamSynchronize(pl.stream);
        std::memcpy(pl.h_sig, sigma_n, pl.M * sizeof(double));
        e = cudaMemcpyAsync(pl.d_sig_in, pl.h_sig, pl.M * sizeof(double), cudaMemcpyHostToDevice, pl.stream);
    }
    if (e != cudaSuccess) return poison(pl, std::string("input copy: ") + cudaGetErrorString(e));
    if (pl.prof && pl.prof_ev.size() > 4096) prof_collect(pl);
    std::string err;
    bool adv = n < pl.P.Nt;
    bool lag_now = pl.P.lag_active && (n - pl.P.L >= 1);
    wfp_status st = enqueue_step(pl, adv, lag_now, dev_out ? nullptr : pl.ev_out, dev_out ? u_n : nullptr,
                                 dev_out ? nullptr : (pin_out ? u_n : pl.h_u), err);
    if (st != WFP_OK) return poison(pl, err);
    if (!dev_out) {
        e = cudaEventSynchronize(pl.ev_out);
        if (e != cudaSuccess) return poison(pl, std::string("step: ") + cudaGetErrorString(e));
        if (device_timed_out(pl)) return poison_timeout(pl);
        if (!pin_out) std::memcpy(u_n, pl.h_u, pl.Mt * sizeof(double));
    }
    pl.step = n;
    return WFP_OK;
}

wfp_status wfp_destroy(wfp_plan plan) {
    if (!plan) return WFP_OK;
    cudaStreamSynchronize(plan->pl.stream);
    plan_free(plan->pl);
    delete plan;
    return WFP_OK;
}

wfp_status wfp_plan_get_info(wfp_plan plan, wfp_info* info) {
    if (!plan || !info) return fail(WFP_EINVAL, "NULL argument");
    Plan& pl = plan->pl;
    fill_info(pl.P, *info);
    info->n_modes = pl.n_modes;
    info->n_far_modes = pl.n_far;
    info->n_kappa = pl.n_kappa;
    info->n_self_soe = pl.n_soe_self;
    info->n_pairs = pl.n_pairs;
    info->n_self = pl.n_self;
    info->device_bytes = pl.mem.bytes;
    info->lag_store = pl.lag_store;
    info->s_levels = pl.R_cur;
    info->spread_tile = pl.spread_ts;
    info->spread_chunk = pl.spread_ch;
    info->local_variant = (pl.NW == 32 && !pl.local_factored) ? pl.local_variant : 0;
    info->local_form = pl.local_factored ? WFP_LOCAL_FACTORED : WFP_LOCAL_STORED;
    info->local_nc = pl.local_factored ? pl.NC : 0;
    info->n_near_pairs = pl.local_factored ? pl.n_near : 0;
    info->n_spread_tiles = pl.n_tiles;
    info->bytes_local = pl.bytes_local;
    info->bytes_grid = pl.bytes_grid;
    info->bytes_history = pl.bytes_history;
    info->bytes_fft_work = pl.bytes_fft_work;
    info->step_order = pl.serial_step ? WFP_ORDER_SERIAL : WFP_ORDER_CONCURRENT;
    return WFP_OK;
}

wfp_status wfp_step_components(wfp_plan plan, double* u_local, double* u_hist, double* u_self) {
    if (!plan) return fail(WFP_EINVAL, "plan is NULL");
    Plan& pl = plan->pl;
    if (pl.poisoned) return fail(WFP_ESTATE, "plan is poisoned");
    if (cudaStreamSynchronize(pl.stream) != cudaSuccess) return poison(pl, "synchronise failed");
    // internal target order -> caller order on the host
    std::vector<int> perm(pl.Mt);
    std::vector<double> buf(pl.Mt);
    if (cudaMemcpy(perm.data(), pl.d_tgt_perm, pl.Mt * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return poison(pl, "copy failed");
    double* srcs[3] = {pl.d_uloc, pl.d_uh, pl.d_uself};
    double* dsts[3] = {u_local, u_hist, u_self};
    for (int k = 0; k < 3; k++) {
        if (!dsts[k]) continue;
        // u_hist of the last completed step: the advance has already replaced d_uh with the next
        // step's value, so it is recovered from the output identity u = u_local + u_hist - u_self.
        if (k == 1) continue;
        if (cudaMemcpy(buf.data(), srcs[k], pl.Mt * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            return poison(pl, "copy failed");
        for (int64_t i = 0; i < pl.Mt; i++) dsts[k][perm[i]] = buf[i];
    }
    if (u_hist) {
        std::vector<double> ul(pl.Mt), us(pl.Mt), uo(pl.Mt);
        if (cudaMemcpy(ul.data(), pl.d_uloc, pl.Mt * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(us.data(), pl.d_uself, pl.Mt * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(uo.data(), pl.d_u_out, pl.Mt * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            return poison(pl, "copy failed");
        for (int64_t i = 0; i < pl.Mt; i++) u_hist[perm[i]] = uo[perm[i]] - ul[i] + us[i];
    }
    return WFP_OK;
}

wfp_status wfp_profile(wfp_plan plan, int enable) {
    if (!plan) return fail(WFP_EINVAL, "plan is NULL");
    Plan& pl = plan->pl;
    prof_collect(pl);
    if (enable && !pl.prof)
        for (int i = 0; i < PP_NPARTS; i++) {
            pl.prof_ms[i] = 0;
            pl.prof_n[i] = 0;
        }
    pl.prof = enable != 0;
    return WFP_OK;
}

wfp_status wfp_profile_read(wfp_plan plan, int max_parts, const char** names, double* total_ms, int64_t* launches,
                            int* n_parts) {
    if (!plan || !n_parts) return fail(WFP_EINVAL, "NULL argument");
    Plan& pl = plan->pl;
    prof_collect(pl);
    *n_parts = PP_NPARTS;
    for (int i = 0; i < PP_NPARTS && i < max_parts; i++) {
        if (names) names[i] = kPartNames[i];
        if (total_ms) total_ms[i] = pl.prof_ms[i];
        if (launches) launches[i] = pl.prof_n[i];
    }
    return WFP_OK;
}

// ------------------------------------------------------------------ host-only diagnostics
wfp_status wfp_debug_eta(double r, double dt, int W, int p, double eps, double band_limit, int ng, double* eta) {
    if (!eta || W < 2 || W > 59 || p < 2 || p > kMaxP || (p & 1) || ng < 2 || ng > 64)
        return fail(WFP_EINVAL, "bad argument");
    int nmax = W + 1 + p / 2;
    if (nmax > kMaxLevels) return fail(WFP_EINVAL, "W + 1 + p/2 too large");
    std::vector<double> phic, gx(ng), gw(ng), wl(p);
    build_phi_table(std::log(1.0 / eps), phic);
    gauss_legendre(ng, gx.data(), gw.data());
    lagrange_ref_weights(p, wl.data());
    std::vector<double> cls;
    double Omega = std::max(band_limit, 1e-3 / dt);
    if (band_limit >= 0) build_ls_cheb(nmax, dt, Omega, kLsIntervals * dt, cls);
    eta_weights(r, dt, W, p, nmax, phic.data(), gx.data(), gw.data(), ng, wl.data(),
                band_limit >= 0 ? cls.data() : nullptr, eta);
    return WFP_OK;
}

wfp_status wfp_debug_eta_table(double r, double dt, int W, int p, double eps, double band_limit, int ng, double* eta) {
    if (!eta || W < 2 || W > 59 || p < 2 || p > kMaxP || (p & 1) || ng < 2 || ng > 64)
        return fail(WFP_EINVAL, "bad argument");
    int nmax = W + 1 + p / 2;
    if (nmax > kMaxLevels) return fail(WFP_EINVAL, "W + 1 + p/2 too large");
    std::vector<double> phic, gx(ng), gw(ng), wl(p);
    build_phi_table(std::log(1.0 / eps), phic);
    gauss_legendre(ng, gx.data(), gw.data());
    lagrange_ref_weights(p, wl.data());
    std::vector<double> cls, tab;
    double Omega = std::max(band_limit, 1e-3 / dt);
    if (band_limit >= 0) build_ls_cheb(nmax, dt, Omega, kLsIntervals * dt, cls);
    const double* C = band_limit >= 0 ? cls.data() : nullptr;
    if (r >= dt && r < W * dt) {
        build_eta_table(dt, W, p, nmax, phic.data(), gx.data(), gw.data(), ng, wl.data(), C, tab);
        eta_from_table(r, dt, W, nmax, tab.data(), eta);
    } else {
        eta_weights(r, dt, W, p, nmax, phic.data(), gx.data(), gw.data(), ng, wl.data(), C, eta);
    }
    return WFP_OK;
}

wfp_status wfp_debug_factored_table(double dt, int W, int p, double eps, double band_limit, int ng, int precision,
                                    int* nc, double* tail, double* tab_out) {
    if (!nc || !tail || W < 2 || W > 59 || p < 2 || p > kMaxP || (p & 1) || ng < 2 || ng > 64 ||
        (precision != WFP_FP64 && precision != WFP_MIXED))
        return fail(WFP_EINVAL, "bad argument");
    int nmax = W + 1 + p / 2;
    if (nmax > kMaxLevels) return fail(WFP_EINVAL, "W + 1 + p/2 too large");
    std::vector<double> phic, gx(ng), gw(ng), wl(p);
    build_phi_table(std::log(1.0 / eps), phic);
    gauss_legendre(ng, gx.data(), gw.data());
    lagrange_ref_weights(p, wl.data());
    std::vector<double> cls, tab;
    double Omega = std::max(band_limit, 1e-3 / dt);
    if (band_limit >= 0) build_ls_cheb(nmax, dt, Omega, kLsIntervals * dt, cls);
    build_eta_table(dt, W, p, nmax, phic.data(), gx.data(), gw.data(), ng, wl.data(),
                    band_limit >= 0 ? cls.data() : nullptr, tab);
    *nc = factored_nc_supported(factored_nc_choice(tab, W, nmax, precision == WFP_FP64), precision == WFP_FP64);
    *tail = factored_tail(tab, W, nmax, std::min(*nc, kEtaChebDeg + 1));
    if (tab_out) std::copy(tab.begin(), tab.end(), tab_out);
    return WFP_OK;
}

wfp_status wfp_debug_taps(double kappa, double dt, int W, double eps, double lagshift, double* taps, double* rot) {
    if (!taps || !rot || W < 2 || W > 59) return fail(WFP_EINVAL, "bad argument");
    double b = std::log(1.0 / eps), delta = W * dt;
    const int ngt = 24;
    std::vector<double> gx(ngt), gw(ngt), sq(ngt), wq(ngt), f1((size_t)W * ngt), f2((size_t)W * ngt);
    gauss_legendre(ngt, gx.data(), gw.data());
    for (int q = 0; q < ngt; q++) {
        sq[q] = 0.5 * dt * (gx[q] + 1.0);
        wq[q] = 0.5 * dt * gw[q];
    }
    for (int m = 0; m < W; m++)
        for (int q = 0; q < ngt; q++) {
            f1[(size_t)m * ngt + q] = dphi_host(sq[q] + m * dt, delta, b);
            f2[(size_t)m * ngt + q] = d2phi_host(sq[q] + m * dt, delta, b);
        }
    mode_taps(kappa, dt, W, lagshift, ngt, sq.data(), wq.data(), f1.data(), f2.data(), TapsPlanar{taps, W}, rot);
    return WFP_OK;
}

wfp_status wfp_debug_phi(double t, double delta, double eps, double* phi, double* dphi, double* d2phi) {
    std::vector<double> phic;
    double b = std::log(1.0 / eps);
    build_phi_table(b, phic);
    if (phi) *phi = phi_host(phic.data(), t, delta);
    if (dphi) *dphi = dphi_host(t, delta, b);
    if (d2phi) *d2phi = d2phi_host(t, delta, b);
    return WFP_OK;
}

wfp_status wfp_debug_hankel(double kappa, double A, double Delta, double eps, double lam_max, int panels, int ng,
                            double* H) {
    if (!H || panels < 1 || panels > 64 || ng < 1 || ng > 64 || !(A > Delta) || !(Delta > 0))
        return fail(WFP_EINVAL, "bad argument");
    std::vector<double> lam, q, phic;
    soe_nodes(lam_max, panels, ng, lam, q);
    build_phi_table(std::log(1.0 / eps), phic);
    // same composite rule as the plan: 32 panels x 16 Gauss-Legendre nodes on [0, A]
    const int npan = 32, ngr = 16;
    double gx[ngr], gw[ngr];
    gauss_legendre(ngr, gx, gw);
    for (size_t l = 0; l < lam.size(); l++) {
        double acc = 0.0;
        for (int k = 0; k < npan; k++)
            for (int i = 0; i < ngr; i++) {
                double a = A * k / npan, b = A * (k + 1) / npan;
                double r = 0.5 * (b - a) * gx[i] + 0.5 * (b + a), wr = 0.5 * (b - a) * gw[i];
                double x = A - r;
                double ph = (x <= 0.0) ? 0.0 : (x >= Delta ? 1.0 : cheb_phi(phic.data(), 2.0 * x / Delta - 1.0));
                acc += wr * std::cyl_bessel_j(0.0, kappa * r) * std::cyl_bessel_i(0.0, lam[l] * r) *
                       std::exp(-lam[l] * A) * ph * r;
            }
        H[l] = q[l] * acc;
    }
    return WFP_OK;
}

wfp_status wfp_debug_soe(double lam_max, int panels, int ng, double* lam, double* q) {
    if (!lam || !q || panels < 1 || panels > 64 || ng < 1 || ng > 64) return fail(WFP_EINVAL, "bad argument");
    std::vector<double> l, w;
    soe_nodes(lam_max, panels, ng, l, w);
    std::memcpy(lam, l.data(), l.size() * sizeof(double));
    std::memcpy(q, w.data(), w.size() * sizeof(double));
    return WFP_OK;
}

wfp_status wfp_debug_self_soe(double dlo, double T, double eps, int cap, double* lam, double* q, int* n) {
    if (!lam || !q || !n || !(dlo > 0.0) || !(T > dlo) || !(eps > 0.0 && eps < 1.0) || cap < 1)
        return fail(WFP_EINVAL, "bad argument");
    std::vector<double> l, w;
    if (!self_soe(dlo, T, eps, l, w)) return fail(WFP_EINVAL, "no candidate sum meets the tolerance");
    *n = (int)l.size();
    if ((int)l.size() > cap) return fail(WFP_EINVAL, "more terms than cap");
    std::memcpy(lam, l.data(), l.size() * sizeof(double));
    std::memcpy(q, w.data(), w.size() * sizeof(double));
    return WFP_OK;
}

}  // extern "C"
