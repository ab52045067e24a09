// Request server of the 2D TK-WFP evaluator: continuous batching of independent evaluations.
//
// Each request is a complete evaluation problem (sources, targets, dt, N_t, band limit, tolerance)
// whose signals come from a device-side generator, so no per-step host traffic is needed.
// wfp_server_tick() (1) admits pending requests whose estimated device footprint fits the free part
// of the server's HBM budget (first fit in arrival order), building each one's plan on its own
// stream; (2) enqueues one step of every active request, each on its own stream, so that the
// kernels of small requests overlap on the device; (3) retires the
// requests that reached N_t, returning their memory to the budget.  The host never waits on a
// request: each may run up to four steps ahead of the device (an event per step, queried without
// blocking), so each request advances at its own pace.  Each request's Fourier
// history stays resident on the device between ticks.  Plans are independent and their kernels
// deterministic, so a request's result does not depend on what else is being served.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "wfp.h"
#include "wfp_plan.h"

using namespace wfp;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// sigma_j(t) = sum_{q<3} a_q exp(-(t - c_q)^2 / (2 s^2)) sin(w (t - c_q)), zero for t <= 0;
// params per source [a1 a2 a3 c1 c2 c3 s w]
__global__ void k_gen_gauss3(int64_t M, const double* __restrict__ par, double t, double* __restrict__ out) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const double* p = par + 8 * j;
    double v = 0.0;
    if (t > 0.0) {
        double s = p[6], w = p[7];
        for (int q = 0; q < 3; q++) {
            double z = t - p[3 + q];
            v += p[q] * exp(-z * z / (2.0 * s * s)) * sin(w * z);
        }
    }
    out[j] = v;
}

// sigma_j(t) = 0.5 (erf(5 (t - t0)) + 1) sin(w (t - t0)) for t > 0, zero for t <= 0 (the switched
// sines of the paper's examples, Sec. 7); params per source [t0 w]
__global__ void k_gen_erf(int64_t M, const double* __restrict__ par, double t, double* __restrict__ out) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const double z = t - par[2 * j];
    out[j] = (t > 0.0) ? 0.5 * (erf(5.0 * z) + 1.0) * sin(par[2 * j + 1] * z) : 0.0;
}

static int params_per_source(int family) { return family == WFP_SIGNAL_ERF ? 2 : 8; }

struct Request {
    int64_t id = 0;
    std::vector<double> src, tgt, par;
    std::vector<int64_t> out_steps;
    int64_t M = 0, Mt = 0, Nt = 0;
    double dt = 0, K0 = 0, tol = 0;
    int family = 0;
    int state = WFP_REQ_PENDING;
    wfp_plan plan = nullptr;
    double* d_par = nullptr;
    double* d_out = nullptr;
    std::vector<double> result;
    int64_t steps_done = 0;
    int64_t bytes = 0, plan_bytes = 0;
    double t_submit = 0, t_admit = 0, t_active = 0, t_done = 0;
    std::string err;
    // admission footprint (stored S history / lagged NUFFT), computed once: counting the local pairs
    // exactly costs O(M_t x neighbours) host time, too much to repeat on every tick while it waits
    int64_t est[2] = {0, 0};
    int est_state = 0;  // 0: not yet computed, 1: valid, -1: invalid request
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // completion of the last enqueued steps
    // plan building on a worker thread (the builder writes plan, buffers, build_status and err,
    // then sets build_done; the server thread reads them only after seeing build_done)
    std::thread builder;
    std::atomic<int> build_done{0};
    wfp_status build_status = WFP_OK;
};

// Device bytes a plan for this request would hold (the allocations of the plan builder, the
// cuFFT work areas counted as one more complex grid, the request's own buffers), with the S
// history stored (bytes[1]) and with the lagged NUFFT instead (bytes[0]).  False if the request's
// parameters are invalid.
bool estimate_bytes(const Request& r, const wfp_opts& o, int64_t bytes[2], std::string& err) {
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    auto acc = [&](const std::vector<double>& xy) {
        for (size_t i = 0; i + 1 < xy.size(); i += 2) {
            xmin = std::min(xmin, xy[i]);
            xmax = std::max(xmax, xy[i]);
            ymin = std::min(ymin, xy[i + 1]);
            ymax = std::max(ymax, xy[i + 1]);
        }
    };
    acc(r.src);
    acc(r.tgt);
    double half = 0.5 * std::max(xmax - xmin, ymax - ymin);
    double mag = std::max({std::fabs(xmin), std::fabs(xmax), std::fabs(ymin), std::fabs(ymax), 1e-300});
    half = (half > 1e-12 * mag) ? half * (1.0 + 1e-9) : 1.0;
    Params P;
    if (select_params(half, r.dt, r.Nt, r.K0, r.tol, o, P, err) != WFP_OK) return false;
    const double cx = 0.5 * (xmin + xmax), cy = 0.5 * (ymin + ymax), sc = 1.0 / half;
    // local pairs: exact count of 0 < r < delta on a cell grid
    int nc = std::max(1, std::min(2048, (int)std::floor(2.0 / P.delta)));
    double cs = 2.0 / nc;
    std::vector<int> head((size_t)nc * nc, -1), next(r.M);
    auto cell = [&](double x, double y, int& ix, int& iy) {
        ix = std::min(nc - 1, std::max(0, (int)std::floor(((x - cx) * sc + 1.0) / cs)));
        iy = std::min(nc - 1, std::max(0, (int)std::floor(((y - cy) * sc + 1.0) / cs)));
    };
    for (int64_t j = 0; j < r.M; j++) {
        int ix, iy;
        cell(r.src[2 * j], r.src[2 * j + 1], ix, iy);
        next[j] = head[(size_t)iy * nc + ix];
        head[(size_t)iy * nc + ix] = (int)j;
    }
    int64_t pairs = 0, near = 0;
    const double d2max = (P.delta / sc) * (P.delta / sc), d2near = (P.dt / sc) * (P.dt / sc);
    for (int64_t i = 0; i < r.Mt; i++) {
        double x = r.tgt[2 * i], y = r.tgt[2 * i + 1];
        int ix, iy;
        cell(x, y, ix, iy);
        for (int gy = std::max(0, iy - 1); gy <= std::min(nc - 1, iy + 1); gy++)
            for (int gx = std::max(0, ix - 1); gx <= std::min(nc - 1, ix + 1); gx++)
                for (int j = head[(size_t)gy * nc + gx]; j >= 0; j = next[j]) {
                    double dx = x - r.src[2 * (size_t)j], dy = y - r.src[2 * (size_t)j + 1];
                    double d2 = dx * dx + dy * dy;
                    if (d2 > 0 && d2 < d2max) pairs++;
                    if (d2 > 0 && d2 < d2near) near++;
                }
    }
    const double s = (P.precision == WFP_FP64) ? 8.0 : 4.0, c = 2 * s;
    const double R2 = (P.Km / P.dk) * (P.Km / P.dk), Rf2 = (P.Kf / P.dk) * (P.Kf / P.dk);
    const double modes = 0.5 * kPi * R2 + 2 * std::sqrt(R2) + 1, far = 0.5 * kPi * Rf2 + 2 * std::sqrt(Rf2) + 1;
    // distinct |k|^2 = dk^2 (n1^2 + n2^2) in the disk: the FIR taps are stored once per |k|
    const int64_t R = (int64_t)std::floor(P.Km / P.dk) + 1;
    std::vector<char> seen((size_t)(R * R + 1), 0);
    double n_kappa = 0;
    for (int64_t a = 0; a <= R; a++)
        for (int64_t q = 0; q <= a && a * a + q * q <= R * R; q++)
            if (!seen[(size_t)(a * a + q * q)]) seen[(size_t)(a * a + q * q)] = 1, n_kappa += 1;
    const int NW = P.nmax <= 32 ? 32 : 64;
    P.M = r.M;
    const bool fac = local_form_of(P, o) == WFP_LOCAL_FACTORED;
    const double nf = P.nf, nh2 = P.nf / 2 + 1, nc1 = P.Nh + 1, nb = P.nb;
    for (int store = 0; store < 2; store++) {
    const bool rec = P.lag_active && !store;
    double b = (double)(r.par.size() + std::max<size_t>(1, r.out_steps.size()) * r.Mt) * 8.0;  // request buffers
    if (fac)  // factored form: pair records, near rows, per-step contraction (at most 36 coefficients)
        b += (pairs - near) * (2 * s) + near * (NW * s + 4) + 2 * (r.Mt + 1) * 8.0 +
             (P.W - 1) * (double)r.M * 36 * s + (P.W - 1) * 32 * 36 * s;
    else
        b += pairs * (NW * s + 4) + (r.Mt + 1) * 8.0;                                  // local part
    const bool keep = store && P.lag_active;  // the S history is stored only while the lag is in use
    b += modes * (8 + 4 + 32 + (keep ? P.L + P.W : P.W) * c + (rec ? P.W * c : 0));   // modes, state, S
    b += n_kappa * (4 * P.W * s + 24);                                                  // taps per |k|
    b += nb * nf * s * (2 + rec) + nf * nh2 * c * (2 + rec) + 2 * nf * nc1 * c * (2 + rec); // grids
    b += nf * nh2 * c;                                                                 // cuFFT work areas
    if (P.far_active) b += far * (8 + P.n_lambda * 16.0 + P.n_lambda * 8.0);            // far history
    b += r.Mt * (8 + 250 * 8.0);                                                       // self term (bound)
    b += r.M * (NW * s + 4 + 2 * P.w * s + 4 + 8 + (rec ? P.L + 1 : 1) * s + 64);      // per source
    b += r.Mt * (2 * P.w * s + 4 + 4 * 8 + 4);                                         // per target
    bytes[store] = (int64_t)b;
    }
    return true;
}

}  // namespace

struct wfp_server_s {
    int64_t budget = 0, used = 0;
    int max_active = 0;
    wfp_opts opts;
    int64_t next_id = 1;
    int64_t n_admitted = 0;  // requests admitted so far
    std::deque<Request*> pending;
    std::vector<Request*> building;  // admitted, plan being built on a worker thread
    std::vector<Request*> active;
    int max_builders = 3;
    std::map<int64_t, std::unique_ptr<Request>> all;
    int device = 0;
};

static wfp_status sfail(wfp_status s, const std::string& m) {
    set_error(m);
    return s;
}

static void release(Request* r) {
    if (r->plan) wfp_destroy(r->plan);  // synchronises the plan's stream first
    for (auto& e : r->ev)
        if (e) cudaEventDestroy(e), e = nullptr;
    if (r->d_par) cudaFree(r->d_par);
    if (r->d_out) cudaFree(r->d_out);
    r->plan = nullptr;
    r->d_par = r->d_out = nullptr;
}

static void retire(wfp_server_s* sv, Request* r, int state) {
    release(r);
    sv->used -= r->bytes;
    r->state = state;
    r->t_done = now_s();
}

// build the plan and device buffers of an admitted request
static wfp_status admit_with(wfp_opts o, Request* r, bool store, std::string& err) {
    o.lag_mode = store ? WFP_LAG_STORE : WFP_LAG_RECOMPUTE;
    o.stream = nullptr;  // every request gets its own stream
    wfp_status st = wfp_plan_create(r->M, r->src.data(), r->Mt, r->tgt.data(), r->dt, r->Nt, r->K0, r->tol, &o,
                                    &r->plan);
    if (st != WFP_OK) {
        err = wfp_last_error();
        return st;
    }
    size_t nout = std::max<size_t>(1, r->out_steps.size());
    if (cudaMalloc(&r->d_par, r->par.size() * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&r->d_out, nout * r->Mt * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        err = "request buffers: out of device memory";
        return WFP_ENOMEM;
    }
    for (auto& e : r->ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            err = "cudaEventCreate failed";
            return WFP_ECUDA;
        }
    if (cudaMemcpy(r->d_par, r->par.data(), r->par.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        err = "request parameters: copy failed";
        return WFP_ECUDA;
    }
    return WFP_OK;
}

// worker thread: build the request's plan and buffers (per-thread default stream, so the steps
// of the active requests keep running)
static void build_worker(int device, const wfp_opts* opts, Request* r, bool store) {
    cudaSetDevice(device);
    std::string err;
    wfp_opts o = *opts;
    r->build_status = admit_with(o, r, store, err);
    if (r->build_status != WFP_OK) r->err = err;
    cudaStreamSynchronize(cudaStreamPerThread);
    r->build_done.store(1, std::memory_order_release);
}

extern "C" {

wfp_status wfp_server_create(int64_t hbm_budget_bytes, int max_active, const wfp_opts* opts, wfp_server* out) {
    if (!out) return sfail(WFP_EINVAL, "out is NULL");
    *out = nullptr;
    if (hbm_budget_bytes <= 0 || max_active < 1) return sfail(WFP_EINVAL, "need a positive budget and max_active");
    auto* sv = new (std::nothrow) wfp_server_s();
    if (!sv) return sfail(WFP_ENOMEM, "host allocation failed");
    sv->budget = hbm_budget_bytes;
    sv->max_active = max_active;
    if (opts)
        sv->opts = *opts;
    else
        wfp_opts_default(&sv->opts);
    cudaGetDevice(&sv->device);
    *out = sv;
    return WFP_OK;
}

wfp_status wfp_server_submit(wfp_server sv, const wfp_request* q, int64_t* id) {
    if (!sv || !q || !id) return sfail(WFP_EINVAL, "NULL argument");
    if (q->M < 1 || q->Mt < 1 || !q->src_xy || !q->signal_params || q->Nt < 1 || q->n_out < 0 ||
        (q->n_out > 0 && !q->out_steps))
        return sfail(WFP_EINVAL, "bad request");
    if (q->signal_family != WFP_SIGNAL_GAUSS3 && q->signal_family != WFP_SIGNAL_ERF)
        return sfail(WFP_EUNSUPPORTED, "unknown signal family");
    auto r = std::make_unique<Request>();
    r->id = sv->next_id++;
    r->M = q->M;
    r->Mt = q->Mt;
    r->src.assign(q->src_xy, q->src_xy + 2 * q->M);
    const double* t = q->tgt_xy ? q->tgt_xy : q->src_xy;
    r->tgt.assign(t, t + 2 * q->Mt);
    r->par.assign(q->signal_params, q->signal_params + params_per_source(q->signal_family) * q->M);
    r->dt = q->dt;
    r->Nt = q->Nt;
    r->K0 = q->band_limit;
    r->tol = q->tol;
    r->family = q->signal_family;
    if (q->n_out > 0)
        r->out_steps.assign(q->out_steps, q->out_steps + q->n_out);
    else
        r->out_steps.push_back(q->Nt);  // default: the field at the final step
    for (int64_t s : r->out_steps)
        if (s < 1 || s > q->Nt) return sfail(WFP_EINVAL, "output step outside 1..Nt");
    std::sort(r->out_steps.begin(), r->out_steps.end());
    r->t_submit = now_s();
    *id = r->id;
    sv->pending.push_back(r.get());
    sv->all[r->id] = std::move(r);
    return WFP_OK;
}

wfp_status wfp_server_tick(wfp_server sv, int* n_active, int* n_pending) {
    if (!sv) return sfail(WFP_EINVAL, "server is NULL");
    cudaSetDevice(sv->device);
    auto fail_pending = [](Request* r, const std::string& why) {
        r->err = why;
        r->state = WFP_REQ_FAILED;
        r->t_done = now_s();
    };
    // (1) admission: arrival order, first fit within the HBM budget and the slot limit; the plan is
    // built on a worker thread while the active requests keep stepping
    for (auto it = sv->pending.begin(); it != sv->pending.end() &&
                                        (int)(sv->active.size() + sv->building.size()) < sv->max_active &&
                                        (int)sv->building.size() < sv->max_builders;) {
        Request* r = *it;
        if (r->est_state == 0) {
            std::string err;
            r->est_state = estimate_bytes(*r, sv->opts, r->est, err) ? 1 : -1;
            if (r->est_state < 0) r->err = err;
        }
        if (r->est_state < 0) {
            fail_pending(r, r->err);
            it = sv->pending.erase(it);
            continue;
        }
        const int64_t* est = r->est;
        const int64_t free_b = sv->budget - sv->used;
        const bool store = est[1] <= free_b;
        const int64_t need = store ? est[1] : est[0];
        if (need > sv->budget) {  // can never fit
            fail_pending(r, "request needs " + std::to_string(need) + " device bytes, more than the server's budget");
            it = sv->pending.erase(it);
            continue;
        }
        if (need > free_b) {
            ++it;
            continue;
        }
        r->bytes = need;  // reserved until the request retires or its build fails
        sv->used += need;
        sv->n_admitted++;
        r->state = WFP_REQ_BUILDING;
        r->t_admit = now_s();
        r->builder = std::thread(build_worker, sv->device, &sv->opts, r, store);
        sv->building.push_back(r);
        it = sv->pending.erase(it);
    }
    // finished builds become active (or fail and give their reservation back)
    for (size_t i = 0; i < sv->building.size();) {
        Request* r = sv->building[i];
        if (!r->build_done.load(std::memory_order_acquire)) {
            i++;
            continue;
        }
        r->builder.join();
        sv->building.erase(sv->building.begin() + i);
        if (r->build_status != WFP_OK) {
            release(r);
            sv->used -= r->bytes;
            r->state = WFP_REQ_FAILED;
            r->t_done = now_s();
            continue;
        }
        wfp_info info;
        wfp_plan_get_info(r->plan, &info);
        r->plan_bytes = info.device_bytes;
        r->state = WFP_REQ_ACTIVE;
        r->t_active = now_s();
        sv->active.push_back(r);
    }
    // (2) enqueue steps of every active request on its own stream without waiting: a request may
    // have up to kInFlight steps in flight (step n is enqueued once step n - kInFlight has completed,
    // which is asked with a non-blocking query), so small requests are not held to the pace of the
    // large ones sharing the device
    constexpr int kInFlight = 4;
    for (Request* r : sv->active) {
        Plan& pl = plan_of(r->plan);
        for (int k = 0; k < kInFlight && r->steps_done < r->Nt; k++) {
            const int64_t n = r->steps_done + 1;
            cudaEvent_t ev = r->ev[n % kInFlight];
            std::string err;
            if (n > kInFlight) {
                const cudaError_t q = cudaEventQuery(ev);
                if (q == cudaErrorNotReady) break;
                if (q != cudaSuccess) {
                    r->err = "a step of this request failed on the device";
                    r->state = WFP_REQ_FAILED;
                    break;
                }
            }
            if (r->family == WFP_SIGNAL_ERF)
                k_gen_erf<<<(unsigned)((r->M + 255) / 256), 256, 0, pl.stream>>>(r->M, r->d_par, n * r->dt,
                                                                                  pl.d_sig_in);
            else
                k_gen_gauss3<<<(unsigned)((r->M + 255) / 256), 256, 0, pl.stream>>>(r->M, r->d_par, n * r->dt,
                                                                                     pl.d_sig_in);
            double* dst = nullptr;
            auto pos = std::lower_bound(r->out_steps.begin(), r->out_steps.end(), n);
            if (pos != r->out_steps.end() && *pos == n) dst = r->d_out + (pos - r->out_steps.begin()) * r->Mt;
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess || plan_step_device(pl, dst, err) != WFP_OK ||
                cudaEventRecord(ev, pl.stream) != cudaSuccess) {
                r->err = err.empty() ? std::string("step launch failed: ") + cudaGetErrorString(e) : err;
                r->state = WFP_REQ_FAILED;
                break;
            }
            r->steps_done = n;
        }
    }
    // (3) retire failed requests and those that took their last step
    for (size_t i = 0; i < sv->active.size();) {
        Request* r = sv->active[i];
        if (r->state == WFP_REQ_FAILED) {
            retire(sv, r, WFP_REQ_FAILED);
            sv->active.erase(sv->active.begin() + i);
            continue;
        }
        if (r->steps_done >= r->Nt) {
            // retire once the last step has completed (non-blocking check)
            const cudaError_t q = cudaEventQuery(r->ev[r->Nt % 4]);
            if (q == cudaErrorNotReady) {
                i++;
                continue;
            }
            int state = WFP_REQ_DONE;
            r->result.resize(r->out_steps.size() * r->Mt);
            if (cudaStreamSynchronize(plan_of(r->plan).stream) != cudaSuccess ||
                cudaMemcpy(r->result.data(), r->d_out, r->result.size() * sizeof(double), cudaMemcpyDeviceToHost) !=
                    cudaSuccess) {
                r->err = "a step of this request failed on the device";
                r->result.clear();
                state = WFP_REQ_FAILED;
            }
            retire(sv, r, state);
            sv->active.erase(sv->active.begin() + i);
            continue;
        }
        i++;
    }
    if (n_active) *n_active = (int)(sv->active.size() + sv->building.size());
    if (n_pending) *n_pending = (int)sv->pending.size();
    return WFP_OK;
}

wfp_status wfp_server_run(wfp_server sv) {
    if (!sv) return sfail(WFP_EINVAL, "server is NULL");
    int a = 1, p = 1;
    while (a > 0 || p > 0) {
        const int64_t before = sv->n_admitted;
        const bool idle = sv->active.empty() && sv->building.empty();
        wfp_status st = wfp_server_tick(sv, &a, &p);
        if (st != WFP_OK) return st;
        // a round that began with nothing admitted admitted nothing: the pending requests never fit
        if (idle && a == 0 && p > 0 && sv->n_admitted == before)
            return sfail(WFP_ENOMEM, "pending requests cannot be admitted");
        if (sv->active.empty() && !sv->building.empty()) std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    return WFP_OK;
}

wfp_status wfp_server_query(wfp_server sv, int64_t id, wfp_request_status* st) {
    if (!sv || !st) return sfail(WFP_EINVAL, "NULL argument");
    auto it = sv->all.find(id);
    if (it == sv->all.end()) return sfail(WFP_EINVAL, "unknown request id");
    const Request& r = *it->second;
    st->state = r.state;
    st->steps_done = r.steps_done;
    st->Nt = r.Nt;
    st->Mt = r.Mt;
    st->n_out = (int)r.out_steps.size();
    st->t_submit = r.t_submit;
    st->t_admit = r.t_admit;
    st->t_done = r.t_done;
    st->t_active = r.t_active;
    st->device_bytes = r.bytes;
    st->plan_bytes = r.plan_bytes;
    return WFP_OK;
}

wfp_status wfp_server_result(wfp_server sv, int64_t id, double* u_out) {
    if (!sv || !u_out) return sfail(WFP_EINVAL, "NULL argument");
    auto it = sv->all.find(id);
    if (it == sv->all.end()) return sfail(WFP_EINVAL, "unknown request id");
    const Request& r = *it->second;
    if (r.state == WFP_REQ_FAILED) return sfail(WFP_ESTATE, "request failed: " + r.err);
    if (r.state != WFP_REQ_DONE) return sfail(WFP_ESTATE, "request not finished");
    std::memcpy(u_out, r.result.data(), r.result.size() * sizeof(double));
    return WFP_OK;
}

wfp_status wfp_server_destroy(wfp_server sv) {
    if (!sv) return WFP_OK;
    for (Request* r : sv->building) {  // let running builds finish, then drop them
        r->builder.join();
        r->err = "abandoned: server destroyed";
        retire(sv, r, WFP_REQ_FAILED);
    }
    for (Request* r : sv->active) {
        r->err = "abandoned: server destroyed";
        retire(sv, r, WFP_REQ_FAILED);
    }
    delete sv;
    return WFP_OK;
}

}  // extern "C"
