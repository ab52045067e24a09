// Checkpoint and resume of a plan's step-to-step state (host buffer, fixed layout).
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "wfp.h"
#include "wfp_plan.h"

namespace wfp {
namespace {

struct Section {
    void* dev;
    size_t bytes;
};

constexpr uint64_t kMagic = 0x3254504b43504657ull;  // "WFPCKPT2"

// Fingerprint of everything the state layout and meaning depend on
struct Header {
    uint64_t magic;
    uint64_t inputs;  // hash of the coordinates, time grid, band limit, tolerance and options
    int64_t step;
    int64_t M, Mt, Nt, n_modes, n_far, n_self, n_soe;
    int64_t R_cur, R_lag, n_hist, NW, lag_store, precision;
    int64_t W, L, p, nf, nb, w, n_lambda;
    double dt, scale, K0, eps;
    int64_t total;
};

std::vector<Section> sections(const Plan& pl) {
    const Params& P = pl.P;
    const size_t s = P.precision == WFP_FP64 ? 8 : 4;
    std::vector<Section> v;
    v.push_back({pl.d_sigwin, (size_t)pl.M * pl.NW * s});
    if (pl.d_siglin) v.push_back({pl.d_siglin, (size_t)pl.M * 32 * s});
    v.push_back({pl.d_sighist, (size_t)pl.n_hist * pl.M * s});
    v.push_back({pl.d_alpha, (size_t)pl.n_modes * 16});
    v.push_back({pl.d_alphad, (size_t)pl.n_modes * 16});
    v.push_back({pl.d_ring, (size_t)pl.R_cur * pl.n_modes * 2 * s});
    if (pl.d_ring_lag != pl.d_ring) v.push_back({pl.d_ring_lag, (size_t)pl.R_lag * pl.n_modes * 2 * s});
    if (pl.d_B) v.push_back({pl.d_B, (size_t)P.n_lambda * pl.n_far * 16});
    if (pl.d_Y) v.push_back({pl.d_Y, (size_t)pl.n_soe_self * pl.n_self * 8});
    v.push_back({pl.d_uh, (size_t)pl.Mt * 2 * 8});
    v.push_back({pl.d_step, 8});
    return v;
}

Header header(const Plan& pl) {
    const Params& P = pl.P;
    Header h;
    std::memset(&h, 0, sizeof(h));
    h.magic = kMagic;
    h.inputs = pl.inputs_hash;
    h.step = pl.step;
    h.M = pl.M;
    h.Mt = pl.Mt;
    h.Nt = P.Nt;
    h.n_modes = pl.n_modes;
    h.n_far = pl.n_far;
    h.n_self = pl.n_self;
    h.n_soe = pl.n_soe_self;
    h.R_cur = pl.R_cur;
    h.R_lag = pl.R_lag;
    h.n_hist = pl.n_hist;
    h.NW = pl.NW;
    h.lag_store = pl.lag_store;
    h.precision = P.precision;
    h.W = P.W;
    h.L = P.L;
    h.p = P.p;
    h.nf = P.nf;
    h.nb = P.nb;
    h.w = P.w;
    h.n_lambda = P.n_lambda;
    h.dt = P.dt;
    h.scale = P.scale;
    h.K0 = P.K0;
    h.eps = P.eps;
    int64_t tot = (int64_t)sizeof(Header);
    for (const Section& sec : sections(pl)) tot += (int64_t)sec.bytes;
    h.total = tot;
    return h;
}

bool same_layout(const Header& a, const Header& b) {
    Header x = a, y = b;
    x.step = y.step = 0;  // the step is state, everything else must match
    return std::memcmp(&x, &y, sizeof(Header)) == 0;
}

}  // namespace
}  // namespace wfp

using namespace wfp;

extern "C" {

wfp_status wfp_checkpoint_size(wfp_plan plan, int64_t* bytes) {
    if (!plan || !bytes) {
        set_error("NULL argument");
        return WFP_EINVAL;
    }
    *bytes = header(plan_of(plan)).total;
    return WFP_OK;
}

wfp_status wfp_checkpoint_save(wfp_plan plan, void* buf, int64_t bytes) {
    if (!plan || !buf) {
        set_error("NULL argument");
        return WFP_EINVAL;
    }
    Plan& pl = plan_of(plan);
    if (pl.poisoned) {
        set_error("plan is poisoned");
        return WFP_ESTATE;
    }
    const Header h = header(pl);
    if (bytes < h.total) {
        set_error("checkpoint buffer too small: need " + std::to_string(h.total) + " bytes");
        return WFP_EINVAL;
    }
    if (cudaStreamSynchronize(pl.stream) != cudaSuccess) {
        pl.poisoned = true;
        set_error("stream synchronise failed");
        return WFP_ECUDA;
    }
    unsigned char* out = (unsigned char*)buf;
    std::memcpy(out, &h, sizeof(h));
    size_t off = sizeof(h);
    for (const Section& sec : sections(pl)) {
        if (cudaMemcpy(out + off, sec.dev, sec.bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
            pl.poisoned = true;
            set_error("checkpoint copy failed");
            return WFP_ECUDA;
        }
        off += sec.bytes;
    }
    return WFP_OK;
}

wfp_status wfp_checkpoint_load(wfp_plan plan, const void* buf, int64_t bytes) {
    if (!plan || !buf) {
        set_error("NULL argument");
        return WFP_EINVAL;
    }
    Plan& pl = plan_of(plan);
    if (pl.poisoned) {
        set_error("plan is poisoned");
        return WFP_ESTATE;
    }
    const Header mine = header(pl);
    Header theirs;
    if (bytes < (int64_t)sizeof(Header)) {
        set_error("not a checkpoint (too short)");
        return WFP_EINVAL;
    }
    std::memcpy(&theirs, buf, sizeof(theirs));
    if (theirs.magic != kMagic || !same_layout(mine, theirs) || bytes < theirs.total || theirs.step < 0 ||
        theirs.step > mine.Nt) {
        set_error("checkpoint does not match this plan (inputs, options or derived parameters differ)");
        return WFP_EINVAL;
    }
    if (cudaStreamSynchronize(pl.stream) != cudaSuccess) {
        pl.poisoned = true;
        set_error("stream synchronise failed");
        return WFP_ECUDA;
    }
    const unsigned char* in = (const unsigned char*)buf;
    size_t off = sizeof(Header);
    for (const Section& sec : sections(pl)) {
        if (cudaMemcpy(sec.dev, in + off, sec.bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            pl.poisoned = true;
            set_error("checkpoint copy failed");
            return WFP_ECUDA;
        }
        off += sec.bytes;
    }
    pl.step = theirs.step;
    return WFP_OK;
}

}  // extern "C"
