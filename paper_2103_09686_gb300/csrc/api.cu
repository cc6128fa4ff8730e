// C ABI of the dmcr library (declared in include/dmcr.h): argument validation, the
// per-level launch plan, the workspace layout and the call sequences of the paper's
// hot path (Sec. 3.1-3.3, App. B).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "dmcr.h"

using namespace dmcr;

namespace {

thread_local char g_err[512] = "";

dmcr_status fail(dmcr_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

dmcr_status cuda_check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) return fail(DMCR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return DMCR_OK;
}

// ---------------------------------------------------------------- per-kernel event timing
struct ProfPending {
    std::string name;
    cudaEvent_t a, b;
};
struct ProfState {
    std::mutex mu;
    bool on = false;
    std::vector<ProfPending> pending;
    std::vector<cudaEvent_t> pool;
    std::vector<std::string> names;
    std::vector<double> ms;
    std::vector<int64_t> count;
};
ProfState& prof() {
    static ProfState p;
    return p;
}
cudaEvent_t prof_event(ProfState& p) {
    if (!p.pool.empty()) {
        cudaEvent_t e = p.pool.back();
        p.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
void prof_collect(ProfState& p) {
    for (auto& r : p.pending) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        size_t i = 0;
        while (i < p.names.size() && p.names[i] != r.name) ++i;
        if (i == p.names.size()) { p.names.push_back(r.name); p.ms.push_back(0.0); p.count.push_back(0); }
        p.ms[i] += ms;
        p.count[i] += 1;
        p.pool.push_back(r.a);
        p.pool.push_back(r.b);
    }
    p.pending.clear();
}
// Records an event pair around the launches of its scope when profiling is on and the
// stream is not being captured into a graph.
class ProfScope {
  public:
    ProfScope(const char* name, int level, cudaStream_t s) : s_(s) {
        ProfState& p = prof();
        if (!p.on) return;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            return;
        }
        std::lock_guard<std::mutex> lk(p.mu);
        name_ = level >= 0 ? std::string(name) + "[L" + std::to_string(level + 1) + "]" : std::string(name);
        a_ = prof_event(p);
        b_ = prof_event(p);
        cudaEventRecord(a_, s);
        active_ = true;
    }
    ~ProfScope() {
        if (!active_) return;
        ProfState& p = prof();
        std::lock_guard<std::mutex> lk(p.mu);
        cudaEventRecord(b_, s_);
        p.pending.push_back({name_, a_, b_});
    }

  private:
    cudaStream_t s_;
    bool active_ = false;
    std::string name_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};

#define DMCR_TRY(expr)                         \
    do {                                       \
        dmcr_status _st = (expr);              \
        if (_st != DMCR_OK) return _st;        \
    } while (0)

constexpr int MAX_LEVELS = 8;
constexpr size_t ALIGN = 256;

size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct Plan {
    int ndim = 2;
    int levels = 1;
    LevelGeom g[MAX_LEVELS];
    float w[MAX_LEVELS];
    int64_t off[MAX_LEVELS];   // descriptor offset of each level block
    int64_t Ktot = 0;
    int64_t N1 = 0;
    ThreshConst tc;
    // workspace offsets (bytes)
    size_t o_scal = 0, o_pen = 0, o_desc = 0, o_pyr[MAX_LEVELS] = {}, o_fwd[MAX_LEVELS] = {},
           o_gd[MAX_LEVELS] = {}, o_adj[MAX_LEVELS] = {};
    size_t bytes = 0;
};

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

void plan_level(LevelGeom& g) {
    g.N = g.n[0] * g.n[1] * g.n[2];
    g.NB = (int)ceil_div(2 * g.P[2] + 1, T);
    g.NG = (int64_t)(g.P[1] + 1) * g.NB + (int64_t)g.P[0] * (2 * g.P[1] + 1) * g.NB;
    g.Khalf = ((int64_t)(2 * g.P[0] + 1) * (2 * g.P[1] + 1) * (2 * g.P[2] + 1) + 1) / 2;
    g.NGT = g.NG * T;
    g.fwdGroupBlocks = (int)ceil_div(g.NG, FWD_THREADS);
    // forward tiles: rows per tile and planes per block chosen for >= ~2400 blocks
    const int64_t target = 2400;
    g.tilesX = (int)ceil_div(g.n[2], TX);
    int TY = (int)std::min<int64_t>(32, g.n[1]);
    while (TY > 8 && (int64_t)ceil_div(g.n[1], TY) * g.tilesX * g.fwdGroupBlocks * g.n[0] < target) TY /= 2;
    g.TY = TY;
    g.tilesY = (int)ceil_div(g.n[1], TY);
    const int64_t perPlane = (int64_t)g.tilesY * g.tilesX * g.fwdGroupBlocks;
    int64_t pcs = std::min<int64_t>(g.n[0], std::max<int64_t>(1, ceil_div(target, perPlane)));
    g.PPB = (int)ceil_div(g.n[0], pcs);
    g.planeChunks = (int)ceil_div(g.n[0], g.PPB);
    g.fwdTiles = (int64_t)g.planeChunks * g.tilesY * g.tilesX;
    // adjoint tiles and shift chunks
    g.adjTilesX = (int)ceil_div(g.n[2], TX);
    g.adjTilesY = (int)ceil_div(g.n[1], 32);
    g.adjTiles = g.n[0] * g.adjTilesY * g.adjTilesX;
    const int wy = 2 * g.P[1] + 1, wz = 2 * g.P[0] + 1;
    int64_t want = std::max<int64_t>(1, ceil_div(target, g.adjTiles));
    int nYc = (int)std::min<int64_t>(wy, want);
    g.RY = (int)ceil_div(wy, nYc);
    if (g.RY > 16) g.RY = 16;
    g.nYc = (int)ceil_div(wy, g.RY);
    int nZc = (int)std::min<int64_t>(wz, ceil_div(want, g.nYc));
    g.RZ = (int)ceil_div(wz, nZc);
    g.nZc = (int)ceil_div(wz, g.RZ);
    g.nChunks = g.nZc * g.nYc;
}

dmcr_status validate_and_plan(const dmcr_params* p, Plan& pl) {
    if (p == nullptr) return fail(DMCR_EINVAL, "params is NULL");
    if (p->ndim != 2 && p->ndim != 3) return fail(DMCR_EINVAL, "ndim must be 2 or 3 (got %d)", p->ndim);
    if (p->levels < 1 || p->levels > MAX_LEVELS)
        return fail(DMCR_EINVAL, "levels must be in [1, %d] (got %d)", MAX_LEVELS, p->levels);
    if (p->threshold != DMCR_SOFT && p->threshold != DMCR_IDENTITY)
        return fail(DMCR_EINVAL, "unknown threshold %d", p->threshold);
    if (p->path != DMCR_PATH_AUTO && p->path != DMCR_PATH_DIRECT)
        return fail(DMCR_ENOTSUP, "path %d is not available in this build", p->path);
    if (p->threshold == DMCR_SOFT && !(p->alpha > 0.f && isfinite(p->alpha)))
        return fail(DMCR_EINVAL, "alpha must be positive and finite");
    pl.ndim = p->ndim;
    pl.levels = p->levels;
    int64_t n[3];
    int P[3];
    if (p->ndim == 2) {
        n[0] = 1; n[1] = p->n[0]; n[2] = p->n[1];
        P[0] = 0; P[1] = p->window[0]; P[2] = p->window[1];
    } else {
        for (int a = 0; a < 3; ++a) { n[a] = p->n[a]; P[a] = p->window[a]; }
    }
    const int first = p->ndim == 2 ? 1 : 0;
    for (int a = first; a < 3; ++a) {
        if (n[a] < 1) return fail(DMCR_EINVAL, "field size must be positive");
        if (P[a] < 0) return fail(DMCR_EINVAL, "window must be >= 0");
        if (n[a] % (1LL << (p->levels - 1)) != 0)
            return fail(DMCR_EINVAL, "size %lld not divisible by 2^(levels-1)", (long long)n[a]);
    }
    if (n[0] * n[1] * n[2] > (1LL << 34)) return fail(DMCR_EINVAL, "field too large");
    const double we = p->level_weight_exp < 0.f ? p->ndim / 2.0 : (double)p->level_weight_exp;
    int64_t off = 0;
    for (int l = 0; l < p->levels; ++l) {
        LevelGeom& g = pl.g[l];
        memset(&g, 0, sizeof(g));
        g.n[0] = p->ndim == 2 ? 1 : n[0] >> l;
        g.n[1] = n[1] >> l;
        g.n[2] = n[2] >> l;
        for (int a = 0; a < 3; ++a) g.P[a] = P[a];
        for (int a = first; a < 3; ++a)
            if (2LL * P[a] > g.n[a])
                return fail(DMCR_EINVAL, "window %d exceeds half the level-%d size %lld on axis %d", P[a], l + 1,
                            (long long)g.n[a], a - first);
        if (p->threshold == DMCR_IDENTITY && g.n[2] % T != 0)
            return fail(DMCR_ENOTSUP, "the identity threshold needs the last axis of every level divisible by 8");
        plan_level(g);
        if (fwd_smem_bytes(g) > (size_t)MAX_DYN_SMEM || adj_smem_bytes(g) > (size_t)MAX_DYN_SMEM)
            return fail(DMCR_ENOTSUP, "window too large for the shared-memory tiles of this build");
        pl.w[l] = (float)pow(2.0, we * l);
        pl.off[l] = off;
        off += g.Khalf;
    }
    pl.Ktot = off;
    pl.N1 = pl.g[0].N;
    // threshold constants (FP64 on the host, rounded once)
    ThreshConst& tc = pl.tc;
    memset(&tc, 0, sizeof(tc));
    tc.identity = p->threshold == DMCR_IDENTITY;
    if (!tc.identity) {
        const double a = p->alpha;
        const double log2e = 1.4426950408889634074;
        // f(x) = c1 sigma(alpha (x - 0.75)) + c3 with f(0) = 0, f(1) = 1
        const double s0 = 1.0 / (1.0 + exp(0.75 * a));
        const double s1 = 1.0 / (1.0 + exp(-0.25 * a));
        const double c1 = 1.0 / (s1 - s0);
        tc.c1 = (float)c1;
        tc.c3 = (float)(-c1 * s0);
        tc.alpha = (float)a;
        tc.kappa = (float)(0.5 * a * log2e);
        tc.cexp = (float)(0.75 * a * log2e);
        tc.lim = (float)std::max(0.0, 100.0 - 0.75 * a * log2e);
    }
    // workspace layout
    size_t o = 0;
    pl.o_scal = o; o = align_up(o + sizeof(Scalars));
    pl.o_pen = o; o = align_up(o + NPEN_BLOCKS * sizeof(double));
    pl.o_desc = o; o = align_up(o + (size_t)pl.Ktot * sizeof(float));
    for (int l = 0; l < pl.levels; ++l) {
        const LevelGeom& g = pl.g[l];
        if (l > 0) { pl.o_pyr[l] = o; o = align_up(o + (size_t)g.N * sizeof(float)); }
        pl.o_fwd[l] = o; o = align_up(o + (size_t)g.fwdTiles * g.Khalf * sizeof(float));
        pl.o_gd[l] = o; o = align_up(o + (size_t)(2 * g.P[0] + 1) * (2 * g.P[1] + 1) * g.NB * T * sizeof(float));
        pl.o_adj[l] = o; o = align_up(o + (size_t)g.nChunks * g.N * sizeof(float));
    }
    pl.bytes = o;
    return DMCR_OK;
}

dmcr_status prepare_device() {
    static std::mutex mu;
    static std::vector<int> ready;
    int dev = 0;
    DMCR_TRY(cuda_check(cudaGetDevice(&dev), "cudaGetDevice"));
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(ready.begin(), ready.end(), dev) != ready.end()) return DMCR_OK;
    set_kernel_attributes();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(e, "cudaFuncSetAttribute");
    ready.push_back(dev);
    return DMCR_OK;
}

struct Ws {
    char* base;
    const Plan* pl;
    Scalars* scal() const { return reinterpret_cast<Scalars*>(base + pl->o_scal); }
    double* pen() const { return reinterpret_cast<double*>(base + pl->o_pen); }
    float* desc() const { return reinterpret_cast<float*>(base + pl->o_desc); }
    float* fwd(int l) const { return reinterpret_cast<float*>(base + pl->o_fwd[l]); }
    float* gd(int l) const { return reinterpret_cast<float*>(base + pl->o_gd[l]); }
    float* adj(int l) const { return reinterpret_cast<float*>(base + pl->o_adj[l]); }
};

dmcr_status check_ws(const Plan& pl, void* ws, size_t ws_bytes) {
    if (ws == nullptr) return fail(DMCR_EINVAL, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % ALIGN != 0) return fail(DMCR_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < pl.bytes)
        return fail(DMCR_ENOMEM, "workspace too small: %zu < %zu bytes", ws_bytes, pl.bytes);
    return DMCR_OK;
}

// Pyramid level pointers: level 0 is the caller's field.
void pyramid(const Plan& pl, const Ws& w, const float* field, const float* lv[MAX_LEVELS], const int* done,
             cudaStream_t s) {
    lv[0] = field;
    for (int l = 1; l < pl.levels; ++l) {
        float* dst = reinterpret_cast<float*>(w.base + pl.o_pyr[l]);
        const LevelGeom& gf = pl.g[l - 1];
        int64_t nf[3] = {gf.n[0], gf.n[1], gf.n[2]};
        ProfScope ps("restrict", l, s);
        launch_restrict(pl.ndim, nf, lv[l - 1], dst, done, s);
        lv[l] = dst;
    }
}

void forward(const Plan& pl, const Ws& w, const float* const lv[MAX_LEVELS], float* desc, const int* done,
             cudaStream_t s) {
    for (int l = 0; l < pl.levels; ++l) {
        {
            ProfScope ps("corr_fwd", l, s);
            launch_corr_fwd(pl.g[l], pl.tc, lv[l], w.fwd(l), done, s);
        }
        ProfScope ps("fwd_reduce", l, s);
        launch_fwd_reduce(pl.g[l], pl.tc, w.fwd(l), pl.w[l], desc + pl.off[l], done, s);
    }
}

// Adjoint of every level for coefficients built from src (- sub), then the fused gradient
// assembly (and Adam step when M != nullptr).
void backward(const Plan& pl, const Ws& w, const float* const lv[MAX_LEVELS], const float* src, const float* sub,
              const Scalars* gsc, const float* field_pen, const Scalars* pensc, float* grad_out, float* M, float* m,
              float* v, float b1, float b2, float eps, const int* done, cudaStream_t s) {
    FinalArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.ndim = pl.ndim;
    fa.levels = pl.levels;
    for (int a = 0; a < 3; ++a) fa.n1[a] = pl.g[0].n[a];
    for (int l = 0; l < pl.levels; ++l) {
        const LevelGeom& g = pl.g[l];
        {
            ProfScope ps("gcoef", l, s);
            launch_gcoef(g, pl.tc, src + pl.off[l], sub != nullptr ? sub + pl.off[l] : nullptr, gsc, pl.w[l],
                         w.gd(l), done, s);
        }
        {
            ProfScope ps("corr_adj", l, s);
            launch_corr_adj(g, pl.tc, lv[l], w.gd(l), w.adj(l), done, s);
        }
        fa.parts[l] = w.adj(l);
        fa.nChunks[l] = g.nChunks;
        fa.Nl[l] = g.N;
        for (int a = 0; a < 3; ++a) fa.nl[l][a] = g.n[a];
    }
    fa.field = field_pen;
    fa.sc = pensc;
    fa.grad_out = grad_out;
    fa.M = M;
    fa.m = m;
    fa.v = v;
    fa.beta1 = b1;
    fa.beta2 = b2;
    fa.eps = eps;
    ProfScope ps(M != nullptr ? "grad_adam" : "grad_assemble", -1, s);
    launch_final(fa, done, s);
}

void penalty_and_loss(const Plan& pl, const Ws& w, const LossParams& lp, const float* field, const float* desc,
                      const float* target, float* loss_out, float* history, const int* done, cudaStream_t s) {
    if (lp.bc_on) {
        ProfScope ps("penalty", -1, s);
        launch_penalty(field, pl.N1, w.pen(), done, s);
    }
    ProfScope ps("loss", -1, s);
    launch_loss(lp, desc, target, lp.bc_on ? w.pen() : nullptr, w.scal(), loss_out, history, s);
}

LossParams make_lp(const Plan& pl, const dmcr_loss_opts* o) {
    LossParams lp;
    memset(&lp, 0, sizeof(lp));
    lp.mode = o ? o->mode : DMCR_LOSS_NORM;
    lp.lambda0 = (o && o->lambda0 >= 0.f) ? o->lambda0 : (float)pl.N1;
    lp.bc_on = o ? o->bc_on : 1;
    lp.Ktot = pl.Ktot;
    lp.N = pl.N1;
    return lp;
}

}  // namespace

// ---------------------------------------------------------------------------- C ABI

extern "C" {

int dmcr_version(void) { return 100; }

const char* dmcr_last_error(void) { return g_err; }

dmcr_status dmcr_descriptor_length(const dmcr_params* p, int64_t* length) {
    Plan pl;
    DMCR_TRY(validate_and_plan(p, pl));
    if (length == nullptr) return fail(DMCR_EINVAL, "length is NULL");
    *length = pl.Ktot;
    return DMCR_OK;
}

dmcr_status dmcr_workspace_size(const dmcr_params* p, size_t* bytes) {
    Plan pl;
    DMCR_TRY(validate_and_plan(p, pl));
    if (bytes == nullptr) return fail(DMCR_EINVAL, "bytes is NULL");
    *bytes = pl.bytes;
    return DMCR_OK;
}

dmcr_status dmcr_descriptor(const dmcr_params* p, const float* field, float* desc, void* ws, size_t ws_bytes,
                            void* stream) {
    Plan pl;
    DMCR_TRY(validate_and_plan(p, pl));
    if (field == nullptr || desc == nullptr) return fail(DMCR_EINVAL, "field/desc is NULL");
    DMCR_TRY(check_ws(pl, ws, ws_bytes));
    DMCR_TRY(prepare_device());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Ws w{static_cast<char*>(ws), &pl};
    const float* lv[MAX_LEVELS];
    pyramid(pl, w, field, lv, nullptr, s);
    forward(pl, w, lv, desc, nullptr, s);
    return cuda_check(cudaGetLastError(), "dmcr_descriptor launch");
}

dmcr_status dmcr_loss_grad(const dmcr_params* p, const dmcr_loss_opts* opts, const float* field,
                           const float* target_desc, float* loss_out, float* grad, float* desc_out, void* ws,
                           size_t ws_bytes, void* stream) {
    Plan pl;
    DMCR_TRY(validate_and_plan(p, pl));
    if (field == nullptr || target_desc == nullptr) return fail(DMCR_EINVAL, "field/target is NULL");
    if (opts != nullptr && opts->mode != DMCR_LOSS_NORM && opts->mode != DMCR_LOSS_SQUARED)
        return fail(DMCR_EINVAL, "unknown loss mode %d", opts->mode);
    DMCR_TRY(check_ws(pl, ws, ws_bytes));
    DMCR_TRY(prepare_device());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Ws w{static_cast<char*>(ws), &pl};
    const float* lv[MAX_LEVELS];
    float* desc = desc_out != nullptr ? desc_out : w.desc();
    const LossParams lp = make_lp(pl, opts);
    pyramid(pl, w, field, lv, nullptr, s);
    forward(pl, w, lv, desc, nullptr, s);
    penalty_and_loss(pl, w, lp, field, desc, target_desc, loss_out, nullptr, nullptr, s);
    if (grad != nullptr)
        backward(pl, w, lv, desc, target_desc, w.scal(), field, lp.bc_on ? w.scal() : nullptr, grad, nullptr, nullptr,
                 nullptr, 0.f, 0.f, 0.f, nullptr, s);
    return cuda_check(cudaGetLastError(), "dmcr_loss_grad launch");
}

dmcr_status dmcr_descriptor_vjp(const dmcr_params* p, const float* field, const float* grad_desc, float* grad_field,
                                void* ws, size_t ws_bytes, void* stream) {
    Plan pl;
    DMCR_TRY(validate_and_plan(p, pl));
    if (field == nullptr || grad_desc == nullptr || grad_field == nullptr)
        return fail(DMCR_EINVAL, "field/grad_desc/grad_field is NULL");
    DMCR_TRY(check_ws(pl, ws, ws_bytes));
    DMCR_TRY(prepare_device());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Ws w{static_cast<char*>(ws), &pl};
    const float* lv[MAX_LEVELS];
    pyramid(pl, w, field, lv, nullptr, s);
    backward(pl, w, lv, grad_desc, nullptr, nullptr, nullptr, nullptr, grad_field, nullptr, nullptr, nullptr, 0.f, 0.f,
             0.f, nullptr, s);
    return cuda_check(cudaGetLastError(), "dmcr_descriptor_vjp launch");
}

dmcr_status dmcr_restrict(int ndim, const int64_t n_fine[3], const float* fine, float* coarse, void* stream) {
    if (ndim != 2 && ndim != 3) return fail(DMCR_EINVAL, "ndim must be 2 or 3");
    if (n_fine == nullptr || fine == nullptr || coarse == nullptr) return fail(DMCR_EINVAL, "NULL argument");
    int64_t nf[3];
    if (ndim == 2) { nf[0] = 1; nf[1] = n_fine[0]; nf[2] = n_fine[1]; }
    else { nf[0] = n_fine[0]; nf[1] = n_fine[1]; nf[2] = n_fine[2]; }
    for (int a = (ndim == 2 ? 1 : 0); a < 3; ++a)
        if (nf[a] < 2 || nf[a] % 2) return fail(DMCR_EINVAL, "fine sizes must be even and >= 2");
    launch_restrict(ndim, nf, fine, coarse, nullptr, static_cast<cudaStream_t>(stream));
    return cuda_check(cudaGetLastError(), "dmcr_restrict launch");
}

dmcr_status dmcr_prolongate(int ndim, const int64_t n_coarse[3], const float* coarse, float* fine, int mode,
                            void* stream) {
    if (ndim != 2 && ndim != 3) return fail(DMCR_EINVAL, "ndim must be 2 or 3");
    if (n_coarse == nullptr || fine == nullptr || coarse == nullptr) return fail(DMCR_EINVAL, "NULL argument");
    if (mode != DMCR_PROLONG_ADJOINT_ACCUMULATE && mode != DMCR_PROLONG_INJECT)
        return fail(DMCR_EINVAL, "unknown prolongation mode %d", mode);
    int64_t nc[3];
    if (ndim == 2) { nc[0] = 1; nc[1] = n_coarse[0]; nc[2] = n_coarse[1]; }
    else { nc[0] = n_coarse[0]; nc[1] = n_coarse[1]; nc[2] = n_coarse[2]; }
    for (int a = (ndim == 2 ? 1 : 0); a < 3; ++a)
        if (nc[a] < 1) return fail(DMCR_EINVAL, "coarse sizes must be positive");
    launch_prolongate(ndim, nc, coarse, fine, mode, static_cast<cudaStream_t>(stream));
    return cuda_check(cudaGetLastError(), "dmcr_prolongate launch");
}

dmcr_status dmcr_init_uniform(float* field, int64_t count, uint64_t seed, void* stream) {
    if (field == nullptr || count < 0) return fail(DMCR_EINVAL, "bad field/count");
    if (count == 0) return DMCR_OK;
    launch_init_uniform(field, count, seed, static_cast<cudaStream_t>(stream));
    return cuda_check(cudaGetLastError(), "dmcr_init_uniform launch");
}

dmcr_status dmcr_reconstruct(const dmcr_params* p, const dmcr_recon_opts* o, const float* target_desc,
                             float* field, dmcr_adam_state* state, float* history, dmcr_recon_report* report,
                             void* ws, size_t ws_bytes, void* stream) {
    Plan pl;
    DMCR_TRY(validate_and_plan(p, pl));
    if (o == nullptr || target_desc == nullptr || field == nullptr || state == nullptr || report == nullptr ||
        state->m == nullptr || state->v == nullptr)
        return fail(DMCR_EINVAL, "NULL argument");
    if (o->max_iters < 0 || o->check_every < 1) return fail(DMCR_EINVAL, "max_iters >= 0 and check_every >= 1");
    if (o->init != DMCR_INIT_CALLER && o->init != DMCR_INIT_UNIFORM_SEEDED)
        return fail(DMCR_EINVAL, "unknown init %d", o->init);
    if (o->loss.mode != DMCR_LOSS_NORM && o->loss.mode != DMCR_LOSS_SQUARED)
        return fail(DMCR_EINVAL, "unknown loss mode %d", o->loss.mode);
    DMCR_TRY(check_ws(pl, ws, ws_bytes));
    DMCR_TRY(prepare_device());
    memset(report, 0, sizeof(*report));
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    dmcr_status st = DMCR_OK;
    Ws w{static_cast<char*>(ws), &pl};
    Scalars* dsc = w.scal();
    const int* done = &dsc->done;
    LossParams lp = make_lp(pl, &o->loss);
    lp.tol_rel = o->tol_rel;
    lp.check_every = o->check_every;
    lp.lr = o->lr;
    lp.beta1 = o->beta1;
    lp.beta2 = o->beta2;
    lp.max_iters = o->max_iters;
    lp.recon = 1;
    const float* lv[MAX_LEVELS];

    do {
        if ((st = cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreate"))) break;
        if ((st = cuda_check(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "cudaEventCreate"))) break;
        if ((st = cuda_check(cudaEventRecord(ev, caller), "cudaEventRecord"))) break;
        if ((st = cuda_check(cudaStreamWaitEvent(s, ev, 0), "cudaStreamWaitEvent"))) break;
        if (o->init == DMCR_INIT_UNIFORM_SEEDED) launch_init_uniform(field, pl.N1, o->seed, s);
        launch_scalars_init(dsc, state->step, s);
        // one iteration, captured once
        if ((st = cuda_check(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "BeginCapture"))) break;
        pyramid(pl, w, field, lv, done, s);
        forward(pl, w, lv, w.desc(), done, s);
        penalty_and_loss(pl, w, lp, field, w.desc(), target_desc, nullptr, history, done, s);
        backward(pl, w, lv, w.desc(), target_desc, dsc, field, lp.bc_on ? dsc : nullptr, nullptr, field, state->m,
                 state->v, o->beta1, o->beta2, o->eps, done, s);
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if ((st = cuda_check(ce, "EndCapture"))) break;
        if ((st = cuda_check(cudaGraphInstantiate(&exec, graph, 0), "GraphInstantiate"))) break;
        Scalars hs;
        int launched = 0;
        while (launched < o->max_iters) {
            const int k = std::min(o->check_every, o->max_iters - launched);
            for (int i = 0; i < k; ++i)
                if ((st = cuda_check(cudaGraphLaunch(exec, s), "GraphLaunch"))) break;
            if (st) break;
            launched += k;
            if ((st = cuda_check(cudaMemcpyAsync(&hs, dsc, sizeof(hs), cudaMemcpyDeviceToHost, s), "scalars D2H")))
                break;
            if ((st = cuda_check(cudaStreamSynchronize(s), "sync"))) break;
            if (hs.done) break;
        }
        if (st) break;
        if ((st = cuda_check(cudaMemcpyAsync(&hs, dsc, sizeof(hs), cudaMemcpyDeviceToHost, s), "scalars D2H"))) break;
        if ((st = cuda_check(cudaStreamSynchronize(s), "sync"))) break;
        report->converged = hs.done == 1;
        report->iterations = (int)(hs.adam_step - state->step);
        state->step = hs.adam_step;
        if (hs.done == 2) {
            st = fail(DMCR_ENONFINITE, "loss became non-finite at iteration %d", hs.iter);
            break;
        }
        // loss of the returned field (not counted as an iteration)
        LossParams lq = make_lp(pl, &o->loss);
        pyramid(pl, w, field, lv, nullptr, s);
        forward(pl, w, lv, w.desc(), nullptr, s);
        penalty_and_loss(pl, w, lq, field, w.desc(), target_desc, nullptr, nullptr, nullptr, s);
        if ((st = cuda_check(cudaMemcpyAsync(&hs, dsc, sizeof(hs), cudaMemcpyDeviceToHost, s), "scalars D2H"))) break;
        if ((st = cuda_check(cudaStreamSynchronize(s), "sync"))) break;
        for (int i = 0; i < DMCR_OUT_COUNT; ++i) report->loss[i] = hs.loss[i];
        if (o->tol_rel > 0.f && hs.loss[DMCR_OUT_REL_ERR] < o->tol_rel) report->converged = 1;
    } while (0);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    if (ev) cudaEventDestroy(ev);
    report->status = st;
    return st;
}

dmcr_status dmcr_adam_step(const dmcr_params* p, const dmcr_recon_opts* o, const float* target_desc, float* field,
                           dmcr_adam_state* state, float* loss_out, void* ws, size_t ws_bytes, void* stream) {
    Plan pl;
    DMCR_TRY(validate_and_plan(p, pl));
    if (o == nullptr || target_desc == nullptr || field == nullptr || state == nullptr || state->m == nullptr ||
        state->v == nullptr)
        return fail(DMCR_EINVAL, "NULL argument");
    if (o->loss.mode != DMCR_LOSS_NORM && o->loss.mode != DMCR_LOSS_SQUARED)
        return fail(DMCR_EINVAL, "unknown loss mode %d", o->loss.mode);
    DMCR_TRY(check_ws(pl, ws, ws_bytes));
    DMCR_TRY(prepare_device());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Ws w{static_cast<char*>(ws), &pl};
    Scalars* dsc = w.scal();
    const int* done = &dsc->done;
    LossParams lp = make_lp(pl, &o->loss);
    lp.tol_rel = 0.f;
    lp.check_every = 1;
    lp.lr = o->lr;
    lp.beta1 = o->beta1;
    lp.beta2 = o->beta2;
    lp.max_iters = 1;
    lp.recon = 1;
    const float* lv[MAX_LEVELS];
    {
        ProfScope ps("scalars_init", -1, s);
        launch_scalars_init(dsc, state->step, s);
    }
    pyramid(pl, w, field, lv, nullptr, s);
    forward(pl, w, lv, w.desc(), nullptr, s);
    penalty_and_loss(pl, w, lp, field, w.desc(), target_desc, loss_out, nullptr, nullptr, s);
    backward(pl, w, lv, w.desc(), target_desc, dsc, field, lp.bc_on ? dsc : nullptr, nullptr, field, state->m,
             state->v, o->beta1, o->beta2, o->eps, done, s);
    DMCR_TRY(cuda_check(cudaGetLastError(), "dmcr_adam_step launch"));
    state->step += 1;
    return DMCR_OK;
}

dmcr_status dmcr_profile_enable(int on) {
    ProfState& p = prof();
    std::lock_guard<std::mutex> lk(p.mu);
    p.on = on != 0;
    return DMCR_OK;
}

dmcr_status dmcr_profile_reset(void) {
    ProfState& p = prof();
    std::lock_guard<std::mutex> lk(p.mu);
    prof_collect(p);
    p.names.clear();
    p.ms.clear();
    p.count.clear();
    return DMCR_OK;
}

dmcr_status dmcr_profile_read(int index, char* name, int name_len, double* total_ms, int64_t* launches) {
    ProfState& p = prof();
    std::lock_guard<std::mutex> lk(p.mu);
    prof_collect(p);
    if (index < 0 || index >= (int)p.names.size()) return fail(DMCR_EINVAL, "no profile entry %d", index);
    if (name != nullptr && name_len > 0) {
        strncpy(name, p.names[index].c_str(), (size_t)name_len - 1);
        name[name_len - 1] = 0;
    }
    if (total_ms != nullptr) *total_ms = p.ms[index];
    if (launches != nullptr) *launches = p.count[index];
    return DMCR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------- allocation-free descriptor
//
// Some callers cannot allocate device memory while they run: code called from a host
// callback or a real-time loop in which cudaMalloc (or any allocating library) is not
// allowed, and deployments that reserve all device memory at start-up.  For them, dmcr_descriptor_noalloc evaluates the same descriptor as dmcr_descriptor with its
// scratch memory taken from one file-scope device array of fixed size, DMCR_NOALLOC_SCRATCH_BYTES,
// that every GPU loading this library holds until the process exits.
namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[DMCR_NOALLOC_SCRATCH_BYTES];

struct NoallocDev {
    int dev;
    void* ptr;
};

// Host-side lookup of the array's device address, once per device with that device current.
dmcr_status noalloc_scratch(void** out) {
    static std::mutex mu;
    static std::vector<NoallocDev> table;
    int dev = 0;
    DMCR_TRY(cuda_check(cudaGetDevice(&dev), "cudaGetDevice"));
    std::lock_guard<std::mutex> lk(mu);
    for (const NoallocDev& d : table)
        if (d.dev == dev) {
            *out = d.ptr;
            return DMCR_OK;
        }
    void* ptr = nullptr;
    DMCR_TRY(cuda_check(cudaGetSymbolAddress(&ptr, g_noalloc_scratch), "cudaGetSymbolAddress(scratch)"));
    table.push_back({dev, ptr});
    *out = ptr;
    return DMCR_OK;
}

}  // namespace

extern "C" dmcr_status dmcr_descriptor_noalloc(const dmcr_params* p, const float* field, float* desc, void* stream) {
    Plan pl;
    DMCR_TRY(validate_and_plan(p, pl));
    if (field == nullptr || desc == nullptr) return fail(DMCR_EINVAL, "field/desc is NULL");
    // compact layout: pyramid levels 2.. and the forward partials of every level
    Plan cp = pl;
    size_t o = 0;
    for (int l = 0; l < cp.levels; ++l) {
        const LevelGeom& g = cp.g[l];
        if (l > 0) { cp.o_pyr[l] = o; o = align_up(o + (size_t)g.N * sizeof(float)); }
        cp.o_fwd[l] = o; o = align_up(o + (size_t)g.fwdTiles * g.Khalf * sizeof(float));
    }
    if (o > (size_t)DMCR_NOALLOC_SCRATCH_BYTES)
        return fail(DMCR_ENOMEM, "dmcr_descriptor_noalloc needs %zu bytes of scratch, more than its fixed %zu bytes; "
                    "use dmcr_descriptor with a caller workspace", o, (size_t)DMCR_NOALLOC_SCRATCH_BYTES);
    void* scratch = nullptr;
    DMCR_TRY(noalloc_scratch(&scratch));
    DMCR_TRY(prepare_device());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Ws w{static_cast<char*>(scratch), &cp};
    const float* lv[MAX_LEVELS];
    // every scratch entry read below is written first in the same call: nothing to clear
    pyramid(cp, w, field, lv, nullptr, s);
    forward(cp, w, lv, desc, nullptr, s);
    return cuda_check(cudaGetLastError(), "dmcr_descriptor_noalloc launch");
}
