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

#include <nvtx3/nvToolsExt.h>

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
// Names the launches of its scope with an NVTX range (for nsys and similar tools; a no-op
// without one attached), and records an event pair around them when profiling is on and the
// stream is not being captured into a graph.
class ProfScope {
  public:
    ProfScope(const char* name, int level, cudaStream_t s) : s_(s) {
        nvtxRangePushA(name);
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
        nvtxRangePop();
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
    int phases = 1;            // phase fields, stacked phase-major (every level of the pyramid too)
    LevelGeom g[MAX_LEVELS];
    float w[MAX_LEVELS];
    int64_t off[MAX_LEVELS];   // descriptor offset of each level block
    int64_t Ktot = 0;
    int64_t N1 = 0;            // finest position count of one phase field
    ThreshConst tc;
    // workspace offsets (bytes)
    size_t o_tab = 0, tab_bytes = 0, o_scal = 0, o_pen = 0, o_desc = 0, o_pyr[MAX_LEVELS] = {},
           o_fwd[MAX_LEVELS] = {}, o_gd[MAX_LEVELS] = {}, o_adj[MAX_LEVELS] = {};
    // FFT levels: two complex FP64 grids, twiddles of the three axes, one FP64 scalar
    size_t o_fx[MAX_LEVELS] = {}, o_fh[MAX_LEVELS] = {}, o_tw[MAX_LEVELS] = {}, o_dc[MAX_LEVELS] = {};
    bool any_fft = false;
    double fh2 = 0.0;          // f(1/2)^2 of the soft threshold (App. A mapping of the FFT path)
    // three-point descriptor: per level E, E^T, W^T (hi/lo where split) and G hi/lo
    int desc_kind = DMCR_DESC_S2;
    float q_tilde = 0.f;       // corrected descriptor: 2 f(1/2)^2
    size_t o_tsum = 0;         // corrected descriptor: per-level residual sums (floats)
    int64_t s3Kpad = 0, s3Npad[MAX_LEVELS] = {};
    size_t o_eh[MAX_LEVELS] = {}, o_el[MAX_LEVELS] = {}, o_eth[MAX_LEVELS] = {}, o_etl[MAX_LEVELS] = {},
           o_w[MAX_LEVELS] = {}, o_gh[MAX_LEVELS] = {}, o_gl[MAX_LEVELS] = {}, o_amax[MAX_LEVELS] = {};
    size_t bytes = 0;
};

bool fft_size_ok(int64_t n) {
    if (n < 1 || n > 4096) return false;
    for (int r : {2, 3, 5})
        while (n % r == 0) n /= r;
    return n == 1;
}

// Identity threshold, AUTO path: the FFT when its estimated cost is lower.  Both costs are
// fitted (relative error) to GB300 measurements of descriptor + gradient on 64^3 and 128^3
// (P = 1..24): the FFT path is ~0.758 ns per grid point + 0.157 ms; the direct kernels
// ~0.148 ps per voxel-shift + 0.127 ns per point + 0.151 ms.  Measured crossovers: P = 8 on
// both grids (at P = 6 the direct path is ahead by 23% on 64^3 and 29% on 128^3).
bool fft_cheaper(const LevelGeom& g) {
    const double kfull = (double)(2 * g.P[0] + 1) * (2 * g.P[1] + 1) * (2 * g.P[2] + 1);
    const double t_direct = (double)g.N * kfull * 1.481e-13 + (double)g.N * 1.266e-10 + 1.506e-4;
    const double t_fft = (double)g.N * 7.577e-10 + 1.568e-4;
    return t_fft < t_direct;
}

// Upper bound of the segment-table bytes of one instance (every phase, 16-B aligned arrays).
size_t table_bound(int levels, int phases) {
    const size_t pp = (size_t)phases * phases;
    return (size_t)levels *
               (pp * (sizeof(FwdSeg) + sizeof(RedSeg) + sizeof(GSeg) + sizeof(AdjSeg)) +
                phases * sizeof(RestrictSeg) + 2 * sizeof(TildeSeg)) +
           sizeof(PenSeg) + sizeof(LossSeg) + phases * sizeof(FinalSeg) + sizeof(InitSeg);
}
size_t table_slack() { return (size_t)(16 + MAX_LEVELS) * 16 + 256; }

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// coefficient grid of one level and phase pair (gcoef's output)
int64_t gd_floats(const LevelGeom& g) { return (int64_t)(2 * g.P[0] + 1) * (2 * g.P[1] + 1) * g.NB * GBLOCK; }

// Forward tile rows for the whole problem (all levels share one fused launch): the tallest
// tile (fewest halo rows per output row) that still gives ~8 blocks per SM summed over levels.
// A small forward (below 2^24 pair evaluations, where the launch is latency bound) may go down
// to tiles of 4 or 2 rows: more blocks, at the price of taller halos relative to the tile.
int forward_rows(const int64_t n[3], const int P[3], int levels, int ndim) {
    const int64_t groups = ceil_div(
        (int64_t)(P[1] + 1) * ceil_div(2 * P[2] + 1, T) + (int64_t)P[0] * (2 * P[1] + 1) * ceil_div(2 * P[2] + 1, T),
        FWD_THREADS);
    int64_t pairs = 0;
    const int64_t khalf = ((int64_t)(2 * P[0] + 1) * (2 * P[1] + 1) * (2 * P[2] + 1) + 1) / 2;
    for (int l = 0; l < levels; ++l)
        pairs += (ndim == 2 ? 1 : n[0] >> l) * (n[1] >> l) * (n[2] >> l) * khalf;
    const int smallest = pairs < (1LL << 24) ? 2 : 8;
    for (int TY = 32; TY > smallest; TY /= 2) {
        int64_t blocks = 0;
        for (int l = 0; l < levels; ++l) {
            const int64_t n0 = ndim == 2 ? 1 : n[0] >> l;
            blocks += n0 * ceil_div(n[1] >> l, TY) * ceil_div(n[2] >> l, TX) * groups;
        }
        if (blocks >= 1216) return TY;
    }
    return smallest;
}

// tune: {forward tile rows (8/16/32; 0 is taken as forward_rows()), adjoint ry rows per
// chunk (0 = auto, else 1..16), adjoint chunk target limit (0 = auto, else 1..64), adjoint rx
// blocks of 8 shifts per chunk at most (0 = auto, else 1..32)}
void plan_level(LevelGeom& g, const int tune[4], int phases, int level) {
    g.N = g.n[0] * g.n[1] * g.n[2];
    g.NB = (int)ceil_div(2 * g.P[2] + 1, T);
    g.NG = (int64_t)(g.P[1] + 1) * g.NB + (int64_t)g.P[0] * (2 * g.P[1] + 1) * g.NB;
    g.Khalf = ((int64_t)(2 * g.P[0] + 1) * (2 * g.P[1] + 1) * (2 * g.P[2] + 1) + 1) / 2;
    g.NGT = g.NG * T;
    g.fwdGroupBlocks = (int)ceil_div(g.NG, FWD_THREADS);
    // forward tiles: rows per tile from forward_rows(); planes per block chosen for
    // >= ~2400 blocks
    const int64_t target = 2400, rows_target = 1216;
    g.tilesX = (int)ceil_div(g.n[2], TX);
    const int TY = (int)std::min<int64_t>(tune[0], g.n[1] + (g.n[1] & 1));   // whole row pairs
    g.TY = TY;
    g.tilesY = (int)ceil_div(g.n[1], TY);
    const int64_t perPlane = (int64_t)g.tilesY * g.tilesX * g.fwdGroupBlocks;
    int64_t pcs = std::min<int64_t>(g.n[0], std::max<int64_t>(1, ceil_div(target, perPlane)));
    g.PPB = (int)ceil_div(g.n[0], pcs);
    // the forward's per-thread block sums hold at most 64 row sums
    g.PPB = std::max(1, std::min(g.PPB, 64 / g.TY));
    g.planeChunks = (int)ceil_div(g.n[0], g.PPB);
    g.fwdTiles = (int64_t)g.planeChunks * g.tilesY * g.tilesX;
    // adjoint tiles and shift chunks
    g.adjTilesX = (int)ceil_div(g.n[2], TX);
    g.adjTilesY = (int)ceil_div(g.n[1], ADJ_ROWS);
    g.adjTiles = g.n[0] * g.adjTilesY * g.adjTilesX;
    const int wy = 2 * g.P[1] + 1, wz = 2 * g.P[0] + 1;
    // shift chunks.  A chunk's halo and coefficient loads are amortised over its
    // RZ x RY x (8 NBc) shifts: the rx blocks are split into balanced chunks of at most 12
    // (96 shifts) and the ry rows per chunk are as many as a 56 KB tile allows (4 CTAs of
    // 128 threads per SM at 128 registers), unless a level has too few tiles for ~8 blocks
    // per SM: then it splits z first and ry next (at most 32 chunks by default for the finest
    // level: levels share one fused launch, so a small level does not have to fill the GPU on
    // its own, and the gradient assembly reads few partials).
    const int nbMax = tune[3] > 0 ? tune[3] : 12;
    g.nXc = (int)ceil_div(g.NB, nbMax);
    g.NBc = (int)ceil_div(g.NB, g.nXc);
    int cap = 16;
    while (cap > 1) {
        g.RYS = cap;
        if (adj_smem_bytes(g) <= 56 * 1024) break;
        --cap;
    }
    // a level of fewer than 8 tiles (a small field) may take up to 64 chunks.  A coarser level
    // of a multigrid problem may take up to 128: its blocks come last in the fused launch
    // (heaviest first), and shorter last blocks leave the SMs less idle time at its end
    // (512^2, +-64, 3 levels: the 256^2 and 128^2 levels in 38 and 86 chunks instead of 30
    // and 30, adjoint 1.1% faster)
    const int64_t chunk_cap = tune[2] > 0 ? tune[2] : (g.adjTiles < 8 ? 64 : (level > 0 ? 128 : 32));
    const int64_t want = std::min<int64_t>(chunk_cap, std::max<int64_t>(1, ceil_div(rows_target, g.adjTiles)));
    const int64_t perX = ceil_div(want, (int64_t)g.nXc);
    const int nZc = (int)std::min<int64_t>(wz, perX);
    g.RY = (int)std::min<int64_t>(ceil_div(wy, ceil_div(perX, nZc)), cap);
    if (tune[1] > 0) g.RY = std::min(tune[1], cap);
    // several phase fields: every ordered pair is a segment of the same launch, so a chunk
    // covers `phases` times as many ry rows (staged in rounds of at most `cap` rows): fewer
    // adjoint partials to write and read back.  phases^2 times as many kept the partials of
    // three 512^2 fields in L2 but made blocks so long that the launch's tail idled: 3.4%
    // slower adjoint; one times spilled the partials: 2x the gradient assembly's time
    if (phases > 1 && tune[1] == 0) g.RY = std::min<int64_t>((int64_t)g.RY * phases, wy);
    g.RY = std::min(g.RY, wy);
    g.RYS = std::min(g.RY, cap);
    g.nYc = (int)ceil_div(wy, g.RY);
    g.RZ = (int)ceil_div(wz, nZc);
    g.nZc = (int)ceil_div(wz, g.RZ);
    // a small field (fewer than 8 tiles) whose rz and ry splits fall short of the chunk
    // target splits the rx blocks further
    if (tune[3] == 0 && g.adjTiles < 8 && (int64_t)g.nZc * g.nYc * g.nXc < want && g.NB > g.nXc) {
        const int nx = (int)std::min<int64_t>(g.NB, ceil_div(want, (int64_t)g.nZc * g.nYc));
        if (nx > g.nXc) {
            g.NBc = (int)ceil_div(g.NB, nx);
            g.nXc = (int)ceil_div(g.NB, g.NBc);
        }
    }
    g.nChunks = g.nZc * g.nYc * g.nXc;
}

dmcr_status validate_and_plan(const dmcr_params* p, Plan& pl) {
    if (p == nullptr) return fail(DMCR_EINVAL, "params is NULL");
    if (p->ndim != 2 && p->ndim != 3) return fail(DMCR_EINVAL, "ndim must be 2 or 3 (got %d)", p->ndim);
    if (p->levels < 1 || p->levels > MAX_LEVELS)
        return fail(DMCR_EINVAL, "levels must be in [1, %d] (got %d)", MAX_LEVELS, p->levels);
    if (p->threshold != DMCR_SOFT && p->threshold != DMCR_IDENTITY)
        return fail(DMCR_EINVAL, "unknown threshold %d", p->threshold);
    if (p->path != DMCR_PATH_AUTO && p->path != DMCR_PATH_DIRECT && p->path != DMCR_PATH_FFT)
        return fail(DMCR_EINVAL, "unknown path %d", p->path);
    if (!(p->tune[0] == 0 || p->tune[0] == 2 || p->tune[0] == 4 || p->tune[0] == 8 || p->tune[0] == 16 ||
          p->tune[0] == 32) || p->tune[1] < 0 ||
        p->tune[1] > 16 || p->tune[2] < 0 || p->tune[2] > 64 || p->tune[3] < 0 || p->tune[3] > 32)
        return fail(DMCR_EINVAL, "tune = {0|2|4|8|16|32, 0..16, 0..64, 0..32} expected");
    if (p->threshold == DMCR_SOFT && !(p->alpha > 0.f && isfinite(p->alpha)))
        return fail(DMCR_EINVAL, "alpha must be positive and finite");
    if (p->descriptor != DMCR_DESC_S2 && p->descriptor != DMCR_DESC_S3 && p->descriptor != DMCR_DESC_S2_TILDE)
        return fail(DMCR_EINVAL, "unknown descriptor %d", p->descriptor);
    if (p->descriptor == DMCR_DESC_S3 && p->path == DMCR_PATH_FFT)
        return fail(DMCR_ENOTSUP, "the three-point descriptor has no FFT path");
    const int phases = p->phases == 0 ? 1 : p->phases;
    if (phases < 1 || phases > MAX_PHASES) return fail(DMCR_EINVAL, "phases must be in [1, %d]", MAX_PHASES);
    if (phases > 1 && p->descriptor != DMCR_DESC_S2)
        return fail(DMCR_ENOTSUP, "several phase fields: the two-point descriptor only");
    if (phases > 1 && p->path == DMCR_PATH_FFT)
        return fail(DMCR_ENOTSUP, "several phase fields: the direct path only");
    pl.phases = phases;

    pl.desc_kind = p->descriptor;
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
        if (n[a] > (1LL << 30)) return fail(DMCR_EINVAL, "field size %lld above 2^30 on axis %d", (long long)n[a], a - first);
        if (2LL * P[a] > n[a])
            return fail(DMCR_EINVAL, "window %d exceeds half the size %lld on axis %d", P[a], (long long)n[a], a - first);
        if (n[a] % (1LL << (p->levels - 1)) != 0)
            return fail(DMCR_EINVAL, "size %lld not divisible by 2^(levels-1)", (long long)n[a]);
    }
    // every axis is <= 2^30 here, so the integer product of three axes and the phase count
    // could pass 2^63; the element count is compared in floating point (exact below 2^53,
    // and any value that rounds is far above the bound)
    if ((double)n[0] * (double)n[1] * (double)n[2] * (double)phases > 0x1p34)
        return fail(DMCR_EINVAL, "field too large: more than 2^34 elements");
    if (!isfinite(p->level_weight_exp)) return fail(DMCR_EINVAL, "level_weight_exp must be finite");
    const double we = p->level_weight_exp < 0.f ? p->ndim / 2.0 : (double)p->level_weight_exp;
    int tune[4] = {p->tune[0], p->tune[1], p->tune[2], p->tune[3]};
    if (tune[0] == 0) tune[0] = forward_rows(n, P, p->levels, p->ndim);
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
        plan_level(g, tune, phases, l);
        const bool fft_sizes = fft_size_ok(g.n[0]) && fft_size_ok(g.n[1]) && fft_size_ok(g.n[2]);
        if (p->path == DMCR_PATH_FFT) {
            if (!fft_sizes)
                return fail(DMCR_ENOTSUP, "FFT path: level %d sizes must factor into 2, 3, 5 and be <= 4096", l + 1);
            g.fft = 1;
        } else if (p->path == DMCR_PATH_AUTO && p->threshold == DMCR_IDENTITY && phases == 1 && fft_sizes &&
                   fft_cheaper(g)) {
            g.fft = 1;
        }
        if (pl.desc_kind == DMCR_DESC_S3) {
            g.fft = 0;
            g.nChunks = (int)ceil_div(g.Khalf, S3_SHIFTS);   // gather partials, one per shift chunk
        }
        if (g.fft) {
            g.nChunks = 1;
            pl.any_fft = true;
        }
        const bool direct2 = !g.fft && pl.desc_kind != DMCR_DESC_S3;
        if (direct2 && p->threshold == DMCR_IDENTITY && g.n[2] % T != 0)
            return fail(DMCR_ENOTSUP, "the direct identity path needs the last axis of every level divisible by 8");
        if (direct2 && (fwd_smem_bytes(g) > (size_t)MAX_DYN_SMEM || adj_smem_bytes(g) > (size_t)MAX_DYN_SMEM))
            return fail(DMCR_ENOTSUP, "window too large for the shared-memory tiles of this build");
        pl.w[l] = (float)pow(2.0, we * l);
        pl.off[l] = off;
        if (pl.desc_kind == DMCR_DESC_S3 && g.Khalf > 16384)
            return fail(DMCR_ENOTSUP, "three-point descriptor: at most 16384 shifts");
        off += pl.desc_kind == DMCR_DESC_S3 ? g.Khalf * g.Khalf : (int64_t)phases * phases * g.Khalf;
    }
    pl.Ktot = off;
    pl.N1 = pl.g[0].N;
    if (pl.desc_kind == DMCR_DESC_S3) {
        pl.s3Kpad = (pl.g[0].Khalf + 255) / 256 * 256;   // whole 256-wide tiles of the W GEMM
        for (int l = 0; l < pl.levels; ++l) pl.s3Npad[l] = (pl.g[l].N + 127) / 128 * 128;
    }
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
        // product form: every pair factor d = 1 + E'_x E_y stays <= 2^62, so the product of
        // two factors that share one reciprocal is finite
        tc.lim = (float)std::max(0.0, 0.5 * (61.0 - 0.75 * a * log2e));
        tc.beta = (float)(-s0);
        const double fh = c1 / (1.0 + exp(0.25 * a)) - c1 * s0;
        pl.fh2 = fh * fh;
    }
    // App. A: f(1/2) of the threshold (1/2 for f(x) = x)
    pl.q_tilde = (float)(tc.identity ? 0.5 : 2.0 * pl.fh2);
    // the workspace, estimated in floating point first: sizes beyond any device are
    // rejected before the exact layout below could wrap around
    {
        const double ph = (double)pl.phases;
        double est = 4.0 * (double)pl.Ktot;
        for (int l = 0; l < pl.levels; ++l) {
            const LevelGeom& g = pl.g[l];
            const double N = (double)g.N;
            const double chunks = pl.desc_kind == DMCR_DESC_S3 || g.fft ? (double)g.nChunks
                                                                        : (double)g.nZc * g.nYc * g.nXc;
            est += 4.0 * ph * N + 4.0 * ph * ph * chunks * N;
            if (g.fft) est += 32.0 * N;
            else if (pl.desc_kind == DMCR_DESC_S3)
                est += 12.0 * (double)pl.s3Npad[l] * (double)pl.s3Kpad + 4.0 * (double)pl.s3Kpad * (double)pl.s3Kpad;
            else est += 4.0 * ph * ph * ((double)g.fwdTiles * (double)g.Khalf + (double)gd_floats(g));
        }
        if (est > 0x1p50) return fail(DMCR_EINVAL, "the problem needs about %.3g bytes of workspace (more than 2^50)", est);
    }
    // workspace layout
    size_t o = 0;
    pl.tab_bytes = align_up(table_bound(pl.levels, pl.phases) + table_slack());
    pl.o_tab = o; o += pl.tab_bytes;
    pl.o_scal = o; o = align_up(o + sizeof(Scalars));
    pl.o_pen = o; o = align_up(o + 3 * NPEN_BLOCKS * sizeof(double));
    pl.o_desc = o; o = align_up(o + (size_t)pl.Ktot * sizeof(float));
    pl.o_tsum = o; o = align_up(o + (size_t)MAX_LEVELS * sizeof(float));
    for (int l = 0; l < pl.levels; ++l) {
        const LevelGeom& g = pl.g[l];
        const size_t ph = (size_t)pl.phases;
        if (l > 0) { pl.o_pyr[l] = o; o = align_up(o + ph * g.N * sizeof(float)); }
        if (g.fft) {
            pl.o_fx[l] = o; o = align_up(o + (size_t)g.N * 16);
            pl.o_fh[l] = o; o = align_up(o + (size_t)g.N * 16);
            pl.o_tw[l] = o; o = align_up(o + (size_t)(g.n[0] + g.n[1] + g.n[2]) * 16);
            pl.o_dc[l] = o; o = align_up(o + 16);
        } else if (pl.desc_kind == DMCR_DESC_S3) {
            const size_t Kp = (size_t)pl.s3Kpad, Np = (size_t)pl.s3Npad[l];
            // FP16 operand pairs, FP32 W^T, two scale sources
            pl.o_eh[l] = o; o = align_up(o + Np * Kp * sizeof(uint16_t));
            pl.o_el[l] = o; o = align_up(o + Np * Kp * sizeof(uint16_t));
            pl.o_eth[l] = o; o = align_up(o + Np * Kp * sizeof(uint16_t));
            pl.o_etl[l] = o; o = align_up(o + Np * Kp * sizeof(uint16_t));
            pl.o_w[l] = o; o = align_up(o + Np * Kp * sizeof(float));
            pl.o_gh[l] = o; o = align_up(o + Kp * Kp * sizeof(uint16_t));
            pl.o_gl[l] = o; o = align_up(o + Kp * Kp * sizeof(uint16_t));
            pl.o_amax[l] = o; o = align_up(o + 2 * sizeof(float));
        } else {
            pl.o_fwd[l] = o; o = align_up(o + ph * ph * g.fwdTiles * g.Khalf * sizeof(float));
        }
        if (pl.desc_kind != DMCR_DESC_S3)
            pl.o_gd[l] = o, o = align_up(o + ph * ph * gd_floats(g) * sizeof(float));
        pl.o_adj[l] = o; o = align_up(o + ph * ph * g.nChunks * g.N * sizeof(float));
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
    set_fft_attributes();
    set_gram_attributes();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(e, "cudaFuncSetAttribute");
    ready.push_back(dev);
    return DMCR_OK;
}

dmcr_status check_ws(const Plan& pl, void* ws, size_t ws_bytes) {
    if (ws == nullptr) return fail(DMCR_EINVAL, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % ALIGN != 0) return fail(DMCR_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < pl.bytes)
        return fail(DMCR_ENOMEM, "workspace too small: %zu < %zu bytes", ws_bytes, pl.bytes);
    return DMCR_OK;
}

// ---------------------------------------------------------------------------- execution engine
//
// Every entry point runs the same fused phases over a set of instances (one for the plain
// calls, many for the batched ones).  The host fills one table buffer with the segment
// arrays of every phase, writes it to the table region with blob_kernel (stream ordered,
// no host synchronisation), then launches one kernel per phase:
//   init -> restrict (per level index) -> corr_fwd -> fwd_reduce -> penalty -> loss
//        -> gcoef -> corr_adj -> final (gradient assembly, optional Adam step).
enum : unsigned {
    F_INIT = 1u,     // reset the per-instance scalars (Adam step counters)
    F_FWD = 2u,      // pyramid + descriptor
    F_LOSS = 4u,     // penalty + loss
    F_BACK = 8u,     // adjoint coefficients + adjoint + gradient assembly
    F_ADAM = 16u     // the assembly applies one Adam step instead of writing the gradient
};

struct Inst {
    const Plan* pl = nullptr;
    char* ws = nullptr;            // this instance's workspace (Plan layout)
    Scalars* sc = nullptr;         // this instance's scalars
    const float* field = nullptr;  // finest field
    float* M = nullptr;            // F_ADAM: the field updated in place
    const float* target = nullptr; // F_LOSS/F_BACK: target descriptor; VJP: upstream gradient
    float* desc = nullptr;         // descriptor output (workspace scratch if the caller gives none)
    float* loss_out = nullptr;
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-7f;
    LossParams lp{};
    float* history = nullptr;
    bool use_done = false;         // kernels skip the instance once its done flag is set
    bool round_eval = false;       // reconstruction: evaluate the rounded result once more
    int64_t step = 0;              // F_INIT: Adam steps taken before this call
    const float* lv[MAX_LEVELS] = {};
};

struct TableBuf {
    std::vector<unsigned char> h;
    size_t add(const void* p, size_t n) {
        const size_t off = (h.size() + 15) & ~size_t(15);
        h.resize(off + n);
        memcpy(h.data() + off, p, n);
        return off;
    }
};

struct Prepared {
    char* tab = nullptr;
    TableBuf tb;
    ThreshConst tc{};
    unsigned flags = 0;
    struct R {
        size_t off;
        int nseg;
        int64_t blocks;
    };
    std::vector<R> restricts;
    R fwd{0, 0, 0}, red{0, 0, 0}, pen{0, 0, 0}, loss{0, 0, 0}, gco{0, 0, 0}, adj{0, 0, 0}, fin{0, 0, 0},
        fin_small{0, 0, 0}, init{0, 0, 0}, tmap{0, 0, 0}, tsum{0, 0, 0};
    size_t smem_fwd = 0, smem_adj = 0;
    struct FftJob {
        LevelGeom g;
        const float* field;
        double2* X;
        double2* H;
        double2* tw;
        double* dc;
        float* desc;
        float weight;
        int mode;
        double fh2;
        const float* Gd;
        float* part;
    };
    std::vector<FftJob> fftf, fftb;
    std::vector<S3Job> s3f, s3b;
    template <typename S>
    const S* at(size_t off) const { return reinterpret_cast<const S*>(tab + off); }
};

template <typename S>
size_t push(TableBuf& tb, const std::vector<S>& v) {
    return v.empty() ? 0 : tb.add(v.data(), v.size() * sizeof(S));
}

bool same_thresh(const ThreshConst& a, const ThreshConst& b) {
    return a.identity == b.identity && a.kappa == b.kappa && a.cexp == b.cexp && a.c1 == b.c1 && a.c3 == b.c3;
}

Prepared::FftJob fft_job(const Inst& x, int l) {
    const Plan& pl = *x.pl;
    Prepared::FftJob j{};
    j.g = pl.g[l];
    j.field = x.lv[l];
    j.X = reinterpret_cast<double2*>(x.ws + pl.o_fx[l]);
    j.H = reinterpret_cast<double2*>(x.ws + pl.o_fh[l]);
    j.tw = reinterpret_cast<double2*>(x.ws + pl.o_tw[l]);
    j.dc = reinterpret_cast<double*>(x.ws + pl.o_dc[l]);
    j.desc = x.desc + pl.off[l];
    j.weight = pl.w[l];
    j.mode = pl.tc.identity ? 0 : 1;
    j.fh2 = pl.fh2;
    return j;
}

S3Job s3_job(const Inst& x, int l, bool loss) {
    const Plan& pl = *x.pl;
    S3Job j{};
    j.g = pl.g[l];
    j.field = x.lv[l];
    j.K = pl.g[l].Khalf;
    j.Kpad = pl.s3Kpad;
    j.Npad = pl.s3Npad[l];
    j.Eh = reinterpret_cast<uint16_t*>(x.ws + pl.o_eh[l]);
    j.El = reinterpret_cast<uint16_t*>(x.ws + pl.o_el[l]);
    j.Eth = reinterpret_cast<uint16_t*>(x.ws + pl.o_eth[l]);
    j.Etl = reinterpret_cast<uint16_t*>(x.ws + pl.o_etl[l]);
    j.W = reinterpret_cast<float*>(x.ws + pl.o_w[l]);
    j.Gh = reinterpret_cast<uint16_t*>(x.ws + pl.o_gh[l]);
    j.Gl = reinterpret_cast<uint16_t*>(x.ws + pl.o_gl[l]);
    j.amax = reinterpret_cast<float*>(x.ws + pl.o_amax[l]);
    j.desc = x.desc + pl.off[l];
    j.src = loss ? x.desc + pl.off[l] : x.target + pl.off[l];
    j.sub = loss ? x.target + pl.off[l] : nullptr;
    j.sc = loss ? x.sc : nullptr;
    j.weight = pl.w[l];
    j.part = reinterpret_cast<float*>(x.ws + pl.o_adj[l]);
    j.done = x.use_done ? &x.sc->done : nullptr;
    j.err = &x.sc->err;
    return j;
}

// Build every table of the requested phases; `tab`/`cap` is the device table region.
dmcr_status prepare(std::vector<Inst>& in, unsigned flags, char* tab, size_t cap, Prepared& P) {
    P.tab = tab;
    P.flags = flags;
    P.tc = in[0].pl->tc;
    int maxL = 0;
    for (Inst& x : in) {
        if (!same_thresh(x.pl->tc, P.tc)) return fail(DMCR_ENOTSUP, "batched instances must share threshold and alpha");
        maxL = std::max(maxL, x.pl->levels);
        x.lv[0] = x.field;
        for (int l = 1; l < x.pl->levels; ++l) x.lv[l] = reinterpret_cast<const float*>(x.ws + x.pl->o_pyr[l]);
    }
    for (const Inst& x : in)
        if (x.pl->desc_kind == DMCR_DESC_S3 && !gram_ready())
            return fail(DMCR_ENOTSUP, "the three-point descriptor needs the driver's TMA tensor-map encoder");
    const bool need_pyr = (flags & (F_FWD | F_BACK)) != 0;
    if ((flags & (F_LOSS | F_BACK)) != 0)
        for (const Inst& x : in)
            if (x.pl->any_fft && !x.pl->tc.identity)
                return fail(DMCR_ENOTSUP, "the FFT path of the soft threshold is exact for binary fields only: "
                                          "descriptor calls only (characterise targets with it)");
    if (flags & F_INIT) {
        std::vector<InitSeg> v;
        for (const Inst& x : in)
            v.push_back({x.sc, x.step, pow((double)x.beta1, (double)x.step), pow((double)x.beta2, (double)x.step)});
        P.init = {push(P.tb, v), (int)v.size(), (int64_t)v.size()};
    }
    if (need_pyr) {
        for (int l = 1; l < maxL; ++l) {
            std::vector<RestrictSeg> v;
            int64_t b = 0;
            for (const Inst& x : in) {
                if (x.pl->levels <= l) continue;
                const LevelGeom& g = x.pl->g[l];
                for (int ph = 0; ph < x.pl->phases; ++ph) {
                    RestrictSeg r{};
                    r.ndim = x.pl->ndim;
                    for (int a = 0; a < 3; ++a) r.c[a] = g.n[a];
                    r.fine = x.lv[l - 1] + (int64_t)ph * x.pl->g[l - 1].N;
                    r.coarse = const_cast<float*>(x.lv[l]) + (int64_t)ph * g.N;
                    r.done = x.use_done ? &x.sc->done : nullptr;
                    r.blockStart = b;
                    b += ceil_div(g.N, ELEM_TH);
                    v.push_back(r);
                }
            }
            P.restricts.push_back({push(P.tb, v), (int)v.size(), b});
        }
    }
    if (flags & F_FWD) {
        struct Item {
            FwdSeg f;
            int64_t work, blocks;
        };
        std::vector<Item> items;
        std::vector<RedSeg> rv;
        int64_t rb = 0;
        for (const Inst& x : in)
            for (int l = 0; l < x.pl->levels; ++l) {
                const LevelGeom& g = x.pl->g[l];
                if (x.pl->desc_kind == DMCR_DESC_S3) {
                    P.s3f.push_back(s3_job(x, l, true));
                    continue;
                }
                if (g.fft) {
                    P.fftf.push_back(fft_job(x, l));
                    continue;
                }
                // block (a, b): tails in phase a, tips in phase b (one field: the single block)
                const int nph = x.pl->phases;
                for (int pa = 0; pa < nph; ++pa)
                    for (int pb = 0; pb < nph; ++pb) {
                        const int64_t blk = (int64_t)pa * nph + pb;
                        Item it{};
                        it.f.g = g;
                        it.f.field = x.lv[l] + pa * g.N;
                        it.f.tip = x.lv[l] + pb * g.N;
                        it.f.partial = reinterpret_cast<float*>(x.ws + x.pl->o_fwd[l]) + blk * g.fwdTiles * g.Khalf;
                        it.f.done = x.use_done ? &x.sc->done : nullptr;
                        it.work = (int64_t)g.TY * g.PPB;
                        it.blocks = g.fwdTiles * g.fwdGroupBlocks;
                        items.push_back(it);
                        RedSeg r{};
                        r.g = g;
                        r.partial = it.f.partial;
                        r.desc = x.desc + x.pl->off[l] + blk * g.Khalf;
                        r.done = it.f.done;
                        r.scale = (float)((double)x.pl->w[l] / (double)g.N);
                        r.blockStart = rb;
                        rb += ceil_div(g.Khalf, RED_K);
                        rv.push_back(r);
                    }
                P.smem_fwd = std::max(P.smem_fwd, fwd_smem_bytes(g));
            }
        // heaviest blocks first: the tail of the launch is made of the light ones
        std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return a.work > b.work; });
        std::vector<FwdSeg> fv;
        int64_t b = 0;
        for (Item& it : items) {
            it.f.blockStart = b;
            b += it.blocks;
            fv.push_back(it.f);
        }
        P.fwd = {push(P.tb, fv), (int)fv.size(), b};
        P.red = {push(P.tb, rv), (int)rv.size(), rb};
        // corrected descriptor: map every level block once the whole block is written
        std::vector<TildeSeg> tv;
        int64_t tb = 0;
        for (const Inst& x : in) {
            if (x.pl->desc_kind != DMCR_DESC_S2_TILDE) continue;
            for (int l = 0; l < x.pl->levels; ++l) {
                TildeSeg t{};
                t.desc = x.desc + x.pl->off[l];
                t.K = x.pl->g[l].Khalf;
                t.q = x.pl->q_tilde;
                t.done = x.use_done ? &x.sc->done : nullptr;
                t.blockStart = tb;
                tb += ceil_div(t.K, ELEM_TH);
                tv.push_back(t);
            }
        }
        P.tmap = {push(P.tb, tv), (int)tv.size(), tb};
    }
    if (flags & F_LOSS) {
        std::vector<PenSeg> pv;
        std::vector<LossSeg> lvv;
        int maxblk = 0;
        for (const Inst& x : in) {
            double* pen = reinterpret_cast<double*>(x.ws + x.pl->o_pen);
            const int64_t Nall = x.pl->N1 * x.pl->phases;
            const int nblk = stats_blocks(x.pl->Ktot, x.lp.bc_on ? Nall : 0);
            maxblk = std::max(maxblk, nblk);
            pv.push_back({x.lp.bc_on ? x.field : nullptr, Nall, x.desc, x.target, x.pl->Ktot, pen,
                          x.use_done ? &x.sc->done : nullptr, nblk});
            LossSeg ls{};
            ls.lp = x.lp;
            ls.desc = x.desc;
            ls.target = x.target;
            ls.pen = pen;
            ls.nblk = nblk;
            ls.sc = x.sc;
            ls.loss_out = x.loss_out;
            ls.history = x.history;
            lvv.push_back(ls);
        }
        P.pen = {push(P.tb, pv), (int)pv.size(), (int64_t)maxblk};
        P.loss = {push(P.tb, lvv), (int)lvv.size(), (int64_t)lvv.size()};
    }
    if (flags & F_BACK) {
        struct Item {
            AdjSeg a;
            int64_t work, blocks;
        };
        std::vector<Item> items;
        std::vector<GSeg> gv;
        std::vector<TildeSeg> tsv;
        // gradient assembly: a small field has few positions for many chunk partials and its
        // segments go to the launch with FIN_SUB threads per position; the others to the one
        // with one thread per position
        std::vector<FinalSeg> fv, fvs;
        int64_t gb = 0, fb = 0, fbs = 0;
        const bool vjp = !(flags & F_LOSS);
        for (const Inst& x : in) {
            const int nph = x.pl->phases;
            FinalSeg fs{};
            FinalArgs& fa = fs.a;
            fa.ndim = x.pl->ndim;
            fa.levels = x.pl->levels;
            for (int a = 0; a < 3; ++a) fa.n1[a] = x.pl->g[0].n[a];
            for (int l = 0; l < x.pl->levels; ++l) {
                const LevelGeom& g = x.pl->g[l];
                float* part = reinterpret_cast<float*>(x.ws + x.pl->o_adj[l]);
                // phase a's gradient sums the partials of its nph blocks (a, b)
                fa.parts[l] = part;
                fa.nChunks[l] = nph * g.nChunks;
                fa.Nl[l] = g.N;
                for (int a = 0; a < 3; ++a) fa.nl[l][a] = g.n[a];
                if (x.pl->desc_kind == DMCR_DESC_S3) {
                    S3Job j = s3_job(x, l, !vjp);
                    j.ens = (flags & F_FWD) ? 0 : 1;
                    P.s3b.push_back(j);
                    continue;
                }
                const float* src = vjp ? x.target + x.pl->off[l] : x.desc + x.pl->off[l];
                const float* sub = vjp ? nullptr : x.target + x.pl->off[l];
                for (int pa = 0; pa < nph; ++pa)
                    for (int pb = 0; pb < nph; ++pb) {
                        const int64_t blk = (int64_t)pa * nph + pb, mir = (int64_t)pb * nph + pa;
                        float* Gd = reinterpret_cast<float*>(x.ws + x.pl->o_gd[l]) + blk * gd_floats(g);
                        GSeg gs{};
                        gs.g = g;
                        gs.src = src + blk * g.Khalf;
                        gs.sub = sub ? sub + blk * g.Khalf : nullptr;
                        gs.src2 = src + mir * g.Khalf;
                        gs.sub2 = sub ? sub + mir * g.Khalf : nullptr;
                        gs.sc = vjp ? nullptr : x.sc;
                        gs.scale = gcoef_scale(g, x.pl->tc, x.pl->w[l]);
                        gs.Gd = Gd;
                        gs.done = x.use_done ? &x.sc->done : nullptr;
                        if (x.pl->desc_kind == DMCR_DESC_S2_TILDE) {
                            TildeSeg t{};
                            t.src = gs.src;
                            t.sub = gs.sub;
                            t.tsum = reinterpret_cast<float*>(x.ws + x.pl->o_tsum) + l;
                            t.K = g.Khalf;
                            t.done = gs.done;
                            tsv.push_back(t);
                            gs.tsum = t.tsum;
                            gs.q = x.pl->q_tilde;
                        }
                        gs.blockStart = gb;
                        gb += ceil_div((int64_t)(2 * g.P[0] + 1) * (2 * g.P[1] + 1) * g.NB * T, GCOEF_TH);
                        gv.push_back(gs);
                        float* pblk = part + blk * g.nChunks * g.N;
                        if (g.fft) {
                            Prepared::FftJob j = fft_job(x, l);
                            j.Gd = Gd;
                            j.part = pblk;
                            P.fftb.push_back(j);
                            continue;
                        }
                        Item it{};
                        it.a.g = g;
                        it.a.field = x.lv[l] + pa * g.N;
                        it.a.tip = x.lv[l] + pb * g.N;
                        it.a.Gd = Gd;
                        it.a.part = pblk;
                        it.a.done = gs.done;
                        it.work = (int64_t)g.RZ * g.RY * g.NBc;
                        it.blocks = g.adjTiles * g.nChunks;
                        items.push_back(it);
                    }
                if (!g.fft) P.smem_adj = std::max(P.smem_adj, adj_smem_bytes(g));
            }
            const bool pen = !vjp && x.lp.bc_on;
            fa.field = pen ? x.field : nullptr;
            fa.sc = pen ? x.sc : nullptr;
            if (flags & F_ADAM) {
                fa.M = x.M;
                fa.m = x.m;
                fa.v = x.v;
                fa.sc = x.sc;
                fa.field = x.field;
                fa.beta1 = x.beta1;
                fa.beta2 = x.beta2;
                fa.eps = x.eps;
            } else {
                fa.grad_out = x.grad;
            }
            fs.done = x.use_done ? &x.sc->done : nullptr;
            // one assembly segment per phase field: its own partial blocks and field slices
            const int64_t N1 = x.pl->N1;
            for (int pa = 0; pa < nph; ++pa) {
                FinalSeg f = fs;
                for (int l = 0; l < x.pl->levels; ++l)
                    if (x.pl->desc_kind != DMCR_DESC_S3)
                        f.a.parts[l] = fs.a.parts[l] + (int64_t)pa * nph * x.pl->g[l].nChunks * x.pl->g[l].N;
                auto slice = [&](auto* ptr) { return ptr != nullptr ? ptr + pa * N1 : ptr; };
                f.a.field = slice(fs.a.field);
                f.a.grad_out = slice(fs.a.grad_out);
                f.a.M = slice(fs.a.M);
                f.a.m = slice(fs.a.m);
                f.a.v = slice(fs.a.v);
                if (N1 < FIN_SUB_BELOW) {
                    f.blockStart = fbs;
                    fbs += ceil_div(N1, ELEM_TH / FIN_SUB);
                    fvs.push_back(f);
                } else {
                    f.blockStart = fb;
                    fb += ceil_div(N1, ELEM_TH);
                    fv.push_back(f);
                }
            }
        }
        std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return a.work > b.work; });
        std::vector<AdjSeg> av;
        int64_t ab = 0;
        for (Item& it : items) {
            it.a.blockStart = ab;
            ab += it.blocks;
            av.push_back(it.a);
        }
        P.gco = {push(P.tb, gv), (int)gv.size(), gb};
        P.tsum = {push(P.tb, tsv), (int)tsv.size(), (int64_t)tsv.size()};
        P.adj = {push(P.tb, av), (int)av.size(), ab};
        P.fin = {push(P.tb, fv), (int)fv.size(), fb};
        P.fin_small = {push(P.tb, fvs), (int)fvs.size(), fbs};
    }
    if (P.tb.h.size() > cap) return fail(DMCR_ENOMEM, "segment tables (%zu bytes) exceed their region", P.tb.h.size());
    // every fused launch indexes its blocks with a 1-D grid
    int64_t most = std::max({P.fwd.blocks, P.red.blocks, P.gco.blocks, P.adj.blocks, P.fin.blocks, P.fin_small.blocks,
                             P.tmap.blocks});
    for (const Prepared::R& r : P.restricts) most = std::max(most, r.blocks);
    if (most > (int64_t)INT32_MAX)
        return fail(DMCR_ENOTSUP, "a fused launch would need %lld thread blocks (more than 2^31 - 1): split the batch "
                                  "or shrink the problem", (long long)most);
    return DMCR_OK;
}

// Axis passes of one grid (last axis first); the first forward pass may read the real field.
void fft_grid(const Prepared::FftJob& j, double2* data, const float* real_in, int sign, cudaStream_t s) {
    const double two_pi = 6.283185307179586476925;
    for (int axis = 2; axis >= 0; --axis) {
        const int len = (int)j.g.n[axis];
        const int64_t tw_off = axis == 2 ? 0 : (axis == 1 ? j.g.n[2] : j.g.n[2] + j.g.n[1]);
        if (len == 1) continue;
        FftPass p{};
        p.data = data;
        p.real_in = real_in;
        real_in = nullptr;
        for (int a = 0; a < 3; ++a) p.n[a] = j.g.n[a];
        p.axis = axis;
        p.sign = sign;
        p.len = len;
        p.L = fft_lines_per_block(len);
        int m = len;
        p.nrad = 0;
        while (m % 4 == 0) { p.rad[p.nrad++] = 4; m /= 4; }
        while (m % 2 == 0) { p.rad[p.nrad++] = 2; m /= 2; }
        while (m % 3 == 0) { p.rad[p.nrad++] = 3; m /= 3; }
        while (m % 5 == 0) { p.rad[p.nrad++] = 5; m /= 5; }
        p.tw = j.tw + tw_off;
        for (int t = 0; t < 3; ++t) p.om3[t] = make_double2(cos(two_pi * t / 3), -sin(two_pi * t / 3));
        for (int t = 0; t < 5; ++t) p.om5[t] = make_double2(cos(two_pi * t / 5), -sin(two_pi * t / 5));
        launch_fft_pass(p, s);
    }
    if (real_in != nullptr) {
        // a 1 x 1 x 1 grid has no pass: copy the value in through a trivial pass of length 1
        FftPass p{};
        p.data = data;
        p.real_in = real_in;
        for (int a = 0; a < 3; ++a) p.n[a] = j.g.n[a];
        p.axis = 2;
        p.sign = sign;
        p.len = 1;
        p.L = 1;
        p.nrad = 0;
        p.tw = j.tw;
        launch_fft_pass(p, s);
    }
}

void fft_twiddles(const Prepared::FftJob& j, cudaStream_t s) {
    int64_t off = 0;
    for (int axis = 2; axis >= 0; --axis) {
        if (j.g.n[axis] > 1) launch_fft_twiddles(j.tw + off, (int)j.g.n[axis], s);
        off += j.g.n[axis];
    }
}

// X = DFT(M) stays in the workspace; the power spectrum and its inverse go to H
void fft_descriptor(const Prepared::FftJob& j, cudaStream_t s) {
    fft_twiddles(j, s);
    fft_grid(j, j.X, j.field, -1, s);
    launch_fft_power(j.X, j.H, j.g.N, s);
    fft_grid(j, j.H, nullptr, +1, s);
    launch_fft_sample(j.g, j.H, j.weight, j.mode, j.fh2, j.desc, s);
}

// x_ready: the descriptor of the same call left X = DFT(M) (and the twiddles) in place
void fft_vjp(const Prepared::FftJob& j, bool x_ready, cudaStream_t s) {
    if (!x_ready) {
        fft_twiddles(j, s);
        fft_grid(j, j.X, j.field, -1, s);
    }
    launch_fft_embed(j.g, j.Gd, j.H, s);
    fft_grid(j, j.H, nullptr, -1, s);
    launch_fft_dc(j.H, j.dc, s);
    launch_fft_xcorr(j.X, j.H, j.g.N, s);
    fft_grid(j, j.H, nullptr, +1, s);
    launch_fft_vjp_combine(j.g.N, j.field, j.H, j.dc, j.part, s);
}

void upload(const Prepared& P, cudaStream_t s) {
    if (P.tb.h.empty()) return;
    ProfScope ps("tables", -1, s);
    launch_blob(P.tb.h.data(), P.tb.h.size(), P.tab, s);
}

void run(const Prepared& P, cudaStream_t s) {
    if (P.flags & F_INIT) {
        ProfScope ps("scalars_init", -1, s);
        launch_scalars_init(P.at<InitSeg>(P.init.off), P.init.nseg, s);
    }
    for (const Prepared::R& r : P.restricts) {
        ProfScope ps("restrict", -1, s);
        launch_restrict(P.at<RestrictSeg>(r.off), r.nseg, r.blocks, s);
    }
    if (P.flags & F_FWD) {
        {
            ProfScope ps("corr_fwd", -1, s);
            launch_corr_fwd(P.at<FwdSeg>(P.fwd.off), P.fwd.nseg, P.fwd.blocks, P.smem_fwd, P.tc, s);
        }
        {
            ProfScope ps("fwd_reduce", -1, s);
            launch_fwd_reduce(P.at<RedSeg>(P.red.off), P.red.nseg, P.red.blocks, s);
        }
        if (!P.fftf.empty()) {
            ProfScope ps("fft_descriptor", -1, s);
            for (const Prepared::FftJob& j : P.fftf) fft_descriptor(j, s);
        }
        if (!P.s3f.empty()) {
            ProfScope ps("s3_gram", -1, s);
            for (const S3Job& j : P.s3f) launch_s3_forward(j, P.tc, j.err, s);
        }
        if (P.tmap.nseg > 0) {
            ProfScope ps("tilde_map", -1, s);
            launch_tilde_map(P.at<TildeSeg>(P.tmap.off), P.tmap.nseg, P.tmap.blocks, s);
        }
    }
    if (P.flags & F_LOSS) {
        {
            ProfScope ps("loss_stats", -1, s);
            launch_penalty(P.at<PenSeg>(P.pen.off), P.pen.nseg, (int)P.pen.blocks, s);
        }
        ProfScope ps("loss", -1, s);
        launch_loss(P.at<LossSeg>(P.loss.off), P.loss.nseg, s);
    }
    if (P.flags & F_BACK) {
        if (P.tsum.nseg > 0) {
            ProfScope ps("tilde_sum", -1, s);
            launch_tilde_sum(P.at<TildeSeg>(P.tsum.off), P.tsum.nseg, s);
        }
        {
            ProfScope ps("gcoef", -1, s);
            launch_gcoef(P.at<GSeg>(P.gco.off), P.gco.nseg, P.gco.blocks, P.tc, s);
        }
        {
            ProfScope ps("corr_adj", -1, s);
            launch_corr_adj(P.at<AdjSeg>(P.adj.off), P.adj.nseg, P.adj.blocks, P.smem_adj, P.tc, s);
        }
        if (!P.fftb.empty()) {
            ProfScope ps("fft_vjp", -1, s);
            for (const Prepared::FftJob& j : P.fftb) fft_vjp(j, (P.flags & F_FWD) != 0, s);
        }
        if (!P.s3b.empty()) {
            ProfScope ps("s3_adjoint", -1, s);
            for (const S3Job& j : P.s3b) launch_s3_backward(j, P.tc, j.err, s);
        }
        ProfScope ps((P.flags & F_ADAM) ? "grad_adam" : "grad_assemble", -1, s);
        launch_final(P.at<FinalSeg>(P.fin.off), P.fin.nseg, P.fin.blocks, 1, s);
        launch_final(P.at<FinalSeg>(P.fin_small.off), P.fin_small.nseg, P.fin_small.blocks, FIN_SUB, s);
    }
}

LossParams make_lp(const Plan& pl, const dmcr_loss_opts* o) {
    LossParams lp;
    memset(&lp, 0, sizeof(lp));
    lp.mode = o ? o->mode : DMCR_LOSS_NORM;
    lp.lambda0 = (o && o->lambda0 >= 0.f) ? o->lambda0 : (float)pl.N1;
    lp.bc_on = o ? o->bc_on : 1;
    lp.Ktot = pl.Ktot;
    lp.N = pl.N1;
    lp.check_every = 1;
    return lp;
}

Inst single(const Plan& pl, void* ws) {
    Inst x;
    x.pl = &pl;
    x.ws = static_cast<char*>(ws);
    x.sc = reinterpret_cast<Scalars*>(x.ws + pl.o_scal);
    x.desc = reinterpret_cast<float*>(x.ws + pl.o_desc);
    return x;
}

char* table_region(const Plan& pl, void* ws) { return static_cast<char*>(ws) + pl.o_tab; }

dmcr_status exec_single(Inst& x, unsigned flags, cudaStream_t s, const char* what) {
    std::vector<Inst> in{x};
    Prepared P;
    DMCR_TRY(prepare(in, flags, table_region(*x.pl, x.ws), x.pl->tab_bytes, P));
    upload(P, s);
    run(P, s);
    return cuda_check(cudaGetLastError(), what);
}

dmcr_status check_loss_opts(const dmcr_loss_opts* o) {
    if (o != nullptr && o->mode != DMCR_LOSS_NORM && o->mode != DMCR_LOSS_SQUARED)
        return fail(DMCR_EINVAL, "unknown loss mode %d", o->mode);
    return DMCR_OK;
}

// ---------------------------------------------------------------------------- batches
//
// Batch workspace: [segment tables][count x Scalars][instance workspaces (Plan layouts)].
struct BatchLayout {
    std::vector<Plan> plans;
    std::vector<size_t> o_inst;
    size_t o_tab = 0, tab_bytes = 0, o_scal = 0, bytes = 0;
};

dmcr_status batch_layout(int count, const dmcr_params* params, BatchLayout& B) {
    if (count < 1) return fail(DMCR_EINVAL, "count must be >= 1");
    if (params == nullptr) return fail(DMCR_EINVAL, "params is NULL");
    B.plans.resize(count);
    size_t tb = table_slack();
    for (int i = 0; i < count; ++i) {
        DMCR_TRY(validate_and_plan(&params[i], B.plans[i]));
        tb += table_bound(B.plans[i].levels, B.plans[i].phases) + 32;
    }
    size_t o = 0;
    B.o_tab = o;
    B.tab_bytes = align_up(tb);
    o += B.tab_bytes;
    B.o_scal = o;
    o = align_up(o + (size_t)count * sizeof(Scalars));
    for (int i = 0; i < count; ++i) {
        B.o_inst.push_back(o);
        o = align_up(o + B.plans[i].bytes);
    }
    B.bytes = o;
    return DMCR_OK;
}

dmcr_status batch_ws(const BatchLayout& B, void* ws, size_t ws_bytes) {
    if (ws == nullptr) return fail(DMCR_EINVAL, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % ALIGN != 0) return fail(DMCR_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < B.bytes) return fail(DMCR_ENOMEM, "workspace too small: %zu < %zu bytes", ws_bytes, B.bytes);
    return DMCR_OK;
}

std::vector<Inst> batch_insts(const BatchLayout& B, void* ws) {
    std::vector<Inst> in(B.plans.size());
    char* base = static_cast<char*>(ws);
    for (size_t i = 0; i < B.plans.size(); ++i) {
        Inst& x = in[i];
        x.pl = &B.plans[i];
        x.ws = base + B.o_inst[i];
        x.sc = reinterpret_cast<Scalars*>(base + B.o_scal) + i;
        x.desc = reinterpret_cast<float*>(x.ws + B.plans[i].o_desc);
    }
    return in;
}

dmcr_status exec_batch(const BatchLayout& B, void* ws, std::vector<Inst>& in, unsigned flags, cudaStream_t s,
                       const char* what) {
    Prepared P;
    DMCR_TRY(prepare(in, flags, static_cast<char*>(ws) + B.o_tab, B.tab_bytes, P));
    upload(P, s);
    run(P, s);
    return cuda_check(cudaGetLastError(), what);
}

// Instantiated graphs of reconstruction iterations, keyed by everything the captured launch
// sequence depends on: the table bytes and where they live, every launch count and grid, the
// FFT and three-point jobs, and the device.  A server ticking the same set of jobs, or a
// caller running a reconstruction in chunks, then captures each iteration once.  The tables
// themselves are uploaded by every call (outside the graph): other calls may have reused
// the workspace in between.
struct ReconGraph {
    std::string key;
    cudaGraphExec_t exec = nullptr;
    uint64_t used = 0;
    int in_use = 0;     // calls launching it now: never evicted while in use
};
constexpr size_t RECON_GRAPH_CACHE = 32;
std::mutex g_recon_mu;
uint64_t g_recon_clock = 0;
std::vector<ReconGraph>& recon_cache() {
    static std::vector<ReconGraph>* c = new std::vector<ReconGraph>();   // lives until exit
    return *c;
}

std::string prepared_key(const Prepared& P) {
    std::string k;
    auto add = [&k](const void* p, size_t n) { k.append(static_cast<const char*>(p), n); };
    int dev = 0;
    cudaGetDevice(&dev);
    add(&dev, sizeof dev);
    add(&P.tab, sizeof P.tab);
    add(&P.flags, sizeof P.flags);
    add(&P.tc, sizeof P.tc);
    for (const Prepared::R& r : P.restricts) add(&r, sizeof r);
    for (const Prepared::R* r : {&P.fwd, &P.red, &P.pen, &P.loss, &P.gco, &P.adj, &P.fin, &P.fin_small, &P.init,
                                   &P.tmap, &P.tsum})
        add(r, sizeof *r);
    add(&P.smem_fwd, sizeof P.smem_fwd);
    add(&P.smem_adj, sizeof P.smem_adj);
    for (const auto* v : {&P.fftf, &P.fftb}) {
        const size_t n = v->size();
        add(&n, sizeof n);
        if (n) add(v->data(), n * sizeof((*v)[0]));
    }
    for (const auto* v : {&P.s3f, &P.s3b}) {
        const size_t n = v->size();
        add(&n, sizeof n);
        if (n) add(v->data(), n * sizeof((*v)[0]));
    }
    add(P.tb.h.data(), P.tb.h.size());
    return k;
}

// Takes the cached graph of `key` for this call (marked in use until recon_graph_release).
cudaGraphExec_t recon_graph_acquire(const std::string& key) {
    std::lock_guard<std::mutex> lk(g_recon_mu);
    for (ReconGraph& g : recon_cache())
        if (g.key == key) {
            g.used = ++g_recon_clock;
            ++g.in_use;
            return g.exec;
        }
    return nullptr;
}

// The call that acquired (or stored) `exec` is done with it: its stream has been synchronized,
// so no launch of it is pending.
void recon_graph_release(cudaGraphExec_t exec) {
    std::lock_guard<std::mutex> lk(g_recon_mu);
    for (ReconGraph& g : recon_cache())
        if (g.exec == exec && g.in_use > 0) {
            --g.in_use;
            return;
        }
}

// Stores a new graph, marked in use by the storing call.  Returns false (the caller keeps
// and destroys the graph) when every cached graph is in use.  An evicted graph has no
// pending launch: its last user synchronized before releasing it.
bool recon_graph_store(const std::string& key, cudaGraphExec_t exec) {
    std::lock_guard<std::mutex> lk(g_recon_mu);
    std::vector<ReconGraph>& c = recon_cache();
    ReconGraph g;
    g.key = key;
    g.exec = exec;
    g.used = ++g_recon_clock;
    g.in_use = 1;
    if (c.size() < RECON_GRAPH_CACHE) {
        c.push_back(g);
        return true;
    }
    ReconGraph* lru = nullptr;
    for (ReconGraph& e : c)
        if (e.in_use == 0 && (lru == nullptr || e.used < lru->used)) lru = &e;
    if (lru == nullptr) return false;
    cudaGraphExecDestroy(lru->exec);
    *lru = g;
    return true;
}

// Graph-captured reconstruction of every instance (each stops on its own device flag).
dmcr_status reconstruct_insts(std::vector<Inst>& in, char* tab, size_t tab_cap, Scalars* scal_base,
                              const std::vector<int>& max_iters, int poll_every, dmcr_recon_report* reports,
                              dmcr_adam_state* states, cudaStream_t caller, bool per_instance_status) {
    const int count = (int)in.size();
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;      // a graph of this call only (the cache was full of graphs in use)
    cudaGraphExec_t cached = nullptr;    // the cache's graph, in use by this call
    dmcr_status st = DMCR_OK;
    std::vector<Scalars> hs(count);
    do {
        // the captured graph runs on a private stream with the caller stream's priority
        int prio = 0;
        if (cudaStreamGetPriority(caller, &prio) != cudaSuccess) {
            cudaGetLastError();
            prio = 0;
        }
        if ((st = cuda_check(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio), "cudaStreamCreate")))
            break;
        if ((st = cuda_check(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "cudaEventCreate"))) break;
        if ((st = cuda_check(cudaEventRecord(ev, caller), "cudaEventRecord"))) break;
        if ((st = cuda_check(cudaStreamWaitEvent(s, ev, 0), "cudaStreamWaitEvent"))) break;
        Prepared P0;
        if ((st = prepare(in, F_INIT, tab, tab_cap, P0))) break;
        upload(P0, s);
        run(P0, s);
        Prepared P;
        if ((st = prepare(in, F_FWD | F_LOSS | F_BACK | F_ADAM, tab, tab_cap, P))) break;
        upload(P, s);
        const std::string key = prepared_key(P);
        cached = recon_graph_acquire(key);
        if (cached == nullptr) {
            if ((st = cuda_check(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "BeginCapture"))) break;
            run(P, s);
            if ((st = cuda_check(cudaStreamEndCapture(s, &graph), "EndCapture"))) break;
            if ((st = cuda_check(cudaGraphInstantiate(&exec, graph, 0), "GraphInstantiate"))) break;
            if (recon_graph_store(key, exec)) {    // the cache owns it from here
                cached = exec;
                exec = nullptr;
            }
        }
        cudaGraphExec_t run_exec = cached != nullptr ? cached : exec;
        int most = 0;
        for (int k : max_iters) most = std::max(most, k);
        // iteration max_iters evaluates the final field and sets the done flag
        int launched = 0;
        while (launched <= most) {
            const int k = std::min(poll_every, most + 1 - launched);
            for (int i = 0; i < k && !st; ++i) st = cuda_check(cudaGraphLaunch(run_exec, s), "GraphLaunch");
            if (st) break;
            launched += k;
            if ((st = cuda_check(cudaMemcpyAsync(hs.data(), scal_base, count * sizeof(Scalars), cudaMemcpyDeviceToHost,
                                                 s), "scalars D2H")))
                break;
            if ((st = cuda_check(cudaStreamSynchronize(s), "sync"))) break;
            bool all = true;
            for (const Scalars& x : hs) all = all && x.done != 0;
            if (all) break;
        }
        if (st) break;
        for (int i = 0; i < count; ++i) {
            memset(&reports[i], 0, sizeof(reports[i]));
            fill_report(hs[i], states[i].step, &reports[i]);
            states[i].step = hs[i].adam_step;
        }
        int bad = 0;
        st = call_status(hs.data(), count, per_instance_status, &bad);
        if (st == DMCR_ETIMEOUT) st = fail(st, "a bounded tensor-core wait timed out in instance %d", bad);
        else if (st == DMCR_ENONFINITE) st = fail(st, "loss became non-finite in instance %d", bad);
        if (st) break;
        // one more evaluation, of the returned fields rounded to phases 0/1 (Sec. 4.1) where
        // asked for: a rounded field goes to its first level's adjoint partials, which no
        // forward pass uses
        std::vector<Inst> rin;
        std::vector<int> rid;
        for (int i = 0; i < count; ++i) {
            reports[i].rounded_rel_err = NAN;
            if (in[i].round_eval) {
                rin.push_back(in[i]);
                rid.push_back(i);
            }
        }
        if (rin.empty()) break;
        for (Inst& y : rin) {
            float* rf = reinterpret_cast<float*>(y.ws + y.pl->o_adj[0]);
            launch_round_field(y.field, rf, y.pl->N1 * y.pl->phases, s);
            y.field = rf;
            y.M = nullptr;
            y.loss_out = nullptr;
            y.grad = nullptr;
            y.m = y.v = nullptr;
            y.history = nullptr;
            y.use_done = false;
            y.lp.recon = 0;
        }
        Prepared PR;
        if ((st = prepare(rin, F_FWD | F_LOSS, tab, tab_cap, PR))) break;
        upload(PR, s);
        run(PR, s);
        if ((st = cuda_check(cudaMemcpyAsync(hs.data(), scal_base, count * sizeof(Scalars), cudaMemcpyDeviceToHost, s),
                             "scalars D2H")))
            break;
        if ((st = cuda_check(cudaStreamSynchronize(s), "sync"))) break;
        for (int i : rid) reports[i].rounded_rel_err = hs[i].err ? NAN : hs[i].loss[5];
    } while (0);
    if (s) cudaStreamSynchronize(s);     // no launch of either graph is pending past here
    if (cached) recon_graph_release(cached);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (s) cudaStreamDestroy(s);
    if (ev) cudaEventDestroy(ev);
    return st;
}

dmcr_status check_recon_opts(const dmcr_recon_opts* o) {
    if (o == nullptr) return fail(DMCR_EINVAL, "opts is NULL");
    if (o->max_iters < 0 || o->check_every < 1) return fail(DMCR_EINVAL, "max_iters >= 0 and check_every >= 1");
    if (o->init != DMCR_INIT_CALLER && o->init != DMCR_INIT_UNIFORM_SEEDED)
        return fail(DMCR_EINVAL, "unknown init %d", o->init);
    return check_loss_opts(&o->loss);
}

void recon_inst(Inst& x, const dmcr_recon_opts* o, const float* target, float* field, const dmcr_adam_state* st,
                float* history) {
    x.field = field;
    x.M = field;
    x.target = target;
    x.m = st->m;
    x.v = st->v;
    x.beta1 = o->beta1;
    x.beta2 = o->beta2;
    x.eps = o->eps;
    x.lp = make_lp(*x.pl, &o->loss);
    x.lp.tol_rel = o->tol_rel;
    x.lp.check_every = o->check_every;
    x.lp.lr = o->lr;
    x.lp.beta1 = o->beta1;
    x.lp.beta2 = o->beta2;
    x.lp.max_iters = o->max_iters;
    x.lp.recon = 1;
    x.history = history;
    x.use_done = true;
    x.round_eval = o->report_rounded != 0;
    x.step = st->step;
}

// ---------------------------------------------------------------------------- cached iteration graphs
//
// dmcr_adam_step(_batched) is called once per iteration with the same arguments over and
// over; for small problems its ten launches, the planning and the table building cost more
// than the arithmetic.  The first call with a given set of arguments therefore captures the
// iteration (table upload + every kernel) into a CUDA graph on a private stream and keeps
// the instantiated graph; a later call with the same arguments launches one small kernel
// that sets the Adam step scalars of this call (passed by value) and the graph.  The key is
// every argument that shapes the launch sequence or that the tables point to: the params
// and options field by field, all pointers, the workspace size and the device.  Calls made
// while the stream is being captured by the caller, or while the library's per-kernel
// timers are on, take the direct launches.
struct KeyBuf {
    std::string b;
    template <typename V>
    void add(const V& v) { b.append(reinterpret_cast<const char*>(&v), sizeof(V)); }
};

void key_params(KeyBuf& k, const dmcr_params& p) {
    k.add(p.ndim);
    for (int a = 0; a < 3; ++a) k.add(p.n[a]), k.add(p.window[a]);
    k.add(p.levels), k.add(p.threshold), k.add(p.alpha), k.add(p.level_weight_exp), k.add(p.path);
    for (int a = 0; a < 4; ++a) k.add(p.tune[a]);
    k.add(p.descriptor), k.add(p.phases);
}

void key_adam_opts(KeyBuf& k, const dmcr_recon_opts& o) {
    k.add(o.lr), k.add(o.beta1), k.add(o.beta2), k.add(o.eps), k.add(o.loss.mode), k.add(o.loss.lambda0),
        k.add(o.loss.bc_on);
}

struct StepGraph {
    std::string key;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;     // recorded after every replay: eviction waits for it
    std::vector<Scalars*> sc;       // per instance
    float beta1 = 0.9f, beta2 = 0.999f;
    uint64_t used = 0;
};

constexpr size_t GRAPH_CACHE = 16;
std::mutex g_graph_mu;
// never freed: the graphs live until the process exits (a destructor at exit could run
// after the CUDA context is gone)
std::vector<StepGraph>& graph_cache() {
    static std::vector<StepGraph>* c = new std::vector<StepGraph>();
    return *c;
}
uint64_t g_graph_clock = 0;

bool graphs_usable(cudaStream_t s) {
    {
        ProfState& p = prof();
        std::lock_guard<std::mutex> lk(p.mu);
        if (p.on) return false;        // per-kernel event timers need the direct launches
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs == cudaStreamCaptureStatusNone;
}

// Launch the cached graph of `key` for Adam steps steps[i] + 1; false if there is none.  The
// launches are enqueued under the cache's lock (no other thread can evict the graph
// meanwhile), followed by an event that an eviction waits for.
bool replay_step_graph(const std::string& key, const int64_t* steps, cudaStream_t s, dmcr_status* st) {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (StepGraph& g : graph_cache())
        if (g.key == key) {
            g.used = ++g_graph_clock;
            std::vector<InitSeg> init;
            for (size_t i = 0; i < g.sc.size(); ++i)
                init.push_back({g.sc[i], steps[i], pow((double)g.beta1, (double)steps[i]),
                                pow((double)g.beta2, (double)steps[i])});
            launch_scalars_set(init.data(), (int)init.size(), s);
            *st = cuda_check(cudaGetLastError(), "scalars set");
            if (*st == DMCR_OK) *st = cuda_check(cudaGraphLaunch(g.exec, s), "cudaGraphLaunch (cached iteration)");
            if (*st == DMCR_OK) *st = cuda_check(cudaEventRecord(g.done, s), "cudaEventRecord (cached iteration)");
            return true;
        }
    return false;
}

// Capture the prepared iteration (tables + kernels, no scalar initialisation) into a graph
// and store it under `key`.  Returns false (and leaves no error pending) if anything fails.
bool capture_step_graph(const std::string& key, const Prepared& P, const std::vector<Inst>& in) {
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        upload(P, cs);
        run(P, cs);
        ok = cudaStreamEndCapture(cs, &graph) == cudaSuccess && graph != nullptr;
    }
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    cudaEvent_t done = nullptr;
    if (ok) ok = cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    cudaGetLastError();
    if (!ok) {
        if (exec) cudaGraphExecDestroy(exec);
        return false;
    }
    StepGraph g;
    g.key = key;
    g.exec = exec;
    g.done = done;
    for (const Inst& x : in) g.sc.push_back(x.sc);
    g.beta1 = in[0].beta1;
    g.beta2 = in[0].beta2;
    std::lock_guard<std::mutex> lk(g_graph_mu);
    std::vector<StepGraph>& c = graph_cache();
    g.used = ++g_graph_clock;
    if (c.size() >= GRAPH_CACHE) {
        auto lru = std::min_element(c.begin(), c.end(), [](const StepGraph& a, const StepGraph& b) { return a.used < b.used; });
        // its last replay may still be queued: wait for it before the graph is destroyed
        cudaEventSynchronize(lru->done);
        cudaGraphExecDestroy(lru->exec);
        cudaEventDestroy(lru->done);
        *lru = g;
    } else {
        c.push_back(g);
    }
    return true;
}

// One Adam iteration of the instances: from the cache when possible, else prepared here
// (and captured for the next call when graphs are usable).
dmcr_status adam_iteration(const std::string& key, std::vector<Inst>& in, char* tab, size_t tab_cap,
                           cudaStream_t s, const char* what) {
    const bool graphs = graphs_usable(s);
    std::vector<int64_t> steps;
    for (const Inst& x : in) steps.push_back(x.step);
    dmcr_status st = DMCR_OK;
    if (graphs && replay_step_graph(key, steps.data(), s, &st)) return st;
    if (graphs) {
        Prepared P;
        DMCR_TRY(prepare(in, F_FWD | F_LOSS | F_BACK | F_ADAM, tab, tab_cap, P));
        if (capture_step_graph(key, P, in) && replay_step_graph(key, steps.data(), s, &st)) return st;
    }
    Prepared P;
    DMCR_TRY(prepare(in, F_INIT | F_FWD | F_LOSS | F_BACK | F_ADAM, tab, tab_cap, P));
    upload(P, s);
    run(P, s);
    return cuda_check(cudaGetLastError(), what);
}

}  // namespace

// ---------------------------------------------------------------------------- C ABI

extern "C" {

int dmcr_version(void) { return 200; }

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
    Inst x = single(pl, ws);
    x.field = field;
    x.desc = desc;
    return exec_single(x, F_FWD, static_cast<cudaStream_t>(stream), "dmcr_descriptor launch");
}

dmcr_status dmcr_loss_grad(const dmcr_params* p, const dmcr_loss_opts* opts, const float* field,
                           const float* target_desc, float* loss_out, float* grad, float* desc_out, void* ws,
                           size_t ws_bytes, void* stream) {
    Plan pl;
    DMCR_TRY(validate_and_plan(p, pl));
    if (field == nullptr || target_desc == nullptr) return fail(DMCR_EINVAL, "field/target is NULL");
    DMCR_TRY(check_loss_opts(opts));
    DMCR_TRY(check_ws(pl, ws, ws_bytes));
    DMCR_TRY(prepare_device());
    Inst x = single(pl, ws);
    x.field = field;
    x.target = target_desc;
    if (desc_out != nullptr) x.desc = desc_out;
    x.loss_out = loss_out;
    x.grad = grad;
    x.lp = make_lp(pl, opts);
    return exec_single(x, F_FWD | F_LOSS | (grad != nullptr ? F_BACK : 0u), static_cast<cudaStream_t>(stream),
                       "dmcr_loss_grad launch");
}

dmcr_status dmcr_descriptor_vjp(const dmcr_params* p, const float* field, const float* grad_desc, float* grad_field,
                                void* ws, size_t ws_bytes, void* stream) {
    Plan pl;
    DMCR_TRY(validate_and_plan(p, pl));
    if (field == nullptr || grad_desc == nullptr || grad_field == nullptr)
        return fail(DMCR_EINVAL, "field/grad_desc/grad_field is NULL");
    DMCR_TRY(check_ws(pl, ws, ws_bytes));
    DMCR_TRY(prepare_device());
    Inst x = single(pl, ws);
    x.field = field;
    x.target = grad_desc;
    x.grad = grad_field;
    return exec_single(x, F_BACK, static_cast<cudaStream_t>(stream), "dmcr_descriptor_vjp launch");
}

dmcr_status dmcr_restrict(int ndim, const int64_t n_fine[3], const float* fine, float* coarse, void* stream) {
    if (ndim != 2 && ndim != 3) return fail(DMCR_EINVAL, "ndim must be 2 or 3");
    if (n_fine == nullptr || fine == nullptr || coarse == nullptr) return fail(DMCR_EINVAL, "NULL argument");
    int64_t nf[3];
    if (ndim == 2) { nf[0] = 1; nf[1] = n_fine[0]; nf[2] = n_fine[1]; }
    else { nf[0] = n_fine[0]; nf[1] = n_fine[1]; nf[2] = n_fine[2]; }
    for (int a = (ndim == 2 ? 1 : 0); a < 3; ++a)
        if (nf[a] < 2 || nf[a] % 2) return fail(DMCR_EINVAL, "fine sizes must be even and >= 2");
    launch_restrict_one(ndim, nf, fine, coarse, static_cast<cudaStream_t>(stream));
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

dmcr_status dmcr_adam_step(const dmcr_params* p, const dmcr_recon_opts* o, const float* target_desc, float* field,
                           dmcr_adam_state* state, float* loss_out, void* ws, size_t ws_bytes, void* stream) {
    if (p == nullptr || o == nullptr || target_desc == nullptr || field == nullptr || state == nullptr ||
        state->m == nullptr || state->v == nullptr)
        return fail(DMCR_EINVAL, "NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    DMCR_TRY(cuda_check(cudaGetDevice(&dev), "cudaGetDevice"));
    KeyBuf k;
    k.add(dev);
    k.add(1);
    key_params(k, *p);
    key_adam_opts(k, *o);
    k.add(target_desc), k.add(field), k.add(state->m), k.add(state->v), k.add(loss_out), k.add(ws), k.add(ws_bytes);
    dmcr_status st = DMCR_OK;
    if (graphs_usable(s) && replay_step_graph(k.b, &state->step, s, &st)) {
        if (st == DMCR_OK) state->step += 1;
        return st;
    }
    Plan pl;
    DMCR_TRY(validate_and_plan(p, pl));
    DMCR_TRY(check_loss_opts(&o->loss));
    DMCR_TRY(check_ws(pl, ws, ws_bytes));
    DMCR_TRY(prepare_device());
    std::vector<Inst> in{single(pl, ws)};
    dmcr_recon_opts one = *o;
    one.max_iters = 1;
    one.tol_rel = 0.f;
    one.check_every = 1;
    recon_inst(in[0], &one, target_desc, field, state, nullptr);
    in[0].loss_out = loss_out;
    DMCR_TRY(adam_iteration(k.b, in, table_region(pl, ws), pl.tab_bytes, s, "dmcr_adam_step launch"));
    state->step += 1;
    return DMCR_OK;
}

dmcr_status dmcr_reconstruct(const dmcr_params* p, const dmcr_recon_opts* o, const float* target_desc, float* field,
                             dmcr_adam_state* state, float* history, dmcr_recon_report* report, void* ws,
                             size_t ws_bytes, void* stream) {
    Plan pl;
    DMCR_TRY(validate_and_plan(p, pl));
    if (target_desc == nullptr || field == nullptr || state == nullptr || report == nullptr ||
        state->m == nullptr || state->v == nullptr)
        return fail(DMCR_EINVAL, "NULL argument");
    DMCR_TRY(check_recon_opts(o));
    DMCR_TRY(check_ws(pl, ws, ws_bytes));
    DMCR_TRY(prepare_device());
    memset(report, 0, sizeof(*report));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (o->init == DMCR_INIT_UNIFORM_SEEDED) launch_init_uniform(field, pl.N1 * pl.phases, o->seed, s);
    std::vector<Inst> in{single(pl, ws)};
    recon_inst(in[0], o, target_desc, field, state, history);
    const dmcr_status st = reconstruct_insts(in, table_region(pl, ws), pl.tab_bytes, in[0].sc, {o->max_iters},
                                             o->check_every, report, state, s, false);
    report->status = st;
    return st;
}

// ---------------------------------------------------------------------------- batched calls

dmcr_status dmcr_batch_workspace_size(int count, const dmcr_params* params, size_t* bytes) {
    BatchLayout B;
    DMCR_TRY(batch_layout(count, params, B));
    if (bytes == nullptr) return fail(DMCR_EINVAL, "bytes is NULL");
    *bytes = B.bytes;
    return DMCR_OK;
}

dmcr_status dmcr_descriptor_batched(int count, const dmcr_params* params, const float* const* fields,
                                    float* const* descs, void* ws, size_t ws_bytes, void* stream) {
    BatchLayout B;
    DMCR_TRY(batch_layout(count, params, B));
    if (fields == nullptr || descs == nullptr) return fail(DMCR_EINVAL, "NULL pointer array");
    DMCR_TRY(batch_ws(B, ws, ws_bytes));
    DMCR_TRY(prepare_device());
    std::vector<Inst> in = batch_insts(B, ws);
    for (int i = 0; i < count; ++i) {
        if (fields[i] == nullptr || descs[i] == nullptr) return fail(DMCR_EINVAL, "NULL pointer in instance %d", i);
        in[i].field = fields[i];
        in[i].desc = descs[i];
    }
    return exec_batch(B, ws, in, F_FWD, static_cast<cudaStream_t>(stream), "dmcr_descriptor_batched launch");
}

dmcr_status dmcr_loss_grad_batched(int count, const dmcr_params* params, const dmcr_loss_opts* opts,
                                   const float* const* fields, const float* const* targets, float* loss_out,
                                   float* const* grads, void* ws, size_t ws_bytes, void* stream) {
    BatchLayout B;
    DMCR_TRY(batch_layout(count, params, B));
    if (fields == nullptr || targets == nullptr) return fail(DMCR_EINVAL, "NULL pointer array");
    DMCR_TRY(check_loss_opts(opts));
    DMCR_TRY(batch_ws(B, ws, ws_bytes));
    DMCR_TRY(prepare_device());
    std::vector<Inst> in = batch_insts(B, ws);
    for (int i = 0; i < count; ++i) {
        if (fields[i] == nullptr || targets[i] == nullptr) return fail(DMCR_EINVAL, "NULL pointer in instance %d", i);
        in[i].field = fields[i];
        in[i].target = targets[i];
        in[i].loss_out = loss_out != nullptr ? loss_out + (size_t)DMCR_OUT_COUNT * i : nullptr;
        in[i].grad = grads != nullptr ? grads[i] : nullptr;
        in[i].lp = make_lp(B.plans[i], opts);
    }
    return exec_batch(B, ws, in, F_FWD | F_LOSS | (grads != nullptr ? F_BACK : 0u), static_cast<cudaStream_t>(stream),
                      "dmcr_loss_grad_batched launch");
}

dmcr_status dmcr_descriptor_vjp_batched(int count, const dmcr_params* params, const float* const* fields,
                                        const float* const* grad_descs, float* const* grad_fields, void* ws,
                                        size_t ws_bytes, void* stream) {
    BatchLayout B;
    DMCR_TRY(batch_layout(count, params, B));
    if (fields == nullptr || grad_descs == nullptr || grad_fields == nullptr)
        return fail(DMCR_EINVAL, "NULL pointer array");
    DMCR_TRY(batch_ws(B, ws, ws_bytes));
    DMCR_TRY(prepare_device());
    std::vector<Inst> in = batch_insts(B, ws);
    for (int i = 0; i < count; ++i) {
        if (fields[i] == nullptr || grad_descs[i] == nullptr || grad_fields[i] == nullptr)
            return fail(DMCR_EINVAL, "NULL pointer in instance %d", i);
        in[i].field = fields[i];
        in[i].target = grad_descs[i];
        in[i].grad = grad_fields[i];
    }
    return exec_batch(B, ws, in, F_BACK, static_cast<cudaStream_t>(stream), "dmcr_descriptor_vjp_batched launch");
}

dmcr_status dmcr_adam_step_batched(int count, const dmcr_params* params, const dmcr_recon_opts* opts,
                                   const float* const* targets, float* const* fields, dmcr_adam_state* states,
                                   float* loss_out, void* ws, size_t ws_bytes, void* stream) {
    if (count < 1) return fail(DMCR_EINVAL, "count must be >= 1");
    if (params == nullptr || opts == nullptr || targets == nullptr || fields == nullptr || states == nullptr)
        return fail(DMCR_EINVAL, "NULL argument");
    for (int i = 0; i < count; ++i)
        if (targets[i] == nullptr || fields[i] == nullptr || states[i].m == nullptr || states[i].v == nullptr)
            return fail(DMCR_EINVAL, "NULL pointer in instance %d", i);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    DMCR_TRY(cuda_check(cudaGetDevice(&dev), "cudaGetDevice"));
    KeyBuf k;
    k.add(dev);
    k.add(count);
    key_adam_opts(k, *opts);
    for (int i = 0; i < count; ++i) {
        key_params(k, params[i]);
        k.add(targets[i]), k.add(fields[i]), k.add(states[i].m), k.add(states[i].v);
    }
    k.add(loss_out), k.add(ws), k.add(ws_bytes);
    std::vector<int64_t> steps(count);
    for (int i = 0; i < count; ++i) steps[i] = states[i].step;
    dmcr_status st = DMCR_OK;
    if (graphs_usable(s) && replay_step_graph(k.b, steps.data(), s, &st)) {
        if (st == DMCR_OK)
            for (int i = 0; i < count; ++i) states[i].step += 1;
        return st;
    }
    BatchLayout B;
    DMCR_TRY(batch_layout(count, params, B));
    DMCR_TRY(check_loss_opts(&opts->loss));
    DMCR_TRY(batch_ws(B, ws, ws_bytes));
    DMCR_TRY(prepare_device());
    std::vector<Inst> in = batch_insts(B, ws);
    dmcr_recon_opts one = *opts;
    one.max_iters = 1;
    one.tol_rel = 0.f;
    one.check_every = 1;
    for (int i = 0; i < count; ++i) {
        recon_inst(in[i], &one, targets[i], fields[i], &states[i], nullptr);
        in[i].loss_out = loss_out != nullptr ? loss_out + (size_t)DMCR_OUT_COUNT * i : nullptr;
    }
    DMCR_TRY(adam_iteration(k.b, in, static_cast<char*>(ws) + B.o_tab, B.tab_bytes, s,
                            "dmcr_adam_step_batched launch"));
    for (int i = 0; i < count; ++i) states[i].step += 1;
    return DMCR_OK;
}

dmcr_status dmcr_reconstruct_batched(int count, const dmcr_params* params, const dmcr_recon_opts* opts,
                                     const float* const* targets, float* const* fields, dmcr_adam_state* states,
                                     dmcr_recon_report* reports, void* ws, size_t ws_bytes, void* stream) {
    BatchLayout B;
    DMCR_TRY(batch_layout(count, params, B));
    if (opts == nullptr || targets == nullptr || fields == nullptr || states == nullptr || reports == nullptr)
        return fail(DMCR_EINVAL, "NULL argument");
    DMCR_TRY(batch_ws(B, ws, ws_bytes));
    DMCR_TRY(prepare_device());
    std::vector<Inst> in = batch_insts(B, ws);
    std::vector<int> iters(count);
    int poll = 1 << 30;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < count; ++i) {
        DMCR_TRY(check_recon_opts(&opts[i]));
        if (targets[i] == nullptr || fields[i] == nullptr || states[i].m == nullptr || states[i].v == nullptr)
            return fail(DMCR_EINVAL, "NULL pointer in instance %d", i);
        recon_inst(in[i], &opts[i], targets[i], fields[i], &states[i], nullptr);
        iters[i] = opts[i].max_iters;
        poll = std::min(poll, opts[i].check_every);
    }
    for (int i = 0; i < count; ++i)
        if (opts[i].init == DMCR_INIT_UNIFORM_SEEDED)
            launch_init_uniform(fields[i], B.plans[i].N1 * B.plans[i].phases, opts[i].seed, s);
    return reconstruct_insts(in, static_cast<char*>(ws) + B.o_tab, B.tab_bytes,
                             reinterpret_cast<Scalars*>(static_cast<char*>(ws) + B.o_scal), iters, poll, reports,
                             states, s, true);
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
    if (pl.desc_kind != DMCR_DESC_S2 || pl.any_fft || pl.phases != 1)
        return fail(DMCR_ENOTSUP, "dmcr_descriptor_noalloc computes the direct two-point descriptor of one field only");
    // compact layout: segment tables, pyramid levels 2.. and the forward partials of every level
    Plan cp = pl;
    size_t o = 0;
    cp.o_tab = o;
    o += cp.tab_bytes;
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
    // every scratch entry read below is written first in the same call: nothing to clear
    Inst x;
    x.pl = &cp;
    x.ws = static_cast<char*>(scratch);
    x.field = field;
    x.desc = desc;
    return exec_single(x, F_FWD, static_cast<cudaStream_t>(stream), "dmcr_descriptor_noalloc launch");
}
