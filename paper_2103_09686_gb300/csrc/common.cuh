// Shared declarations of the dmcr CUDA library (kernels + C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "scalars.h"

namespace dmcr {

constexpr int T = 8;            // shifts per thread (forward) / positions per strip (adjoint)
constexpr int TX = 32;          // tile width in positions (fastest axis)
constexpr int FWD_THREADS = 128;
constexpr int ADJ_THREADS = 128;   // 32 row pairs (lane, lane + 32) x 4 strips of 8 positions
constexpr int ADJ_ROWS = 64;       // adjoint tile rows
constexpr int GBLOCK = 48;         // coefficient floats per block of 8 shifts (packed pairs)
constexpr int S3_SHIFTS = 32;      // three-point gradient gather: shifts per partial sum

// offset of C_m inside a coefficient block: (C_m, C_m, C_m+1, C_m+1) after the 8 (A, A, B, B)
__host__ __device__ inline int gblock_c(int m) { return 4 * T + 2 * m; }
constexpr int NPEN_BLOCKS = 1024;  // most blocks of the loss statistics of one instance

// Double-float sums: an FP32 pair hi + lo carries about 48 significant bits.  FP64
// arithmetic is slow on this part, and the reductions below sit on the critical path of
// every iteration, so they add double-floats in fixed orders instead.
struct DF {
    float hi, lo;
};

// a + b exactly as hi + lo (Knuth's two-sum; no ordering of |a|, |b| needed); commutative
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    const DF s = df_two_sum(a.hi, b.hi);
    const float lo = s.lo + (a.lo + b.lo);
    const float hi = s.hi + lo;
    return {hi, lo - (hi - s.hi)};
}

// fixed-order sum over the block (blockDim.x a multiple of 32, <= 1024): xor butterflies in
// each warp, then over the warp results in warp 0; the result is valid in thread 0.  sh holds
// 32 entries.
__device__ __forceinline__ DF block_sum_df(DF v, DF* sh) {
    for (int o = 16; o > 0; o >>= 1)
        v = df_add(v, DF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();   // sh may still be read by a previous call
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? sh[lane] : DF{0.f, 0.f};
        for (int o = 16; o > 0; o >>= 1)
            v = df_add(v, DF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
    }
    return v;
}
constexpr int MAX_DYN_SMEM = 200 * 1024;   // dynamic shared memory limit of the correlation kernels
constexpr int MAX_PHASES = 8;      // phase fields of one problem (their ordered pairs each get a block)

// One multigrid level, every field handled as 3-D (2-D fields have n[0] = 1, P[0] = 0).
struct LevelGeom {
    int64_t n[3];
    int64_t N;
    int P[3];
    int NB;           // rx blocks of T covering [-P2, P2]
    int64_t NG;       // shift groups (rz, ry, b) of the half window
    int64_t Khalf;
    int64_t NGT;      // NG * T (columns of one forward partial row)
    // forward tiling
    int TY;           // tile rows
    int PPB;          // planes per block
    int tilesY, tilesX, planeChunks;
    int64_t fwdTiles; // planeChunks * tilesY * tilesX
    int fwdGroupBlocks;
    // adjoint tiling
    int adjTilesY, adjTilesX;
    int64_t adjTiles;  // n[0] * adjTilesY * adjTilesX
    int nZc, nYc, RZ, RY;   // shift chunks over rz and ry
    int RYS;                // ry rows staged in shared memory at a time (RY may be larger: rounds)
    int nXc, NBc;           // shift chunks over the rx blocks: NBc blocks of T per chunk
    int nChunks;
    int fft;          // 1: this level runs on the FFT path (identity threshold / binary target)
};

// Soft-threshold constants in the product form used on the device:
//   P = E'_x E_y,  E_y = 2^(-kappa M_y),  E'_x = 2^(cexp - kappa M_x)
//   s = 1/(1+P) = sigma(alpha (a - 0.75)),  f = c1 s + c3.
struct ThreshConst {
    float kappa;     // (alpha/2) log2(e)
    float cexp;      // 0.75 alpha log2(e)
    float c1, c3;
    float alpha;
    float lim;       // product form when |kappa M| <= lim everywhere in a block
    float beta;      // c3 / c1: f = c1 (s + beta)
    int identity;    // f(x) = x
};

struct LossParams {
    int mode;           // 0 norm, 1 squared
    float lambda0;
    int bc_on;
    int64_t Ktot;
    int64_t N;          // finest pixel count
    float tol_rel;      // <=0: no stopping test
    int check_every;
    float lr, beta1, beta2;
    int max_iters;
    int recon;          // 1: update iteration / Adam bookkeeping
};

struct FinalArgs {
    int ndim;
    int levels;
    int64_t n1[3];               // finest sizes (3-D embedded)
    const float* parts[8];       // adjoint partials per level
    int nChunks[8];
    int64_t Nl[8];
    int64_t nl[8][3];
    const float* field;          // finest field (penalty), may be null when no penalty
    const Scalars* sc;           // pen_coef (null: no penalty)
    float* grad_out;             // may be null
    float* M;                    // Adam: field to update (null: no Adam)
    float* m;
    float* v;
    float beta1, beta2, eps;
};

// ---------------------------------------------------------------- segment tables
// A fused launch covers several (instance, level) segments; every segment owns the
// contiguous block range [blockStart, next blockStart) of a 1-D grid and the kernels find
// their segment by binary search.  Tables live in device memory (written by blob_kernel).
struct FwdSeg {
    LevelGeom g;
    const float* field;     // tails of the pairs (x)
    const float* tip;       // tips of the pairs (x + r): the same field, or another phase's
    float* partial;
    const int* done;
    int64_t blockStart;
};
struct RedSeg {
    LevelGeom g;
    const float* partial;
    float* desc;
    const int* done;
    float scale;             // w_l / N_l
    int64_t blockStart;
};
struct AdjSeg {
    LevelGeom g;
    const float* field;     // own positions y (the gradient's field)
    const float* tip;       // partners y + r: the same field, or another phase's
    const float* Gd;
    float* part;
    const int* done;
    int64_t blockStart;
};
struct GSeg {
    LevelGeom g;
    const float* src;       // dL/dS (or S - S_des) of the block (a, b), shifts r of the half window
    const float* sub;
    const float* src2;      // the block (b, a), which holds -r; src2 = src, sub2 = sub for a = b
    const float* sub2;
    const Scalars* sc;
    float scale;
    float* Gd;
    const int* done;
    const float* tsum;      // corrected descriptor: sum_{k >= 1} (src - sub) of the block, else null
    float q;                // corrected descriptor: 2 f(1/2)^2
    int64_t blockStart;
};
// Corrected two-point descriptor (App. A, Eq. s2rfroms2rbar), one (instance, level) block:
// forward, the block is mapped in place, S_tilde(k) = (S_bar(k) - q S_bar(0)) / (1 - q) for
// k >= 1; backward, tsum = sum_{k >= 1} (src - sub) feeds the transposed map in gcoef.
struct TildeSeg {
    float* desc;
    const float* src;
    const float* sub;
    float* tsum;
    int64_t K;
    float q;
    const int* done;
    int64_t blockStart;
};
struct RestrictSeg {
    int ndim;
    int64_t c[3];               // coarse sizes (3-D embedded)
    const float* fine;
    float* coarse;
    const int* done;
    int64_t blockStart;
};
struct PenSeg {
    const float* field;      // null: no box penalty
    int64_t N;
    const float* desc;
    const float* target;
    int64_t K;
    double* partials;        // 3 x nblk
    const int* done;
    int nblk;                // blocks of this instance: a function of its own sizes only
};
struct LossSeg {
    LossParams lp;
    const float* desc;
    const float* target;
    const double* pen;
    int nblk;
    Scalars* sc;
    float* loss_out;
    float* history;
};
struct FinalSeg {
    FinalArgs a;
    const int* done;
    int64_t blockStart;
};
struct InitSeg {
    Scalars* sc;
    int64_t step;
    double b1t, b2t;
};

// Three-point descriptor, one (instance, level) (gram.cu).  K = half-window shifts, Kpad =
// K rounded up to 256, Npad = the level's position count rounded up to 128.
struct S3Job {
    LevelGeom g;
    const float* field;     // this level's field
    int64_t K, Kpad, Npad;
    // GEMM operands as FP16 bit patterns: x s = hi + lo (hi = fp16(x s), lo = fp16(x s - hi)),
    // s a power of two that brings max |x| into [1/2, 1) (E: f(x) = x only; G: always)
    uint16_t *Eh, *El;      // E (Npad x Kpad)
    uint16_t *Eth, *Etl;    // E^T (Kpad x Npad)
    float* W;               // W^T (Kpad x Npad)
    uint16_t *Gh, *Gl;      // G (Kpad x Kpad)
    float* amax;            // [0] max |G|, [1] max |field| (f(x) = x): the scales' sources
    float* desc;            // this level's K x K block of the descriptor (w * S_bar3)
    const float* src;       // G = weight * (sc ? gscale : 1) * (src - sub): src = desc (loss) or
    const float* sub;       //   the upstream gradient (VJP, sub = null, sc = null)
    const Scalars* sc;
    float weight;
    float* part;            // this level's gradient
    const int* done;
    int ens;                // backward: build E first (no forward ran in this call)
    int* err;               // set on a tensor-core wait timeout
};

// One mixed-radix Stockham pass over the lines of one axis (fft.cu).
struct FftPass {
    double2* data;            // complex grid, transformed in place
    const float* real_in;     // non-null: read the real input from here instead of `data`
    int64_t n[3];
    int axis;                 // 0, 1, 2
    int sign;                 // -1 forward, +1 inverse (unnormalised)
    int len;                  // n[axis]
    int L;                    // lines per block
    int nrad;
    int rad[16];
    const double2* tw;        // tw[t] = exp(-2 pi i t / len)
    double2 om3[3], om5[5];   // exp(-2 pi i t / 3), exp(-2 pi i t / 5)
};

// ---------------------------------------------------------------- launchers
void launch_blob(const void* host, size_t bytes, void* dst, cudaStream_t s);
void launch_restrict(const RestrictSeg* segs, int nseg, int64_t blocks, cudaStream_t s);
void launch_restrict_one(int ndim, const int64_t nf[3], const float* fine, float* coarse, cudaStream_t s);
void launch_prolongate(int ndim, const int64_t nc[3], const float* coarse, float* fine, int mode,
                       cudaStream_t s);
void launch_corr_fwd(const FwdSeg* segs, int nseg, int64_t blocks, size_t smem, const ThreshConst& tc,
                     cudaStream_t s);
void launch_fwd_reduce(const RedSeg* segs, int nseg, int64_t blocks, cudaStream_t s);
void launch_penalty(const PenSeg* segs, int nseg, int maxblk, cudaStream_t s);
int stats_blocks(int64_t K, int64_t N);
void launch_loss(const LossSeg* segs, int nseg, cudaStream_t s);
void launch_gcoef(const GSeg* segs, int nseg, int64_t blocks, const ThreshConst& tc, cudaStream_t s);
void launch_tilde_map(const TildeSeg* segs, int nseg, int64_t blocks, cudaStream_t s);
void launch_tilde_sum(const TildeSeg* segs, int nseg, cudaStream_t s);
void launch_corr_adj(const AdjSeg* segs, int nseg, int64_t blocks, size_t smem, const ThreshConst& tc,
                     cudaStream_t s);
// sub = threads per position: 1, or FIN_SUB for segments of fields below FIN_SUB_BELOW positions
void launch_final(const FinalSeg* segs, int nseg, int64_t blocks, int sub, cudaStream_t s);
void launch_init_uniform(float* field, int64_t count, uint64_t seed, cudaStream_t s);
void launch_round_field(const float* src, float* dst, int64_t count, cudaStream_t s);
void launch_scalars_init(const InitSeg* segs, int nseg, cudaStream_t s);
void launch_scalars_set(const InitSeg* host_segs, int nseg, cudaStream_t s);   // segments by value
void set_kernel_attributes();
void set_gram_attributes();
size_t gemm_smem_bytes();
bool gram_ready();   // the TMA tensor-map encoder is available
void launch_s3_forward(const S3Job& j, const ThreshConst& tc, int* err, cudaStream_t s);
void launch_s3_backward(const S3Job& j, const ThreshConst& tc, int* err, cudaStream_t s);
void set_fft_attributes();
size_t fft_smem_bytes(int len, int L);
int fft_lines_per_block(int len);
void launch_fft_pass(const FftPass& p, cudaStream_t s);
void launch_fft_twiddles(double2* tw, int len, cudaStream_t s);
void launch_fft_power(const double2* X, double2* P, int64_t N, cudaStream_t s);
void launch_fft_xcorr(const double2* X, double2* H, int64_t N, cudaStream_t s);
void launch_fft_sample(const LevelGeom& g, const double2* X, float weight, int mode, double fh2, float* desc,
                       cudaStream_t s);
void launch_fft_embed(const LevelGeom& g, const float* Gd, double2* H, cudaStream_t s);
void launch_fft_dc(const double2* H, double* out, cudaStream_t s);
void launch_fft_vjp_combine(int64_t N, const float* M, const double2* Z, const double* sumA, float* part,
                            cudaStream_t s);
size_t fwd_smem_bytes(const LevelGeom& g);
size_t adj_smem_bytes(const LevelGeom& g);
float gcoef_scale(const LevelGeom& g, const ThreshConst& tc, float weight);

constexpr int RED_K = 32;      // shifts per fwd_reduce block
constexpr int GCOEF_TH = 256;  // entries per gcoef block
constexpr int ELEM_TH = 256;   // pixels per restrict block; threads per final block
constexpr int FIN_SUB = 4;     // gradient assembly of a small field: threads per position (each sums
                               // every 4th chunk; the combine adds exactly four partials)
constexpr int64_t FIN_SUB_BELOW = 1 << 16;   // fields of fewer positions use FIN_SUB threads each

// Segment of linear block b: the last segment whose blockStart <= b.
template <typename S>
__device__ __forceinline__ int find_segment(const S* __restrict__ segs, int nseg, int64_t b) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].blockStart <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace dmcr
