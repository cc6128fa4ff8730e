// Memory-bound kernels around the correlation: multigrid restriction / prolongation
// (Sec. 3.3), the box-penalty reduction and the loss (Sec. 3.1, Eq. L_func_dMCR), the
// fused gradient assembly + Adam update (Eq. M-update, App. B) and the counter-based
// uniform start field.  All reductions use fixed grids and fixed summation orders, so
// every result is bitwise reproducible run to run.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace dmcr {

// --------------------------------------------------------------------- multigrid

// coarse[c] = mean of the 2^d children of c (children summed in a fixed order).
__device__ __forceinline__ void restrict_one(int ndim, int64_t c0, int64_t c1, int64_t c2, const float* __restrict__ fine,
                                             float* __restrict__ coarse, int64_t i) {
    const int64_t x = i % c2, y = (i / c2) % c1, z = i / (c1 * c2);
    const int64_t f1 = 2 * c1, f2 = 2 * c2;
    float s;
    if (ndim == 2) {
        const float* r0 = fine + (2 * y) * f2 + 2 * x;
        const float* r1 = r0 + f2;
        s = ((r0[0] + r0[1]) + (r1[0] + r1[1])) * 0.25f;
    } else {
        const float* p0 = fine + ((2 * z) * f1 + 2 * y) * f2 + 2 * x;
        const float* p1 = p0 + f1 * f2;
        s = (((p0[0] + p0[1]) + (p0[f2] + p0[f2 + 1])) + ((p1[0] + p1[1]) + (p1[f2] + p1[f2 + 1]))) * 0.125f;
    }
    coarse[i] = s;
}

__global__ void restrict_kernel(const RestrictSeg* __restrict__ segs, int nseg) {
    const int si = find_segment(segs, nseg, (int64_t)blockIdx.x);
    const RestrictSeg& sg = segs[si];
    if (sg.done != nullptr && *sg.done) return;
    const int64_t i = ((int64_t)blockIdx.x - sg.blockStart) * ELEM_TH + threadIdx.x;
    if (i >= sg.c[0] * sg.c[1] * sg.c[2]) return;
    restrict_one(sg.ndim, sg.c[0], sg.c[1], sg.c[2], sg.fine, sg.coarse, i);
}

__global__ void restrict_plain_kernel(int ndim, int64_t c0, int64_t c1, int64_t c2, const float* __restrict__ fine,
                                      float* __restrict__ coarse) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c0 * c1 * c2) return;
    restrict_one(ndim, c0, c1, c2, fine, coarse, i);
}

void launch_restrict(const RestrictSeg* segs, int nseg, int64_t blocks, cudaStream_t s) {
    if (blocks <= 0) return;
    restrict_kernel<<<(unsigned)blocks, ELEM_TH, 0, s>>>(segs, nseg);
}

void launch_restrict_one(int ndim, const int64_t nf[3], const float* fine, float* coarse, cudaStream_t s) {
    const int64_t c0 = (ndim == 2) ? 1 : nf[0] / 2;
    const int64_t c1 = nf[1] / 2, c2 = nf[2] / 2;
    const int64_t Nc = c0 * c1 * c2;
    restrict_plain_kernel<<<(unsigned)((Nc + ELEM_TH - 1) / ELEM_TH), ELEM_TH, 0, s>>>(ndim, c0, c1, c2, fine, coarse);
}

// fine[f] += coarse[parent(f)] / 2^d   (transpose of restrict)   or   fine[f] = coarse[parent(f)]
__global__ void prolongate_kernel(int ndim, int64_t c0, int64_t c1, int64_t c2, const float* __restrict__ coarse,
                                  float* __restrict__ fine, int mode) {
    const int64_t f0 = (ndim == 2) ? 1 : 2 * c0, f1 = 2 * c1, f2 = 2 * c2;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= f0 * f1 * f2) return;
    const int64_t x = i % f2, y = (i / f2) % f1, z = i / (f1 * f2);
    const int64_t pz = (ndim == 2) ? 0 : z / 2;
    const float v = coarse[(pz * c1 + y / 2) * c2 + x / 2];
    if (mode == 1) fine[i] = v;
    else fine[i] += v * (ndim == 2 ? 0.25f : 0.125f);
}

void launch_prolongate(int ndim, const int64_t nc[3], const float* coarse, float* fine, int mode, cudaStream_t s) {
    const int64_t c0 = (ndim == 2) ? 1 : nc[0];
    const int64_t Nf = (ndim == 2 ? 4 : 8) * c0 * nc[1] * nc[2];
    const int th = 256;
    prolongate_kernel<<<(unsigned)((Nf + th - 1) / th), th, 0, s>>>(ndim, c0, nc[1], nc[2], coarse, fine, mode);
}

// --------------------------------------------------------------------- loss

// Box excess of Sec. 3.1: (M-1) H(M-1) - M H(-M), H(0) = 0.
__device__ __forceinline__ float box_excess(float M) {
    return M > 1.f ? M - 1.f : (M < 0.f ? -M : 0.f);
}

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
    // fixed-order tree over the block (blockDim.x a power of two <= 1024)
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// grid (max nblk, instances): double-float partial sums of one loss evaluation over the
// instance's own nblk blocks (a fixed grid per problem size) -- sum (D - D_des)^2 and
// sum D_des^2 over the descriptor, and sum ex^2 of the box excess over the field (when the
// penalty is on).
// partials[3 b + {0, 1, 2}] for block b.
__global__ void stats_kernel(const PenSeg* __restrict__ segs) {
    const PenSeg& sg = segs[blockIdx.y];
    if (sg.done != nullptr && *sg.done) return;
    if ((int)blockIdx.x >= sg.nblk) return;
    __shared__ DF sh[32];
    const int64_t stride = (int64_t)sg.nblk * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // per-thread compensated (Kahan) FP32 sums in a fixed order -- FP64 arithmetic is slow on
    // this part and a thread sums only about 8 terms (stats_blocks) -- then a double-float
    // (two-sum) tree across the block
    float r2 = 0.f, r2c = 0.f, t2 = 0.f, t2c = 0.f, e2 = 0.f, e2c = 0.f;
    auto kahan = [](float& sum, float& comp, float v) {
        const float y = v - comp;
        const float t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    };
    // the terms of this thread in order; their loads issued four at a time (the same sums)
    int64_t k = i0;
    for (; k + 3 * stride < sg.K; k += 4 * stride) {
        float tv[4], dv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            tv[u] = sg.target[k + u * stride];
            dv[u] = sg.desc[k + u * stride];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float r = dv[u] - tv[u];
            kahan(r2, r2c, r * r);
            kahan(t2, t2c, tv[u] * tv[u]);
        }
    }
    for (; k < sg.K; k += stride) {
        const float t = sg.target[k];
        const float r = sg.desc[k] - t;
        kahan(r2, r2c, r * r);
        kahan(t2, t2c, t * t);
    }
    if (sg.field != nullptr) {
        int64_t i = i0;
        for (; i + 3 * stride < sg.N; i += 4 * stride) {
            float fv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) fv[u] = sg.field[i + u * stride];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float e = box_excess(fv[u]);
                kahan(e2, e2c, e * e);
            }
        }
        for (; i < sg.N; i += stride) {
            const float e = box_excess(sg.field[i]);
            kahan(e2, e2c, e * e);
        }
    }
    // Kahan's (sum, comp) stands for sum - comp
    const DF R2 = block_sum_df(df_two_sum(r2, -r2c), sh);
    const DF T2 = block_sum_df(df_two_sum(t2, -t2c), sh);
    const DF E2 = block_sum_df(df_two_sum(e2, -e2c), sh);
    if (threadIdx.x == 0) {
        float2* part = reinterpret_cast<float2*>(sg.partials);
        part[3 * blockIdx.x + 0] = make_float2(R2.hi, R2.lo);
        part[3 * blockIdx.x + 1] = make_float2(T2.hi, T2.lo);
        part[3 * blockIdx.x + 2] = make_float2(E2.hi, E2.lo);
    }
}

void launch_penalty(const PenSeg* segs, int nseg, int maxblk, cudaStream_t s) {
    if (nseg <= 0) return;
    stats_kernel<<<dim3(maxblk, nseg), 256, 0, s>>>(segs);
}

// blocks of the loss statistics: about 2048 terms per block, 256 .. NPEN_BLOCKS, a power of two
int stats_blocks(int64_t K, int64_t N) {
    const int64_t work = K > N ? K : N;
    int b = 256;
    while (b < NPEN_BLOCKS && (int64_t)b * 2048 < work) b *= 2;
    return b;
}

// Corrected two-point descriptor, forward: map every block in place (entry 0 is read, never
// written, so the map needs no second buffer).
__global__ void tilde_map_kernel(const TildeSeg* __restrict__ segs, int nseg) {
    const int si = find_segment(segs, nseg, (int64_t)blockIdx.x);
    const TildeSeg& sg = segs[si];
    if (sg.done != nullptr && *sg.done) return;
    const int64_t k = ((int64_t)blockIdx.x - sg.blockStart) * ELEM_TH + threadIdx.x;
    if (k < 1 || k >= sg.K) return;
    sg.desc[k] = (sg.desc[k] - sg.q * sg.desc[0]) / (1.f - sg.q);
}

void launch_tilde_map(const TildeSeg* segs, int nseg, int64_t blocks, cudaStream_t s) {
    if (blocks <= 0) return;
    tilde_map_kernel<<<(unsigned)blocks, ELEM_TH, 0, s>>>(segs, nseg);
}

// Corrected two-point descriptor, backward: one block per segment, sum_{k >= 1} (src - sub)
// in FP64 in a fixed order.
__global__ void tilde_sum_kernel(const TildeSeg* __restrict__ segs) {
    const TildeSeg& sg = segs[blockIdx.x];
    if (sg.done != nullptr && *sg.done) return;
    __shared__ double sh[256];
    double acc = 0.0;
    for (int64_t k = 1 + threadIdx.x; k < sg.K; k += blockDim.x)
        acc += (double)sg.src[k] - (sg.sub != nullptr ? (double)sg.sub[k] : 0.0);
    acc = block_sum_d(acc, sh);
    if (threadIdx.x == 0) *sg.tsum = (float)acc;
}

void launch_tilde_sum(const TildeSeg* segs, int nseg, cudaStream_t s) {
    if (nseg <= 0) return;
    tilde_sum_kernel<<<nseg, 256, 0, s>>>(segs);
}

// One block per instance: sums the stats partials in a fixed tree, then E, E^2, E_bc,
// lambda, L, rel_err and the gradient scalars; in a reconstruction also the stopping test
// and the Adam step bookkeeping.
__global__ void __launch_bounds__(NPEN_BLOCKS) loss_kernel(const LossSeg* __restrict__ segs) {
    const LossSeg& sg = segs[blockIdx.x];
    const LossParams lp = sg.lp;
    const double* __restrict__ pen = sg.pen;
    Scalars* sc = sg.sc;
    float* loss_out = sg.loss_out;
    float* history = sg.history;
    if (lp.recon && sc->done) return;
    __shared__ DF sh[32];
    // the instance's nblk double-float partials (the remaining threads add zeros)
    const int b = threadIdx.x;
    const float2* part = reinterpret_cast<const float2*>(pen);
    const DF zero{0.f, 0.f};
    auto get = [&](int q) { return b < sg.nblk ? DF{part[3 * b + q].x, part[3 * b + q].y} : zero; };
    const DF e2s = block_sum_df(get(0), sh);
    const DF t2s = block_sum_df(get(1), sh);
    const DF x2s = block_sum_df(get(2), sh);
    if (threadIdx.x != 0) return;
    // the scalars in FP64 on this one thread (a few dozen FP64 operations once per
    // evaluation): the double-float sums keep about 48 bits, and the square roots and
    // quotients below keep them, so E, rel_err and L reach the output rounded once to FP32
    const double E2 = (double)e2s.hi + (double)e2s.lo;
    const double T2 = (double)t2s.hi + (double)t2s.lo;
    const double ex2 = (double)x2s.hi + (double)x2s.lo;
    const double N = (double)lp.N;
    const double lam0 = lp.bc_on ? (double)lp.lambda0 : 0.0;
    const double E = sqrt(E2);
    const double Ebc = ex2 / (N * N);
    const double phi = lp.mode == 0 ? E : E2;
    const double lam = lam0 * phi;
    const double L = phi + lam * Ebc;
    const double rel = T2 > 0.0 ? E / sqrt(T2) : (double)INFINITY;
    const float out[6] = {(float)E, (float)E2, (float)Ebc, (float)lam, (float)L, (float)rel};
    for (int i = 0; i < 6; ++i) sc->loss[i] = out[i];
    if (loss_out != nullptr)
        for (int i = 0; i < 6; ++i) loss_out[i] = out[i];
    // dL/dD = phi'(E) (1 + lam0 E_bc) dE/dD ;  dL/dM (penalty) = lam0 phi dE_bc/dM
    double gs;
    if (lp.mode == 0) gs = E > 0.0 ? (1.0 + lam0 * Ebc) / E : 0.0;
    else gs = 2.0 * (1.0 + lam0 * Ebc);
    sc->gscale = (float)gs;
    sc->pen_coef = (float)(2.0 * lam0 * phi / (N * N));
    if (!lp.recon) return;
    const int it = sc->iter;
    if (history != nullptr && it < lp.max_iters) {
        history[3 * it + 0] = out[0];
        history[3 * it + 1] = out[4];
        history[3 * it + 2] = out[5];
    }
    sc->iter = it + 1;
    if (!isfinite(out[4])) { sc->done = 2; return; }
    if (lp.tol_rel > 0.f && (it % lp.check_every) == 0 && out[5] < lp.tol_rel) { sc->done = 1; return; }
    if (it + 1 > lp.max_iters) { sc->done = 3; return; }
    sc->adam_step = sc->adam_step + 1;
    // beta^t products stay FP64: they are multiplied once per step over many steps
    const double b1t = sc->b1t * (double)lp.beta1;
    const double b2t = sc->b2t * (double)lp.beta2;
    sc->b1t = b1t;
    sc->b2t = b2t;
    sc->lr_t = (float)((double)lp.lr * sqrt(1.0 - b2t) / (1.0 - b1t));
}

void launch_loss(const LossSeg* segs, int nseg, cudaStream_t s) {
    if (nseg <= 0) return;
    loss_kernel<<<nseg, NPEN_BLOCKS, 0, s>>>(segs);
}

// --------------------------------------------------------------------- gradient + Adam

// g(y) = sum_l 2^{-d(l-1)} sum_chunks part_l[chunk][ancestor_l(y)]  (+ penalty gradient),
// then either written out, or used for one Adam step (Keras form) on the field.  Position i's
// chunk sums for the chunks c = q (mod SUB) of every level, each level's chunks in order,
// their loads issued eight at a time.
template <int SUB>
__device__ __forceinline__ float chunk_sums(const FinalArgs& a, int64_t i, int q) {
    const int64_t x = i % a.n1[2], y = (i / a.n1[2]) % a.n1[1], z = i / (a.n1[1] * a.n1[2]);
    float g = 0.f, scale = 1.f;
    const float step = a.ndim == 2 ? 0.25f : 0.125f;
    for (int l = 0; l < a.levels; ++l) {
        const int64_t lz = a.ndim == 2 ? 0 : (z >> l);
        const int64_t li = (lz * a.nl[l][1] + (y >> l)) * a.nl[l][2] + (x >> l);
        const int64_t jump = SUB * a.Nl[l];
        const float* p = a.parts[l] + li + q * a.Nl[l];
        const int nc = a.nChunks[l];
        float s = 0.f;
        int c = q;
        for (; c + 7 * SUB < nc; c += 8 * SUB) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u, p += jump) v[u] = *p;
#pragma unroll
            for (int u = 0; u < 8; ++u) s += v[u];
        }
        for (; c < nc; c += SUB, p += jump) s += *p;
        g = fmaf(scale, s, g);
        scale *= step;
    }
    return g;
}

// A block covers ELEM_TH / SUB positions with SUB threads each.  SUB = 1 (a large field):
// one thread per position, a warp reads 32 consecutive positions of a chunk.  SUB = FIN_SUB
// (a small field: few positions for many chunk partials): thread (q, p) -- q = threadIdx.x /
// positions, so a warp still reads consecutive positions of one chunk -- sums the chunks
// c = q (mod FIN_SUB) and the FIN_SUB partials are added in a fixed order through shared
// memory.  Two instantiations, so that SUB = 1 keeps the 32 registers with which 8 blocks
// stay resident per SM (a 512^2 field is one wave).
template <int SUB>
__global__ void __launch_bounds__(ELEM_TH) final_kernel(const FinalSeg* __restrict__ segs, int nseg) {
    const int si = find_segment(segs, nseg, (int64_t)blockIdx.x);
    const FinalSeg& sg = segs[si];
    if (sg.done != nullptr && *sg.done) return;
    const FinalArgs& a = sg.a;
    const int64_t N1 = a.n1[0] * a.n1[1] * a.n1[2];
    const int64_t b = (int64_t)blockIdx.x - sg.blockStart;
    int64_t i;
    float g;
    if constexpr (SUB == 1) {
        i = b * ELEM_TH + threadIdx.x;
        if (i >= N1) return;
        g = chunk_sums<1>(a, i, 0);
    } else {
        static_assert(SUB == 4, "the combine below adds four partials");
        constexpr int NPOS = ELEM_TH / SUB;
        __shared__ float part[SUB][NPOS];
        const int q = threadIdx.x / NPOS, pl = threadIdx.x % NPOS;
        i = b * NPOS + pl;
        const bool valid = i < N1;
        part[q][pl] = valid ? chunk_sums<SUB>(a, i, q) : 0.f;
        __syncthreads();
        if (q != 0 || !valid) return;
        g = (part[0][pl] + part[1][pl]) + (part[2][pl] + part[3][pl]);
    }
    if (a.sc != nullptr && a.field != nullptr) {
        const float M = a.field[i];
        const float ex = box_excess(M);
        const float dex = M > 1.f ? 1.f : (M < 0.f ? -1.f : 0.f);
        g = fmaf(a.sc->pen_coef * ex, dex, g);
    }
    if (a.grad_out != nullptr) a.grad_out[i] = g;
    if (a.M != nullptr) {
        const float m = fmaf(a.beta1, a.m[i], (1.f - a.beta1) * g);
        const float v = fmaf(a.beta2, a.v[i], (1.f - a.beta2) * g * g);
        a.m[i] = m;
        a.v[i] = v;
        a.M[i] = a.M[i] - a.sc->lr_t * m / (sqrtf(v) + a.eps);
    }
}

void launch_final(const FinalSeg* segs, int nseg, int64_t blocks, int sub, cudaStream_t s) {
    if (blocks <= 0) return;
    if (sub == 1)
        final_kernel<1><<<(unsigned)blocks, ELEM_TH, 0, s>>>(segs, nseg);
    else
        final_kernel<FIN_SUB><<<(unsigned)blocks, ELEM_TH, 0, s>>>(segs, nseg);
}

__device__ __forceinline__ void scalars_init_one(const InitSeg& g) {
    Scalars* sc = g.sc;
    for (int k = 0; k < 6; ++k) sc->loss[k] = 0.f;
    sc->gscale = 0.f;
    sc->pen_coef = 0.f;
    sc->lr_t = 0.f;
    sc->done = 0;
    sc->iter = 0;
    sc->adam_step = g.step;
    sc->b1t = g.b1t;
    sc->b2t = g.b2t;
    sc->err = 0;
}

__global__ void scalars_init_kernel(const InitSeg* __restrict__ segs, int nseg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nseg) return;
    scalars_init_one(segs[i]);
}

void launch_scalars_init(const InitSeg* segs, int nseg, cudaStream_t s) {
    if (nseg <= 0) return;
    scalars_init_kernel<<<(nseg + 127) / 128, 128, 0, s>>>(segs, nseg);
}

// The same initialisation with the segments passed by value (no table in device memory):
// used before a replay of a cached iteration graph, whose captured tables cannot carry the
// Adam step count of the current call.
constexpr int SET_MAX = 960;
struct InitBatch {
    int n;
    InitSeg seg[SET_MAX];
};

__global__ void scalars_set_kernel(const InitBatch b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.n) return;
    scalars_init_one(b.seg[i]);
}

void launch_scalars_set(const InitSeg* segs, int nseg, cudaStream_t s) {
    static thread_local InitBatch b;
    for (int off = 0; off < nseg; off += SET_MAX) {
        const int k = nseg - off < SET_MAX ? nseg - off : SET_MAX;
        b.n = k;
        memcpy(b.seg, segs + off, (size_t)k * sizeof(InitSeg));
        scalars_set_kernel<<<(k + 127) / 128, 128, 0, s>>>(b);
    }
}

// Writes up to BLOB_BYTES of host data, passed by value as a kernel parameter, to device
// memory: stream ordered, no host synchronisation, and valid inside a graph capture.
constexpr int BLOB_BYTES = 30720;
struct Blob {
    unsigned int words;
    unsigned int data[BLOB_BYTES / 4];
};

__global__ void blob_kernel(const Blob b, unsigned int* __restrict__ dst) {
    for (unsigned int i = threadIdx.x; i < b.words; i += blockDim.x) dst[i] = b.data[i];
}

void launch_blob(const void* host, size_t bytes, void* dst, cudaStream_t s) {
    const unsigned char* src = static_cast<const unsigned char*>(host);
    unsigned char* out = static_cast<unsigned char*>(dst);
    size_t off = 0;
    static thread_local Blob b;
    while (off < bytes) {
        const size_t n = bytes - off < (size_t)BLOB_BYTES ? bytes - off : (size_t)BLOB_BYTES;
        const size_t words = (n + 3) / 4;
        memset(b.data, 0, words * 4);
        memcpy(b.data, src + off, n);
        b.words = (unsigned int)words;
        blob_kernel<<<1, 256, 0, s>>>(b, reinterpret_cast<unsigned int*>(out + off));
        off += words * 4;
    }
}

// --------------------------------------------------------------------- start field

// SplitMix64 (Steele, Lea & Flood 2014): state seed + (i+1) * golden gamma, then the
// published three-step mix; value = top 24 bits * 2^-24.
__global__ void init_uniform_kernel(float* __restrict__ f, int64_t count, uint64_t seed) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    f[i] = (float)(z >> 40) * (1.0f / 16777216.0f);
}

void launch_init_uniform(float* field, int64_t count, uint64_t seed, cudaStream_t s) {
    const int th = 256;
    init_uniform_kernel<<<(unsigned)((count + th - 1) / th), th, 0, s>>>(field, count, seed);
}

// The rounded field used to evaluate a reconstruction (Sec. 4.1): values >= 1/2 become
// phase 1, the rest phase 0.
__global__ void round_field_kernel(const float* __restrict__ src, float* __restrict__ dst, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    dst[i] = src[i] >= 0.5f ? 1.f : 0.f;
}

void launch_round_field(const float* src, float* dst, int64_t count, cudaStream_t s) {
    if (count <= 0) return;
    const int th = 256;
    round_field_kernel<<<(unsigned)((count + th - 1) / th), th, 0, s>>>(src, dst, count);
}

}  // namespace dmcr
