// Direct correlation kernels of the soft-thresholded two-point descriptor and its adjoint
// (sm_103a).  Paper: arXiv 2103.09686, Sec. 3.2.2-3.2.4 (convolve -> threshold ->
// quadratic reduce) and the gradient of Sec. 3.1/3.3.
//
// Product form.  With kappa = (alpha/2) log2 e and cexp = 0.75 alpha log2 e, every pixel
// is mapped once to E_y = 2^(-kappa M_y) (tip side) and E'_x = 2^(cexp - kappa M_x)
// (tail side); a shifted pair then needs no exponential at all:
//     P = E'_x E_y = exp(-alpha (a - 0.75)),  a = (M_x + M_y)/2,
//     s = 1 / (1 + P) = sigma(alpha (a - 0.75)),   f(a) = c1 s + c3.
// One FFMA and one MUFU reciprocal per pair.  The pair (x, x+0) gives a = M_x, so r = 0
// needs no special case.  Blocks whose pixels leave |kappa M| <= lim take an exact slow
// path (P = 2^(cexp - kappa M_x - kappa M_y) per pair), so arbitrary finite fields are
// handled; the choice is block-uniform.
//
// Forward (half window).  A thread owns T = 8 consecutive rx shifts of one (rz, ry) and
// walks the positions of its block's tile; per 8-position chunk it reads 8 tail values
// (broadcast) and 16 tip values (4 x LDS.128) and evaluates 64 pairs.  Consecutive lanes
// own consecutive ry, i.e. consecutive shared-memory rows whose stride is 4 mod 32 words,
// so the LDS.128 reads are bank-conflict free.  Per-thread sums are hierarchical (row,
// plane, block) in FP32, written per tile and reduced across tiles in FP64 in fixed order:
// the result is deterministic.
//
// Adjoint (full window, gather form).  A thread owns 8 consecutive positions of one row;
// lanes own consecutive rows.  For every shift of its block's chunk it accumulates
//     g_y += G'(r) * h(a_y(r)),  h = f f' = c1 alpha s (1 - s) (c1 s + c3),
// with G'(r) = dL/dS_bar(|r|) / N (2 dL/dS_bar(0) / N at r = 0), recomputing every pair
// (the N x K ensemble is never stored).  No atomics; per-chunk partials are summed in a
// fixed order by the final kernel.
#include <algorithm>

#include "common.cuh"

namespace dmcr {

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int64_t wrapi(int64_t i, int64_t n) {
    int64_t m = i % n;
    return m < 0 ? m + n : m;
}

// v mod n for v within a few periods of [0, n) (the halos reach at most one window past a tile)
__device__ __forceinline__ int64_t wrap1(int64_t v, int64_t n) {
    while (v < 0) v += n;
    while (v >= n) v -= n;
    return v;
}

__host__ __device__ inline int stride_4mod32(int cols) {
    // smallest s >= cols with s % 32 == 4
    int s = ((cols - 4 + 31) / 32) * 32 + 4;
    return s < 4 ? 4 : s;
}

// Group gi of the half window -> (rz, ry, b); order: rz, then b, then ry fastest.
__host__ __device__ inline void decode_group(const LevelGeom& g, int64_t gi, int& rz, int& ry, int& b) {
    const int64_t n0 = (int64_t)(g.P[1] + 1) * g.NB;
    if (gi < n0) {
        rz = 0;
        b = (int)(gi / (g.P[1] + 1));
        ry = (int)(gi % (g.P[1] + 1));
    } else {
        const int64_t w = 2 * g.P[1] + 1;
        const int64_t r = gi - n0;
        const int64_t per = w * g.NB;
        rz = 1 + (int)(r / per);
        const int64_t rem = r % per;
        b = (int)(rem / w);
        ry = (int)(rem % w) - g.P[1];
    }
}

// Canonical half-window index of (rz, ry, rx), -1 if (rz, ry, rx) is not in the half window.
__host__ __device__ inline int64_t canon_index(const LevelGeom& g, int rz, int ry, int rx) {
    const int Px = g.P[2], Py = g.P[1];
    if (rx < -Px || rx > Px) return -1;
    if (rz == 0 && ry == 0) return rx >= 0 ? rx : -1;
    if (rz == 0) return ry > 0 ? (Px + 1) + (int64_t)(ry - 1) * (2 * Px + 1) + (rx + Px) : -1;
    if (rz < 0) return -1;
    return (Px + 1) + (int64_t)Py * (2 * Px + 1) +
           ((int64_t)(rz - 1) * (2 * Py + 1) + (ry + Py)) * (2 * Px + 1) + (rx + Px);
}

// Block bounding box of the shift groups [gfirst, glast].
struct GroupBox {
    int rzA, rzB, rylo, ryhi, blo, bhi;
};

__host__ __device__ inline GroupBox group_box(const LevelGeom& g, int64_t gfirst, int64_t glast) {
    int rzA, ryA, bA, rzB, ryB, bB;
    decode_group(g, gfirst, rzA, ryA, bA);
    decode_group(g, glast, rzB, ryB, bB);
    GroupBox bx;
    bx.rzA = rzA;
    bx.rzB = rzB;
    if (rzA == rzB && bA == bB) {
        bx.rylo = ryA; bx.ryhi = ryB; bx.blo = bA; bx.bhi = bA;
    } else if (rzA == rzB) {
        bx.rylo = (rzA == 0) ? 0 : -g.P[1]; bx.ryhi = g.P[1]; bx.blo = bA; bx.bhi = bB;
    } else {
        bx.rylo = -g.P[1]; bx.ryhi = g.P[1]; bx.blo = 0; bx.bhi = g.NB - 1;
    }
    return bx;
}

struct FwdSmem {
    int planesH, rowsH, colsH, strideH;
};

__host__ __device__ inline FwdSmem fwd_smem_shape(const LevelGeom& g, const GroupBox& bx) {
    FwdSmem s;
    s.planesH = bx.rzB - bx.rzA + 1;
    s.rowsH = g.TY + bx.ryhi - bx.rylo;
    s.colsH = T * (bx.bhi - bx.blo) + TX + T;
    s.strideH = stride_4mod32(s.colsH);
    return s;
}

// ------------------------------------------------------------------------- pair math

enum { MODE_FAST = 0, MODE_SLOW = 1, MODE_IDENT = 2 };

// 64 pairs of one chunk: tails x[0..8), tips y[0..16); pair (k, m) uses y[k+m].
template <int MODE>
__device__ __forceinline__ void fwd_chunk(const float (&x)[T], const float (&y)[2 * T], float (&r1)[T],
                                          float (&r2)[T]) {
#pragma unroll
    for (int k = 0; k < T; ++k) {
        if (MODE == MODE_FAST) {
            // two pairs per reciprocal: s_a = d_b / (d_a d_b), s_b = d_a / (d_a d_b); on the fast
            // path every d <= 2^62, so d_a d_b stays finite (d >= 1 always)
#pragma unroll
            for (int m = 0; m < T / 2; ++m) {
                const float da = fmaf(x[k], y[k + m], 1.0f);
                const float db = fmaf(x[k], y[k + m + T / 2], 1.0f);
                const float r = rcp_approx(da * db);
                const float sa = db * r, sb = da * r;
                r1[m] += sa;
                r2[m] = fmaf(sa, sa, r2[m]);
                r1[m + T / 2] += sb;
                r2[m + T / 2] = fmaf(sb, sb, r2[m + T / 2]);
            }
        } else {
#pragma unroll
            for (int m = 0; m < T; ++m) {
                if (MODE == MODE_IDENT) {
                    const float a = x[k] + y[k + m];
                    r2[m] = fmaf(a, a, r2[m]);
                } else {
                    const float s = rcp_approx(ex2_approx(x[k] - y[k + m]) + 1.0f);
                    r1[m] += s;
                    r2[m] = fmaf(s, s, r2[m]);
                }
            }
        }
    }
}

// acc[k] += sum_m G[m] H(s_km) with H(s) = s (1 - s) (c1 s + c3), written with the
// per-shift coefficients A = -c1 G, B = (c1 - c3) G, C = c3 G as  s (C + s (B + A s)).
// Shared-memory coefficient layout per block of 8 shifts: for mp = 0..3 the two quads
// (A, B, C, 0) of shifts mp and mp + 4, i.e. 32 floats.
template <int MODE>
__device__ __forceinline__ void adj_chunk(const float (&x)[T], const float (&y)[2 * T], const float* gq,
                                          float (&acc)[T]) {
    // all 24 coefficients of the 8 shifts live in registers for the 8 positions
    float4 ca[T / 2], cb[T / 2];
#pragma unroll
    for (int mp = 0; mp < T / 2; ++mp) {
        ca[mp] = *reinterpret_cast<const float4*>(gq + 8 * mp);
        cb[mp] = *reinterpret_cast<const float4*>(gq + 8 * mp + 4);
    }
#pragma unroll
    for (int k = 0; k < T; ++k) {
#pragma unroll
        for (int mp = 0; mp < T / 2; ++mp) {
            if (MODE == MODE_FAST) {
                const float da = fmaf(x[k], y[k + mp], 1.0f);
                const float db = fmaf(x[k], y[k + mp + T / 2], 1.0f);
                const float r = rcp_approx(da * db);
                const float sa = db * r, sb = da * r;
                float qa = fmaf(ca[mp].x, sa, ca[mp].y);
                qa = fmaf(qa, sa, ca[mp].z);
                acc[k] = fmaf(qa, sa, acc[k]);
                float qb = fmaf(cb[mp].x, sb, cb[mp].y);
                qb = fmaf(qb, sb, cb[mp].z);
                acc[k] = fmaf(qb, sb, acc[k]);
            } else if (MODE == MODE_IDENT) {
                acc[k] = fmaf(ca[mp].x, x[k] + y[k + mp], acc[k]);
                acc[k] = fmaf(cb[mp].x, x[k] + y[k + mp + T / 2], acc[k]);
            } else {
                const float sa = rcp_approx(ex2_approx(x[k] - y[k + mp]) + 1.0f);
                const float sb = rcp_approx(ex2_approx(x[k] - y[k + mp + T / 2]) + 1.0f);
                float qa = fmaf(ca[mp].x, sa, ca[mp].y);
                qa = fmaf(qa, sa, ca[mp].z);
                acc[k] = fmaf(qa, sa, acc[k]);
                float qb = fmaf(cb[mp].x, sb, cb[mp].y);
                qb = fmaf(qb, sb, cb[mp].z);
                acc[k] = fmaf(qb, sb, acc[k]);
            }
        }
    }
}

__device__ __forceinline__ void load8(const float* p, float (&v)[T]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    const float4 b = *reinterpret_cast<const float4*>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

__device__ __forceinline__ void load16(const float* p, float (&v)[2 * T]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 a = *reinterpret_cast<const float4*>(p + 4 * i);
        v[4 * i + 0] = a.x; v[4 * i + 1] = a.y; v[4 * i + 2] = a.z; v[4 * i + 3] = a.w;
    }
}

// ------------------------------------------------------------------------- forward

// One plane of the block's tile; row sums (<= 32 terms) are added to the block sums, which
// hold at most 64 row sums (plans keep TY x planes-per-block <= 64).
template <int MODE>
__device__ __forceinline__ void fwd_plane(const float* xs, const float* ybase, int strideH, int rowsValid,
                                          int chunksValid, float (&t1)[T], float (&t2)[T]) {
    for (int iy = 0; iy < rowsValid; ++iy) {
        float r1[T], r2[T];
#pragma unroll
        for (int m = 0; m < T; ++m) { r1[m] = 0.f; r2[m] = 0.f; }
        const float* xrow = xs + iy * TX;
        const float* yrow = ybase + iy * strideH;
#pragma unroll 1
        for (int c = 0; c < chunksValid; ++c) {
            float x[T], y[2 * T];
            load8(xrow + c * T, x);
            load16(yrow + c * T, y);
            fwd_chunk<MODE>(x, y, r1, r2);
        }
#pragma unroll
        for (int m = 0; m < T; ++m) { t1[m] += r1[m]; t2[m] += r2[m]; }
    }
}

template <bool IDENT>
__global__ void __launch_bounds__(FWD_THREADS, 5)
corr_fwd_kernel(const FwdSeg* __restrict__ segs, int nseg, ThreshConst tc) {
    const int si = find_segment(segs, nseg, (int64_t)blockIdx.x);
    const FwdSeg& sg = segs[si];
    if (sg.done != nullptr && *sg.done) return;
    const LevelGeom g = sg.g;
    const float* __restrict__ field = sg.field;
    float* __restrict__ partial = sg.partial;
    const int64_t local = (int64_t)blockIdx.x - sg.blockStart;
    extern __shared__ __align__(16) float smem[];
    const int tid = threadIdx.x;
    const int64_t ts = local % g.fwdTiles;
    const int tx = (int)(ts % g.tilesX);
    const int ty = (int)((ts / g.tilesX) % g.tilesY);
    const int pc = (int)(ts / ((int64_t)g.tilesX * g.tilesY));
    const int64_t x0 = (int64_t)tx * TX, y0 = (int64_t)ty * g.TY;
    const int64_t z0 = (int64_t)pc * g.PPB;
    const int64_t z1 = min(z0 + (int64_t)g.PPB, g.n[0]);
    const int64_t n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];

    const int64_t gfirst = (local / g.fwdTiles) * FWD_THREADS;
    const int64_t glast = min(gfirst + FWD_THREADS, g.NG) - 1;
    const GroupBox bx = group_box(g, gfirst, glast);
    const FwdSmem sh = fwd_smem_shape(g, bx);

    float* xs = smem;                       // TY x TX tails
    float* ys = smem + g.TY * TX;           // planesH x rowsH x strideH tips

    const int64_t gi = gfirst + tid;
    const bool gvalid = gi < g.NG;
    int rz = bx.rzA, ry = bx.rylo, b = bx.blo;
    if (gvalid) decode_group(g, gi, rz, ry, b);
    const float* ybase = ys + ((int64_t)(rz - bx.rzA) * sh.rowsH + (ry - bx.rylo)) * sh.strideH + T * (b - bx.blo);

    const int rowsValid = (int)min((int64_t)g.TY, n1 - y0);
    const int colsValid = (int)min((int64_t)TX, n2 - x0);
    const int chunksValid = (colsValid + T - 1) / T;

    float t1[T], t2[T];
#pragma unroll
    for (int m = 0; m < T; ++m) { t1[m] = 0.f; t2[m] = 0.f; }

    const int warp = tid >> 5, lane = tid & 31;
    constexpr int NW = FWD_THREADS / 32;
    const int rowsAll = sh.planesH * sh.rowsH;
    const int64_t hx0 = x0 - g.P[2] + (int64_t)T * bx.blo;
    const float kinf = __int_as_float(0x7f800000);

    for (int64_t z = z0; z < z1; ++z) {
        __syncthreads();
        bool bad = false;
        // tails: one row per warp, one column per lane; +inf marks positions outside the field (s = 0)
        for (int iy = warp; iy < g.TY; iy += NW) {
            const bool valid = (y0 + iy < n1) && (x0 + lane < n2);
            const float v = valid ? field[(z * n1 + y0 + iy) * n2 + x0 + lane] : 0.f;
            bad |= valid && !(fabsf(tc.kappa * v) <= tc.lim) && !isnan(v);
            xs[iy * TX + lane] = IDENT ? (valid ? 0.5f * v : 0.f)
                                       : (valid ? ex2_approx(fmaf(-tc.kappa, v, tc.cexp)) : 0x1p100f);
        }
        // tips: the periodic halo, one row per warp, columns strided by the lanes
        for (int pr = warp; pr < rowsAll; pr += NW) {
            const int p = pr / sh.rowsH, r = pr - p * sh.rowsH;
            const float* src = field + (wrap1(z + bx.rzA + p, n0) * n1 + wrap1(y0 + bx.rylo + r, n1)) * n2;
            float* dst = ys + pr * sh.strideH;
            int64_t gx = wrap1(hx0 + lane, n2);
            for (int c = lane; c < sh.colsH; c += 32) {
                const float v = src[gx];
                bad |= !(fabsf(tc.kappa * v) <= tc.lim) && !isnan(v);
                dst[c] = IDENT ? 0.5f * v : ex2_approx(-tc.kappa * v);
                gx += 32;
                while (gx >= n2) gx -= n2;
            }
        }
        const int slow = __syncthreads_or(bad);
        if (!IDENT && slow) {
            // rare: the block holds values outside the fast range; rewrite both tiles in the
            // exact form (exponents, combined per pair) from the field
            for (int iy = warp; iy < g.TY; iy += NW) {
                const bool valid = (y0 + iy < n1) && (x0 + lane < n2);
                const float v = valid ? field[(z * n1 + y0 + iy) * n2 + x0 + lane] : 0.f;
                xs[iy * TX + lane] = valid ? fmaf(-tc.kappa, v, tc.cexp) : kinf;
            }
            for (int pr = warp; pr < rowsAll; pr += NW) {
                const int p = pr / sh.rowsH, r = pr - p * sh.rowsH;
                const float* src = field + (wrap1(z + bx.rzA + p, n0) * n1 + wrap1(y0 + bx.rylo + r, n1)) * n2;
                float* dst = ys + pr * sh.strideH;
                int64_t gx = wrap1(hx0 + lane, n2);
                for (int c = lane; c < sh.colsH; c += 32) {
                    dst[c] = tc.kappa * src[gx];
                    gx += 32;
                    while (gx >= n2) gx -= n2;
                }
            }
        }
        __syncthreads();
        if (IDENT) fwd_plane<MODE_IDENT>(xs, ybase, sh.strideH, rowsValid, chunksValid, t1, t2);
        else if (slow) fwd_plane<MODE_SLOW>(xs, ybase, sh.strideH, rowsValid, chunksValid, t1, t2);
        else fwd_plane<MODE_FAST>(xs, ybase, sh.strideH, rowsValid, chunksValid, t1, t2);
    }

    if (!gvalid) return;
    // sum_x f^2 = c1^2 sum s^2 + 2 c1 c3 sum s + n c3^2 (identity: sum a^2 directly)
    const float nvalid = (float)((z1 - z0) * (int64_t)rowsValid * colsValid);
    float* out = partial + ts * g.Khalf;
#pragma unroll
    for (int m = 0; m < T; ++m) {
        const int rx = -g.P[2] + T * b + m;
        const int64_t k = canon_index(g, rz, ry, rx);
        if (k < 0) continue;
        float v;
        if (IDENT) v = t2[m];
        else v = fmaf(tc.c1 * tc.c1, t2[m], fmaf(2.f * tc.c1 * tc.c3, t1[m], nvalid * tc.c3 * tc.c3));
        out[k] = v;
    }
}

// Fixed-order FP64 sum over tiles, scaled by w_l / N_l.  A block owns 32 consecutive
// shifts (one per lane, coalesced rows); warp w sums the tiles t = w (mod 8) in order and
// the 8 warp sums are combined in a fixed order.
__global__ void __launch_bounds__(256) fwd_reduce_kernel(const RedSeg* __restrict__ segs, int nseg) {
    const int si = find_segment(segs, nseg, (int64_t)blockIdx.x);
    const RedSeg& sg = segs[si];
    if (sg.done != nullptr && *sg.done) return;
    const int64_t Khalf = sg.g.Khalf, tiles = sg.g.fwdTiles;
    __shared__ double sh[8][RED_K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k = ((int64_t)blockIdx.x - sg.blockStart) * RED_K + lane;
    // compensated (Kahan) FP32 sum over this warp's tiles, then an FP64 sum of the 8 warps
    float sum = 0.f, comp = 0.f;
    if (k < Khalf)
        for (int64_t t = warp; t < tiles; t += 8) {
            const float y = sg.partial[t * Khalf + k] - comp;
            const float u = sum + y;
            comp = (u - sum) - y;
            sum = u;
        }
    sh[warp][lane] = (double)sum - (double)comp;
    __syncthreads();
    if (warp == 0 && k < Khalf) {
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += sh[w][lane];
        sg.desc[k] = (float)((double)sg.weight * tot / (double)sg.g.N);
    }
}

// ------------------------------------------------------------------------- adjoint

template <int MODE>
__device__ __forceinline__ void adj_rows(const float* ys, const float* Gs, int strideH, int NB, int ryN, int lane,
                                         int strip, const float (&x)[T], float (&acc)[T]) {
    for (int r = 0; r < ryN; ++r) {
        const float* yrow = ys + (lane + r) * strideH + T * strip;
        const float* grow = Gs + r * (NB * 4 * T);
#pragma unroll 1
        for (int bb = 0; bb < NB; ++bb) {
            float y[2 * T];
            load16(yrow + T * bb, y);
            adj_chunk<MODE>(x, y, grow + 4 * T * bb, acc);
        }
    }
}

template <bool IDENT>
__global__ void __launch_bounds__(ADJ_THREADS, 4)
corr_adj_kernel(const AdjSeg* __restrict__ segs, int nseg, ThreshConst tc) {
    const int si = find_segment(segs, nseg, (int64_t)blockIdx.x);
    const AdjSeg& sg = segs[si];
    if (sg.done != nullptr && *sg.done) return;
    const LevelGeom g = sg.g;
    const float* __restrict__ field = sg.field;
    const float* __restrict__ Gd = sg.Gd;
    float* __restrict__ part = sg.part;
    const int64_t local = (int64_t)blockIdx.x - sg.blockStart;
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31, strip = threadIdx.x >> 5;
    const int64_t tile = local % g.adjTiles;
    const int tx = (int)(tile % g.adjTilesX);
    const int ty = (int)((tile / g.adjTilesX) % g.adjTilesY);
    const int64_t z = tile / ((int64_t)g.adjTilesX * g.adjTilesY);
    const int64_t x0 = (int64_t)tx * TX, y0 = (int64_t)ty * 32;
    const int64_t n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    const int chunk = (int)(local / g.adjTiles);
    const int zc = chunk / g.nYc, yc = chunk % g.nYc;
    const int rzA = -g.P[0] + zc * g.RZ;
    const int rzB = min(rzA + g.RZ, g.P[0] + 1);
    const int ryA = -g.P[1] + yc * g.RY;
    const int ryB = min(ryA + g.RY, g.P[1] + 1);
    const int ryN = ryB - ryA;
    const int WB = g.NB * T;
    const int rowsH = 32 + ryN - 1;
    const int colsH = WB + 3 * T + 2 * T;   // 8 NB + 32 (see strip/bb read extents)
    const int strideH = stride_4mod32(colsH);
    float* ys = smem;
    float* Gs = smem + rowsH * strideH;
    const int64_t hx0 = x0 - g.P[2];

    // own positions: row y0 + lane, columns x0 + 8 strip + k (values reloaded per rz plane)
    const int64_t py = y0 + lane;
    const float* xrow = field + (z * n1 + (py < n1 ? py : 0)) * n2;
    bool xbad = false;
#pragma unroll
    for (int k = 0; k < T; ++k) {
        const int64_t px = x0 + T * strip + k;
        const float v = (py < n1 && px < n2) ? xrow[px] : 0.f;
        xbad |= !(fabsf(tc.kappa * v) <= tc.lim) && !isnan(v);
    }
    float acc[T];
#pragma unroll
    for (int k = 0; k < T; ++k) acc[k] = 0.f;

    const int ng = ryN * 4 * WB;
    const int warp = threadIdx.x >> 5;
    constexpr int NW = ADJ_THREADS / 32;
    for (int rz = rzA; rz < rzB; ++rz) {
        __syncthreads();
        const int64_t gz = wrap1(z + rz, n0);
        bool bad = xbad;
        for (int r = warp; r < rowsH; r += NW) {
            const float* src = field + (gz * n1 + wrap1(y0 + ryA + r, n1)) * n2;
            float* dst = ys + r * strideH;
            int64_t gx = wrap1(hx0 + lane, n2);
            for (int c = lane; c < colsH; c += 32) {
                const float v = src[gx];
                bad |= !(fabsf(tc.kappa * v) <= tc.lim) && !isnan(v);
                dst[c] = IDENT ? 0.5f * v : ex2_approx(-tc.kappa * v);
                gx += 32;
                while (gx >= n2) gx -= n2;
            }
        }
        const float4* grow0 = reinterpret_cast<const float4*>(
            Gd + ((int64_t)(rz + g.P[0]) * (2 * g.P[1] + 1) + (ryA + g.P[1])) * 4 * WB);
        for (int i = threadIdx.x; i < ng / 4; i += ADJ_THREADS) reinterpret_cast<float4*>(Gs)[i] = grow0[i];
        const int slow = __syncthreads_or(bad);
        if (!IDENT && slow) {
            for (int r = warp; r < rowsH; r += NW) {
                const float* src = field + (gz * n1 + wrap1(y0 + ryA + r, n1)) * n2;
                float* dst = ys + r * strideH;
                int64_t gx = wrap1(hx0 + lane, n2);
                for (int c = lane; c < colsH; c += 32) {
                    dst[c] = tc.kappa * src[gx];
                    gx += 32;
                    while (gx >= n2) gx -= n2;
                }
            }
        }
        float x[T];
#pragma unroll
        for (int k = 0; k < T; ++k) {
            const int64_t px = x0 + T * strip + k;
            const float v = (py < n1 && px < n2) ? xrow[px] : 0.f;
            const float u = fmaf(-tc.kappa, v, tc.cexp);
            x[k] = IDENT ? 0.5f * v : (slow ? u : ex2_approx(u));
        }
        __syncthreads();
        if (IDENT) adj_rows<MODE_IDENT>(ys, Gs, strideH, g.NB, ryN, lane, strip, x, acc);
        else if (slow) adj_rows<MODE_SLOW>(ys, Gs, strideH, g.NB, ryN, lane, strip, x, acc);
        else adj_rows<MODE_FAST>(ys, Gs, strideH, g.NB, ryN, lane, strip, x, acc);
    }

    if (py >= n1) return;
    float* out = part + (int64_t)chunk * g.N + (z * n1 + py) * n2;
#pragma unroll
    for (int k = 0; k < T; ++k) {
        const int64_t px = x0 + T * strip + k;
        if (px < n2) out[px] = acc[k];
    }
}

// Dense full-window coefficient grid of one level:
//   Gd[rz][ry][col], rx = col - P2 (zero where rx > P2),
//   value = scale * (src[k] - sub[k]) * (2 if r = 0),  k = canonical index of +-r,
//   scale = weight * (gscale from the loss, or 1) * (c1 alpha / N_l, or 1 / N_l for f(x)=x).
// Dense full-window coefficient grid of one level, in adjoint order:
//   G(r) = scale * (src[k] - sub[k]) * (2 if r = 0),  k = canonical index of +-r,
//   scale = weight * (gscale from the loss, or 1) * (c1 alpha / N_l, or 1 / N_l for f(x)=x),
//   quad (A, B, C, 0) = (-c1 G, (c1 - c3) G, c3 G, 0)   (f(x) = x: (G, 0, 0, 0)),
// zero where rx > P2 (padding of the last rx block).  Row (rz, ry) holds NB blocks of 8
// shifts; a block stores for mp = 0..3 the quads of shifts mp and mp + 4 (32 floats).
__global__ void gcoef_kernel(const GSeg* __restrict__ segs, int nseg, ThreshConst tc) {
    const int si = find_segment(segs, nseg, (int64_t)blockIdx.x);
    const GSeg& sg = segs[si];
    if (sg.done != nullptr && *sg.done) return;
    const LevelGeom& g = sg.g;
    const int WB = g.NB * T;
    const int64_t total = (int64_t)(2 * g.P[0] + 1) * (2 * g.P[1] + 1) * WB;
    const int64_t i = ((int64_t)blockIdx.x - sg.blockStart) * GCOEF_TH + threadIdx.x;
    if (i >= total) return;
    const int col = (int)(i % WB);
    const int64_t row = i / WB;
    const int ryi = (int)(row % (2 * g.P[1] + 1));
    const int rzi = (int)(row / (2 * g.P[1] + 1));
    const int rz = rzi - g.P[0], ry = ryi - g.P[1], rx = col - g.P[2];
    float v = 0.f;
    if (rx <= g.P[2]) {
        int64_t k = canon_index(g, rz, ry, rx);
        if (k < 0) k = canon_index(g, -rz, -ry, -rx);
        const float d = sg.src[k] - (sg.sub != nullptr ? sg.sub[k] : 0.f);
        float sc = sg.scale * (sg.sc != nullptr ? sg.sc->gscale : 1.f);
        if (rz == 0 && ry == 0 && rx == 0) sc *= 2.f;
        v = sc * d;
    }
    const int b = col / T, m = col % T;
    float4 q;
    if (tc.identity) q = make_float4(v, 0.f, 0.f, 0.f);
    else q = make_float4(-tc.c1 * v, (tc.c1 - tc.c3) * v, tc.c3 * v, 0.f);
    float4* dst = reinterpret_cast<float4*>(sg.Gd + (row * g.NB + b) * (4 * T)) + (2 * (m % (T / 2)) + m / (T / 2));
    *dst = q;
}

// ------------------------------------------------------------------------- launchers

size_t fwd_smem_bytes(const LevelGeom& g) {
    int maxFloats = 0;
    for (int gb = 0; gb < g.fwdGroupBlocks; ++gb) {
        const int64_t gfirst = (int64_t)gb * FWD_THREADS;
        const int64_t glast = std::min<int64_t>(gfirst + FWD_THREADS, g.NG) - 1;
        const GroupBox bx = group_box(g, gfirst, glast);
        const FwdSmem sh = fwd_smem_shape(g, bx);
        const int f = g.TY * TX + sh.planesH * sh.rowsH * sh.strideH;
        if (f > maxFloats) maxFloats = f;
    }
    return (size_t)maxFloats * sizeof(float);
}

void launch_corr_fwd(const FwdSeg* segs, int nseg, int64_t blocks, size_t smem, const ThreshConst& tc,
                     cudaStream_t s) {
    if (blocks <= 0) return;
    if (tc.identity) corr_fwd_kernel<true><<<(unsigned)blocks, FWD_THREADS, smem, s>>>(segs, nseg, tc);
    else corr_fwd_kernel<false><<<(unsigned)blocks, FWD_THREADS, smem, s>>>(segs, nseg, tc);
}

void launch_fwd_reduce(const RedSeg* segs, int nseg, int64_t blocks, cudaStream_t s) {
    if (blocks <= 0) return;
    fwd_reduce_kernel<<<(unsigned)blocks, 256, 0, s>>>(segs, nseg);
}

size_t adj_smem_bytes(const LevelGeom& g) {
    const int WB = g.NB * T;
    const int rowsH = 32 + g.RY - 1;
    const int colsH = WB + 5 * T;
    return (size_t)(rowsH * stride_4mod32(colsH) + 4 * g.RY * WB) * sizeof(float);
}

void launch_corr_adj(const AdjSeg* segs, int nseg, int64_t blocks, size_t smem, const ThreshConst& tc,
                     cudaStream_t s) {
    if (blocks <= 0) return;
    if (tc.identity) corr_adj_kernel<true><<<(unsigned)blocks, ADJ_THREADS, smem, s>>>(segs, nseg, tc);
    else corr_adj_kernel<false><<<(unsigned)blocks, ADJ_THREADS, smem, s>>>(segs, nseg, tc);
}

void set_kernel_attributes() {
    const int bytes = MAX_DYN_SMEM;
    cudaFuncSetAttribute(corr_fwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(corr_fwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(corr_adj_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(corr_adj_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Coefficient scale of one level: w_l * c1 * alpha / N_l (soft; h = c1 alpha H(s)) or w_l / N_l.
float gcoef_scale(const LevelGeom& g, const ThreshConst& tc, float weight) {
    return tc.identity ? (float)((double)weight / (double)g.N)
                       : (float)((double)weight * (double)tc.c1 * (double)tc.alpha / (double)g.N);
}

void launch_gcoef(const GSeg* segs, int nseg, int64_t blocks, const ThreshConst& tc, cudaStream_t s) {
    if (blocks <= 0) return;
    gcoef_kernel<<<(unsigned)blocks, GCOEF_TH, 0, s>>>(segs, nseg, tc);
}

}  // namespace dmcr
