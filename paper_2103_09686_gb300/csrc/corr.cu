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
// plane, block) in FP32, written per tile and reduced across tiles in fixed order with
// compensated sums (Kahan per warp, then a double-float two-sum of the warps): the result
// is deterministic.
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
    int planesH, rowsH, colsH, strideP;
};

// Halo of a forward block: rows rylo .. ryhi + TY (one more row for the shifts that take
// the tail rows offset by one), rounded up to whole row pairs; a pair row stores float2
// (row 2p, row 2p + 1) per column, stride 4 mod 32 words.
__host__ __device__ inline FwdSmem fwd_smem_shape(const LevelGeom& g, const GroupBox& bx) {
    FwdSmem s;
    s.planesH = bx.rzB - bx.rzA + 1;
    const int rows = g.TY + bx.ryhi - bx.rylo + 1;
    s.rowsH = rows + (rows & 1);
    s.colsH = T * (bx.bhi - bx.blo) + TX + T;
    s.strideP = stride_4mod32(2 * s.colsH);
    return s;
}

// ------------------------------------------------------------------------- pair math
//
// Packed FP32x2 arithmetic: the two halves of a float2 belong to two different position
// rows (forward: rows iy, iy+1 of the tile; adjoint: rows lane, lane+32), so one FFMA2
// issues the same step for two pairs.  The kernels are bound by the FP32 pipe (128 lane
// operations per SM and clock; an FFMA2 counts twice) together with the MUFU reciprocal
// (16 per SM and clock).  Two pairs share one reciprocal: with d = 1 + E'_x E_y >= 1,
//     r = 1 / (d_a d_b),   (d_a, d_b) * (r, r) = (1/d_b, 1/d_a) = (s_b, s_a),
// valid while every d <= 2^62 (|kappa M| <= lim); the product lands with the halves
// swapped, which the accumulators absorb (they read the rows back crosswise).  The
// adjoint gives a few positions one reciprocal per pair (s = 1/d), which moves work from
// the FP32 pipe to the otherwise idle share of the MUFU.  Blocks with values beyond lim
// take the exact per-pair form (one exponential per pair).

enum { MODE_FAST = 0, MODE_SLOW = 1, MODE_IDENT = 2 };

// adjoint: positions k < ADJ_SINGLE of every 8 use one reciprocal per pair (measured: 4 is
// 0.6% faster than 3 and 1.4% faster than 2 with the staged block)
constexpr int ADJ_SINGLE = 4;

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// exact form, halves swapped like the product form: e = cexp - kappa (M_x + M_y) per half
__device__ __forceinline__ float2 sig_exact_swapped(float2 e) {
    return make_float2(rcp_approx(ex2_approx(e.y) + 1.0f), rcp_approx(ex2_approx(e.x) + 1.0f));
}

// Forward, one chunk of a row pair: x2[k] tails at column k, y2[j] tips at column j; pair
// (k, m) uses y2[k + m].  acc[m] += (s + beta)^2 per row (beta = c3 / c1, so c1 (s + beta) = f);
// identity: acc[m] += a^2.  The soft modes leave the rows swapped in acc (row iy in .y).
// Columns k >= kv are outside the field (ragged last chunk).
template <int MODE, bool FULL>
__device__ __forceinline__ void fwd_chunk(const float2 (&x2)[T], const float2 (&y2)[2 * T], float2 (&acc)[T],
                                          float beta, int kv) {
    const float2 one2 = make_float2(1.0f, 1.0f);
    const float2 b2 = make_float2(beta, beta);
#pragma unroll
    for (int k = 0; k < T; ++k) {
        if (!FULL && k >= kv) continue;
        if (MODE == MODE_FAST) {
            // stage by stage over the 8 shifts (all d, the reciprocals, then u and u^2)
            float2 d[T];
            float r[T];
#pragma unroll
            for (int m = 0; m < T; ++m) d[m] = ffma2(x2[k], y2[k + m], one2);
#pragma unroll
            for (int m = 0; m < T; ++m) r[m] = rcp_approx(d[m].x * d[m].y);
#pragma unroll
            for (int m = 0; m < T; ++m) {
                const float2 u = ffma2(d[m], make_float2(r[m], r[m]), b2);
                acc[m] = ffma2(u, u, acc[m]);
            }
            continue;
        }
#pragma unroll
        for (int m = 0; m < T; ++m) {
            float2 u;
            if (MODE == MODE_IDENT) {
                u = fadd2(x2[k], y2[k + m]);
            } else if (MODE == MODE_SLOW) {
                u = fadd2(sig_exact_swapped(fadd2(x2[k], y2[k + m])), b2);
            } else {
                const float2 d = ffma2(x2[k], y2[k + m], one2);
                const float r = rcp_approx(d.x * d.y);
                u = ffma2(d, make_float2(r, r), b2);
            }
            acc[m] = ffma2(u, u, acc[m]);
        }
    }
}

// Adjoint, one block of 8 shifts: x2[k] own values at column k (rows lane, lane+32),
// y2[j] partners at column j; pair (k, m) uses y2[k + m].  acc[k] += G(r_m) h(s) per row with
// h(s) written s (C + s (B + A s)), A = -c1 G, B = (c1 - c3) G, C = c3 G (identity: G a).
// The soft modes leave the rows swapped in acc (row lane in .y).  Coefficients per block:
// (A, A, B, B) for m = 0..7, then (C_m, C_m, C_m+1, C_m+1) for even m.  PARTIAL: only the
// first mv shifts lie in the window (the last block of a row; the others have zero
// coefficients, so skipping them leaves acc bitwise unchanged).
template <int MODE, bool PARTIAL = false>
__device__ __forceinline__ void adj_block(const float2 (&x2)[T], const float2 (&y2)[2 * T],
                                          const float4* __restrict__ cf, float2 (&acc)[T], int mv = T) {
    const float2 one2 = make_float2(1.0f, 1.0f);
#pragma unroll
    for (int m = 0; m < T; ++m) {
        if (PARTIAL && m >= mv) break;
        const float4 ab = cf[m];
        const float4 cc = cf[T + m / 2];
        const float2 A2 = make_float2(ab.x, ab.y);
        const float2 B2 = make_float2(ab.z, ab.w);
        const float2 C2 = (m & 1) ? make_float2(cc.z, cc.w) : make_float2(cc.x, cc.y);
        if (MODE == MODE_FAST) {
            // stage by stage over the 8 positions (all d, the reciprocals, s, then Horner):
            // independent operations sit next to each other, which hides the MUFU latency
            float2 d[T], s[T];
            float r[T];
#pragma unroll
            for (int k = 0; k < T; ++k) d[k] = ffma2(x2[k], y2[k + m], one2);
#pragma unroll
            for (int k = ADJ_SINGLE; k < T; ++k) r[k] = rcp_approx(d[k].x * d[k].y);
#pragma unroll
            for (int k = 0; k < ADJ_SINGLE; ++k) s[k] = make_float2(rcp_approx(d[k].y), rcp_approx(d[k].x));
#pragma unroll
            for (int k = ADJ_SINGLE; k < T; ++k) s[k] = fmul2(d[k], make_float2(r[k], r[k]));
#pragma unroll
            for (int k = 0; k < T; ++k) {
                float2 q = ffma2(A2, s[k], B2);
                q = ffma2(q, s[k], C2);
                acc[k] = ffma2(q, s[k], acc[k]);
            }
            continue;
        }
#pragma unroll
        for (int k = 0; k < T; ++k) {
            if (MODE == MODE_IDENT) {
                acc[k] = ffma2(A2, fadd2(x2[k], y2[k + m]), acc[k]);
                continue;
            }
            float2 s;
            if (MODE == MODE_SLOW) {
                s = sig_exact_swapped(fadd2(x2[k], y2[k + m]));
            } else {
                const float2 d = ffma2(x2[k], y2[k + m], one2);
                if (k < ADJ_SINGLE) {
                    s = make_float2(rcp_approx(d.y), rcp_approx(d.x));
                } else {
                    const float r = rcp_approx(d.x * d.y);
                    s = fmul2(d, make_float2(r, r));
                }
            }
            float2 q = ffma2(A2, s, B2);
            q = ffma2(q, s, C2);
            acc[k] = ffma2(q, s, acc[k]);
        }
    }
}

__device__ __forceinline__ void load_pairs8(const float* p, float2 (&v)[T]) {
#pragma unroll
    for (int i = 0; i < T / 2; ++i) {
        const float4 a = *reinterpret_cast<const float4*>(p + 4 * i);
        v[2 * i] = make_float2(a.x, a.y);
        v[2 * i + 1] = make_float2(a.z, a.w);
    }
}

__device__ __forceinline__ void load_pairs16(const float* p, float2 (&v)[2 * T]) {
#pragma unroll
    for (int i = 0; i < T; ++i) {
        const float4 a = *reinterpret_cast<const float4*>(p + 4 * i);
        v[2 * i] = make_float2(a.x, a.y);
        v[2 * i + 1] = make_float2(a.z, a.w);
    }
}

// Asynchronous global -> shared copies (cp.async): the halo loads of a block are issued
// back to back and waited for once, instead of one dependent round trip per column.
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// waits for this thread's own copies (visible to this thread; other threads need a barrier)
__device__ __forceinline__ void cp_async_wait_own() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// value stored in the shared tiles for one field value (tail side adds cexp)
template <int MODE>
__device__ __forceinline__ float tile_value(const ThreshConst& tc, float v, bool tail) {
    if (MODE == MODE_IDENT) return 0.5f * v;
    if (MODE == MODE_SLOW) return tail ? fmaf(-tc.kappa, v, tc.cexp) : -tc.kappa * v;
    return ex2_approx(tail ? fmaf(-tc.kappa, v, tc.cexp) : -tc.kappa * v);
}

// 1 when |kappa v| > lim (the block takes the exact form); NaN counts as in range: it
// propagates on any path
__device__ __forceinline__ int out_of_range(const ThreshConst& tc, float v) {
    return fabsf(tc.kappa * v) > tc.lim;
}

// ------------------------------------------------------------------------- forward

// One plane of the block's tile.  Row pairs q hold tail rows (2q + cls, 2q + cls + 1); the
// second row of the last pair lies outside the tile when rowsValid is odd.  Per-pair sums
// (<= 32 terms per row) are added to the block sums, which hold at most 64 row sums (plans
// keep TY x planes-per-block <= 64).
template <int MODE>
__device__ __forceinline__ void fwd_plane(const float* xbase, const float* ybase, int strideP, int rowsValid,
                                          int colsValid, float beta, float (&tsum)[T]) {
    const int nPairs = (rowsValid + 1) >> 1;
    const int chunksFull = colsValid / T, kvLast = colsValid % T;
    for (int q = 0; q < nPairs; ++q) {
        float2 acc[T];
#pragma unroll
        for (int m = 0; m < T; ++m) acc[m] = make_float2(0.f, 0.f);
        const float* xrow = xbase + 2 * q * TX;
        const float* yrow = ybase + q * strideP;
#pragma unroll 1
        for (int c = 0; c < chunksFull; ++c) {
            float2 x2[T], y2[2 * T];
            load_pairs8(xrow + 2 * T * c, x2);
            load_pairs16(yrow + 2 * T * c, y2);
            fwd_chunk<MODE, true>(x2, y2, acc, beta, T);
        }
        if (kvLast) {
            float2 x2[T], y2[2 * T];
            load_pairs8(xrow + 2 * T * chunksFull, x2);
            load_pairs16(yrow + 2 * T * chunksFull, y2);
            fwd_chunk<MODE, false>(x2, y2, acc, beta, kvLast);
        }
        // the first row of the pair sits in .y in the soft modes (halves swapped), in .x otherwise
        const bool second = 2 * q + 1 < rowsValid;
#pragma unroll
        for (int m = 0; m < T; ++m)
            tsum[m] += second ? acc[m].x + acc[m].y : (MODE == MODE_IDENT ? acc[m].x : acc[m].y);
    }
}

template <bool IDENT>
__global__ void __launch_bounds__(FWD_THREADS, 4)
corr_fwd_kernel(const FwdSeg* __restrict__ segs, int nseg, ThreshConst tc) {
    const int si = find_segment(segs, nseg, (int64_t)blockIdx.x);
    const FwdSeg& sg = segs[si];
    if (sg.done != nullptr && *sg.done) return;
    const LevelGeom g = sg.g;
    const float* __restrict__ field = sg.field;
    const float* __restrict__ tipf = sg.tip;
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
    const int pairRowsH = sh.rowsH / 2;

    // tails: two tiles of TY/2 row pairs x TX columns (float2 per column), rows (2q, 2q+1)
    // and (2q+1, 2q+2); tips: planesH x pairRowsH x strideP, rows (2p, 2p+1) of the halo
    const int xtile = g.TY * TX + 4;
    float* xs = smem;
    float* ys = smem + 2 * xtile;

    const int64_t gi = gfirst + tid;
    const bool gvalid = gi < g.NG;
    int rz = bx.rzA, ry = bx.rylo, b = bx.blo;
    if (gvalid) decode_group(g, gi, rz, ry, b);
    // shifts at an odd row offset from the halo start take the tail rows shifted by one:
    // positions are periodic, so rows y0+1 .. y0+TY cover the same set once over all tiles
    const int cls = (ry - bx.rylo) & 1;
    const int rrel = ry - bx.rylo + cls;
    const float* ybase = ys + ((int64_t)(rz - bx.rzA) * pairRowsH + rrel / 2) * sh.strideP + 2 * T * (b - bx.blo);
    const float* xbase = xs + cls * xtile;

    const int rowsValid = (int)min((int64_t)g.TY, n1 - y0);
    const int colsValid = (int)min((int64_t)TX, n2 - x0);
    const float beta = tc.beta;

    float tsum[T];
#pragma unroll
    for (int m = 0; m < T; ++m) tsum[m] = 0.f;

    const int warp = tid >> 5, lane = tid & 31;
    constexpr int NW = FWD_THREADS / 32;
    const int prAll = sh.planesH * pairRowsH;
    const int64_t hx0 = x0 - g.P[2] + (int64_t)T * bx.blo;
    const bool colOk = x0 + lane < n2;

    for (int64_t z = z0; z < z1; ++z) {
        __syncthreads();
        // tails (row rho of the tile is valid for class 0 when rho < rowsValid, for class 1
        // when 1 <= rho <= rowsValid; invalid entries hold 0, i.e. d = 1) and the tips (the
        // periodic halo, one pair of rows per warp, columns strided by the lanes): raw values
        // copied asynchronously, then transformed in place by the thread that copied them
        for (int pr = warp; pr < g.TY; pr += NW) {
            const int t = pr / (g.TY / 2), q = pr - t * (g.TY / 2);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int rho = 2 * q + t + h;
                const bool valid = colOk && (t == 0 ? rho < rowsValid : rho <= rowsValid);
                float* d = xs + t * xtile + 2 * (q * TX + lane) + h;
                if (valid) cp_async4(d, field + (z * n1 + wrap1(y0 + rho, n1)) * n2 + x0 + lane);
                else *d = 0.f;
            }
        }
        for (int pr = warp; pr < prAll; pr += NW) {
            const int p = pr / pairRowsH, r = pr - p * pairRowsH;
            const int64_t zz = wrap1(z + bx.rzA + p, n0);
            const float* srcA = tipf + (zz * n1 + wrap1(y0 + bx.rylo + 2 * r, n1)) * n2;
            const float* srcB = tipf + (zz * n1 + wrap1(y0 + bx.rylo + 2 * r + 1, n1)) * n2;
            float* dst = ys + (int64_t)pr * sh.strideP;
            int64_t gx = wrap1(hx0 + lane, n2);
            for (int c = lane; c < sh.colsH; c += 32) {
                cp_async4(dst + 2 * c, srcA + gx);
                cp_async4(dst + 2 * c + 1, srcB + gx);
                gx += 32;
                while (gx >= n2) gx -= n2;
            }
        }
        cp_async_wait_own();
        int rc = 0;
        for (int pr = warp; pr < g.TY; pr += NW) {
            const int t = pr / (g.TY / 2), q = pr - t * (g.TY / 2);
            float* d = xs + t * xtile + 2 * (q * TX + lane);
            float e[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int rho = 2 * q + t + h;
                const bool valid = colOk && (t == 0 ? rho < rowsValid : rho <= rowsValid);
                const float v = d[h];
                if (valid) rc |= out_of_range(tc, v);
                e[h] = !valid ? 0.f : (IDENT ? 0.5f * v : tile_value<MODE_FAST>(tc, v, true));
            }
            *reinterpret_cast<float2*>(d) = make_float2(e[0], e[1]);
        }
        for (int pr = warp; pr < prAll; pr += NW) {
            float* dst = ys + (int64_t)pr * sh.strideP;
            for (int c = lane; c < sh.colsH; c += 32) {
                const float2 v = *reinterpret_cast<const float2*>(dst + 2 * c);
                rc |= out_of_range(tc, v.x) | out_of_range(tc, v.y);
                float2 e;
                if (IDENT) e = make_float2(0.5f * v.x, 0.5f * v.y);
                else e = make_float2(tile_value<MODE_FAST>(tc, v.x, false), tile_value<MODE_FAST>(tc, v.y, false));
                *reinterpret_cast<float2*>(dst + 2 * c) = e;
            }
        }
        const int slow = __syncthreads_or(rc);
        if (!IDENT && slow) {
            // rare: values outside the product range; rewrite both tiles in exponent form
            for (int pr = warp; pr < g.TY; pr += NW) {
                const int t = pr / (g.TY / 2), q = pr - t * (g.TY / 2);
                float e[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int rho = 2 * q + t + h;
                    const bool valid = colOk && (t == 0 ? rho < rowsValid : rho <= rowsValid);
                    const float v = valid ? field[(z * n1 + wrap1(y0 + rho, n1)) * n2 + x0 + lane] : 0.f;
                    e[h] = valid ? tile_value<MODE_SLOW>(tc, v, true) : 0.f;
                }
                *reinterpret_cast<float2*>(xs + t * xtile + 2 * (q * TX + lane)) = make_float2(e[0], e[1]);
            }
            for (int pr = warp; pr < prAll; pr += NW) {
                const int p = pr / pairRowsH, r = pr - p * pairRowsH;
                const int64_t zz = wrap1(z + bx.rzA + p, n0);
                const float* srcA = tipf + (zz * n1 + wrap1(y0 + bx.rylo + 2 * r, n1)) * n2;
                const float* srcB = tipf + (zz * n1 + wrap1(y0 + bx.rylo + 2 * r + 1, n1)) * n2;
                float* dst = ys + (int64_t)pr * sh.strideP;
                int64_t gx = wrap1(hx0 + lane, n2);
                for (int c = lane; c < sh.colsH; c += 32) {
                    *reinterpret_cast<float2*>(dst + 2 * c) = make_float2(
                        tile_value<MODE_SLOW>(tc, srcA[gx], false), tile_value<MODE_SLOW>(tc, srcB[gx], false));
                    gx += 32;
                    while (gx >= n2) gx -= n2;
                }
            }
        }
        __syncthreads();
        if (IDENT) fwd_plane<MODE_IDENT>(xbase, ybase, sh.strideP, rowsValid, colsValid, beta, tsum);
        else if (slow) fwd_plane<MODE_SLOW>(xbase, ybase, sh.strideP, rowsValid, colsValid, beta, tsum);
        else fwd_plane<MODE_FAST>(xbase, ybase, sh.strideP, rowsValid, colsValid, beta, tsum);
    }

    if (!gvalid) return;
    // sum_x f^2 = c1^2 sum (s + c3/c1)^2 (identity: sum a^2 directly)
    const float c1sq = tc.c1 * tc.c1;
    float* out = partial + ts * g.Khalf;
#pragma unroll
    for (int m = 0; m < T; ++m) {
        const int rx = -g.P[2] + T * b + m;
        const int64_t k = canon_index(g, rz, ry, rx);
        if (k < 0) continue;
        out[k] = IDENT ? tsum[m] : c1sq * tsum[m];
    }
}

// Fixed-order sum over tiles, scaled by w_l / N_l.  A block owns 32 consecutive shifts (one
// per lane, coalesced rows); warp w sums the tiles t = w (mod 8) in order (Kahan, FP32) and
// the 8 warp sums are combined in a fixed order as double-floats.
__global__ void __launch_bounds__(256) fwd_reduce_kernel(const RedSeg* __restrict__ segs, int nseg) {
    const int si = find_segment(segs, nseg, (int64_t)blockIdx.x);
    const RedSeg& sg = segs[si];
    if (sg.done != nullptr && *sg.done) return;
    const int64_t Khalf = sg.g.Khalf, tiles = sg.g.fwdTiles;
    __shared__ DF sh[8][RED_K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k = ((int64_t)blockIdx.x - sg.blockStart) * RED_K + lane;
    // compensated (Kahan) FP32 sum over this warp's tiles, then a double-float (two-sum)
    // combination of the 8 warps
    float sum = 0.f, comp = 0.f;
    auto kahan = [&](float v) {
        const float y = v - comp;
        const float u = sum + y;
        comp = (u - sum) - y;
        sum = u;
    };
    if (k < Khalf) {
        // this warp's tiles in order, their loads issued four at a time
        int64_t t = warp;
        for (; t + 24 < tiles; t += 32) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = sg.partial[(t + 8 * u) * Khalf + k];
#pragma unroll
            for (int u = 0; u < 4; ++u) kahan(v[u]);
        }
        for (; t < tiles; t += 8) kahan(sg.partial[t * Khalf + k]);
    }
    sh[warp][lane] = df_two_sum(sum, -comp);
    __syncthreads();
    if (warp == 0 && k < Khalf) {
        DF tot = sh[0][lane];
        for (int w = 1; w < 8; ++w) tot = df_add(tot, sh[w][lane]);
        sg.desc[k] = (tot.hi + tot.lo) * sg.scale;
    }
}

// ------------------------------------------------------------------------- adjoint

// lastValid: shifts of the chunk's last rx block inside the window (T unless the chunk ends
// the row and 2 P2 + 1 is not a multiple of T); block-uniform
template <int MODE>
__device__ __forceinline__ void adj_rows(const float* ys, const float* Gs, int strideP, int NB, int ryN, int lane,
                                         int strip, const float2 (&x2)[T], float2 (&acc)[T], int lastValid) {
    const int nFull = lastValid < T ? NB - 1 : NB;
    for (int r = 0; r < ryN; ++r) {
        const float* yrow = ys + (lane + r) * strideP + 2 * T * strip;
        const float4* grow = reinterpret_cast<const float4*>(Gs + r * (NB * GBLOCK));
#pragma unroll 1
        for (int bb = 0; bb < nFull; ++bb) {
            float2 y2[2 * T];
            load_pairs16(yrow + 2 * T * bb, y2);
            adj_block<MODE>(x2, y2, grow + (GBLOCK / 4) * bb, acc);
        }
        if (nFull < NB) {
            float2 y2[2 * T];
            load_pairs16(yrow + 2 * T * nFull, y2);
            adj_block<MODE, true>(x2, y2, grow + (GBLOCK / 4) * nFull, acc, lastValid);
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
    const float* __restrict__ tipf = sg.tip;
    const float* __restrict__ Gd = sg.Gd;
    float* __restrict__ part = sg.part;
    const int64_t local = (int64_t)blockIdx.x - sg.blockStart;
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31, strip = threadIdx.x >> 5;
    const int64_t tile = local % g.adjTiles;
    const int tx = (int)(tile % g.adjTilesX);
    const int ty = (int)((tile / g.adjTilesX) % g.adjTilesY);
    const int64_t z = tile / ((int64_t)g.adjTilesX * g.adjTilesY);
    const int64_t x0 = (int64_t)tx * TX, y0 = (int64_t)ty * ADJ_ROWS;
    const int64_t n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    // shift chunk: (rz range, ry range, rx-block range), rx blocks fastest
    const int chunk = (int)(local / g.adjTiles);
    const int xc = chunk % g.nXc, yc = (chunk / g.nXc) % g.nYc, zc = chunk / (g.nXc * g.nYc);
    const int rzA = -g.P[0] + zc * g.RZ;
    const int rzB = min(rzA + g.RZ, g.P[0] + 1);
    const int ryA = -g.P[1] + yc * g.RY;
    const int ryB = min(ryA + g.RY, g.P[1] + 1);
    const int bbA = xc * g.NBc;
    const int nbb = min(g.NBc, g.NB - bbA);
    const int lastValid = bbA + nbb == g.NB ? 2 * g.P[2] + 1 - T * (g.NB - 1) : T;
    const int colsH = T * nbb + 4 * T;      // read extent: 8 strip + 8 bb + 16 columns
    const int strideP = stride_4mod32(2 * colsH);
    // the chunk's ry rows are staged in rounds of at most RYS rows (pair row i of a round
    // holds halo rows i and i + 32); the accumulators carry over the rounds
    float* ys = smem;
    float* Gs = smem + (32 + g.RYS - 1) * strideP;
    const int64_t hx0 = x0 - g.P[2] + (int64_t)T * bbA;

    // own positions: rows y0 + lane and y0 + lane + 32, columns x0 + 8 strip + k
    const int64_t pyA = y0 + lane, pyB = pyA + 32;
    const float* xrowA = field + (z * n1 + (pyA < n1 ? pyA : 0)) * n2;
    const float* xrowB = field + (z * n1 + (pyB < n1 ? pyB : 0)) * n2;
    int xrc = 0;
#pragma unroll
    for (int k = 0; k < T; ++k) {
        const int64_t px = x0 + T * strip + k;
        if (px < n2) {
            if (pyA < n1) xrc |= out_of_range(tc, xrowA[px]);
            if (pyB < n1) xrc |= out_of_range(tc, xrowB[px]);
        }
    }
    float2 acc[T];
#pragma unroll
    for (int k = 0; k < T; ++k) acc[k] = make_float2(0.f, 0.f);

    const int rowG = nbb * GBLOCK;          // coefficient floats of one ry row of the chunk
    const int warp = threadIdx.x >> 5;
    constexpr int NW = ADJ_THREADS / 32;
    for (int rz = rzA; rz < rzB; ++rz)
    for (int ryS = ryA; ryS < ryB; ryS += g.RYS) {
        const int ryN = min(g.RYS, ryB - ryS);
        const int pairRows = 32 + ryN - 1;
        __syncthreads();
        const int64_t gz = wrap1(z + rz, n0);
        // raw halo (pair rows i, i + 32) and the chunk's coefficient rows, copied asynchronously
        for (int i = warp; i < pairRows; i += NW) {
            const float* srcA = tipf + (gz * n1 + wrap1(y0 + ryS + i, n1)) * n2;
            const float* srcB = tipf + (gz * n1 + wrap1(y0 + ryS + i + 32, n1)) * n2;
            float* dst = ys + i * strideP;
            int64_t gx = wrap1(hx0 + lane, n2);
            for (int c = lane; c < colsH; c += 32) {
                cp_async4(dst + 2 * c, srcA + gx);
                cp_async4(dst + 2 * c + 1, srcB + gx);
                gx += 32;
                while (gx >= n2) gx -= n2;
            }
        }
        const float* grow0 = Gd + (((int64_t)(rz + g.P[0]) * (2 * g.P[1] + 1) + (ryS + g.P[1])) * g.NB + bbA) * GBLOCK;
        for (int i = threadIdx.x; i < ryN * (rowG / 4); i += ADJ_THREADS) {
            const int r = i / (rowG / 4), c = i - r * (rowG / 4);
            cp_async16(Gs + r * rowG + 4 * c, grow0 + (int64_t)r * g.NB * GBLOCK + 4 * c);
        }
        cp_async_wait_own();
        // every thread transforms the halo entries it copied
        int rc = xrc;
        for (int i = warp; i < pairRows; i += NW) {
            float* dst = ys + i * strideP;
            for (int c = lane; c < colsH; c += 32) {
                const float2 v = *reinterpret_cast<const float2*>(dst + 2 * c);
                rc |= out_of_range(tc, v.x) | out_of_range(tc, v.y);
                float2 e;
                if (IDENT) e = make_float2(0.5f * v.x, 0.5f * v.y);
                else e = make_float2(tile_value<MODE_FAST>(tc, v.x, false), tile_value<MODE_FAST>(tc, v.y, false));
                *reinterpret_cast<float2*>(dst + 2 * c) = e;
            }
        }
        const int slow = __syncthreads_or(rc);
        if (!IDENT && slow) {
            for (int i = warp; i < pairRows; i += NW) {
                const float* srcA = tipf + (gz * n1 + wrap1(y0 + ryS + i, n1)) * n2;
                const float* srcB = tipf + (gz * n1 + wrap1(y0 + ryS + i + 32, n1)) * n2;
                float* dst = ys + i * strideP;
                int64_t gx = wrap1(hx0 + lane, n2);
                for (int c = lane; c < colsH; c += 32) {
                    *reinterpret_cast<float2*>(dst + 2 * c) = make_float2(
                        tile_value<MODE_SLOW>(tc, srcA[gx], false), tile_value<MODE_SLOW>(tc, srcB[gx], false));
                    gx += 32;
                    while (gx >= n2) gx -= n2;
                }
            }
        }
        // own values; positions outside the field hold 0 (d = 1) and are not written back
        float2 x2[T];
#pragma unroll
        for (int k = 0; k < T; ++k) {
            const int64_t px = x0 + T * strip + k;
            const float va = (pyA < n1 && px < n2) ? xrowA[px] : 0.f;
            const float vb = (pyB < n1 && px < n2) ? xrowB[px] : 0.f;
            if (IDENT) {
                x2[k] = make_float2(0.5f * va, 0.5f * vb);
            } else if (slow) {
                x2[k] = make_float2(tile_value<MODE_SLOW>(tc, va, true), tile_value<MODE_SLOW>(tc, vb, true));
            } else {
                x2[k] = make_float2((pyA < n1 && px < n2) ? tile_value<MODE_FAST>(tc, va, true) : 0.f,
                                    (pyB < n1 && px < n2) ? tile_value<MODE_FAST>(tc, vb, true) : 0.f);
            }
        }
        __syncthreads();
        if (IDENT) adj_rows<MODE_IDENT>(ys, Gs, strideP, nbb, ryN, lane, strip, x2, acc, lastValid);
        else if (slow) adj_rows<MODE_SLOW>(ys, Gs, strideP, nbb, ryN, lane, strip, x2, acc, lastValid);
        else adj_rows<MODE_FAST>(ys, Gs, strideP, nbb, ryN, lane, strip, x2, acc, lastValid);
    }

#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t py = h ? pyB : pyA;
        if (py >= n1) continue;
        float* out = part + (int64_t)chunk * g.N + (z * n1 + py) * n2;
#pragma unroll
        for (int k = 0; k < T; ++k) {
            const int64_t px = x0 + T * strip + k;
            // soft modes hold row lane in .y and row lane + 32 in .x (halves swapped)
            if (px < n2) out[px] = (h != 0) == IDENT ? acc[k].y : acc[k].x;
        }
    }
}

// Dense full-window coefficient grid of one level (one phase pair (a, b)), in adjoint order:
//   G(r) = scale * (src[k] - sub[k]) for r in the half window (k its canonical index),
//   G(r) = scale * (src2[k] - sub2[k]) for -r in it (k the index of -r),
//   G(0) = scale * ((src - sub) + (src2 - sub2))[0]   (2 (src - sub)[0] for one field),
//   scale = weight * (gscale from the loss, or 1) * (c1 alpha / N_l, or 1 / N_l for f(x)=x),
//   (A, B, C) = (-c1 G, (c1 - c3) G, c3 G)   (f(x) = x: (G, 0, 0)),
// zero where rx > P2 (padding of the last rx block).  Row (rz, ry) holds NB blocks of 8
// shifts; a block of GBLOCK = 48 floats stores (A, A, B, B) for m = 0..7 and then
// (C_m, C_m, C_m+1, C_m+1) for even m: both halves of a packed pair get the same coefficient.
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
        // dL/dS of one block entry; corrected descriptor: dL/dS_bar = A^T dL/dS_tilde (App. A
        // map, transposed)
        auto delta = [&](const float* src, const float* sub, int64_t k) {
            float d = src[k] - (sub != nullptr ? sub[k] : 0.f);
            if (sg.tsum != nullptr) d = k == 0 ? d - sg.q / (1.f - sg.q) * *sg.tsum : d / (1.f - sg.q);
            return d;
        };
        // r of the half window: block (a, b); -r of it: block (b, a) at r; r = 0 pairs the
        // position with itself in both blocks (2 dL/dS(0) for a = b)
        const int64_t k = canon_index(g, rz, ry, rx);
        float d;
        if (k == 0) d = delta(sg.src, sg.sub, 0) + delta(sg.src2, sg.sub2, 0);
        else if (k > 0) d = delta(sg.src, sg.sub, k);
        else d = delta(sg.src2, sg.sub2, canon_index(g, -rz, -ry, -rx));
        v = sg.scale * (sg.sc != nullptr ? sg.sc->gscale : 1.f) * d;
    }
    const int b = col / T, m = col % T;
    float A, B, C;
    if (tc.identity) { A = v; B = 0.f; C = 0.f; }
    else { A = -tc.c1 * v; B = (tc.c1 - tc.c3) * v; C = tc.c3 * v; }
    float* blk = sg.Gd + (row * g.NB + b) * GBLOCK;
    *reinterpret_cast<float4*>(blk + 4 * m) = make_float4(A, A, B, B);
    *reinterpret_cast<float2*>(blk + gblock_c(m)) = make_float2(C, C);
}

// ------------------------------------------------------------------------- launchers

size_t fwd_smem_bytes(const LevelGeom& g) {
    int maxFloats = 0;
    for (int gb = 0; gb < g.fwdGroupBlocks; ++gb) {
        const int64_t gfirst = (int64_t)gb * FWD_THREADS;
        const int64_t glast = std::min<int64_t>(gfirst + FWD_THREADS, g.NG) - 1;
        const GroupBox bx = group_box(g, gfirst, glast);
        const FwdSmem sh = fwd_smem_shape(g, bx);
        const int f = 2 * (g.TY * TX + 4) + sh.planesH * (sh.rowsH / 2) * sh.strideP;
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
    const int pairRows = 32 + g.RYS - 1;
    const int colsH = T * g.NBc + 4 * T;
    return (size_t)(pairRows * stride_4mod32(2 * colsH) + g.RYS * g.NBc * GBLOCK) * sizeof(float);
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
