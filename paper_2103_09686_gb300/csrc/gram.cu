// Three-point descriptor (sm_103a): the quadratic reduction of the ensemble, Eq. s3,
//     S_bar3(r_a, r_b) = (1/N) sum_x e_x(r_a) e_x(r_b),   e_x(r) = f((M_x + M_{x+r}) / 2),
// i.e. the Gram matrix E^T E / N of the N x K ensemble (paper, Sec. 3.2.2-3.2.4 and the
// footnote of Sec. 3.4), and the gradient of a loss on it.
//
//   ens_kernel      e and f' never leave the chip except as the GEMM operands: E (N x K)
//                   and E^T (K x N), each split into two FP16 parts, e s = hi + lo with
//                   hi = fp16(e s), lo = fp16(e s - hi) (22 significant bits; s = 1 for the
//                   soft threshold, whose f is bounded, and a power of two bringing max |M|
//                   into [1/2, 1) for f(x) = x);
//   tc_gemm_kernel  C = A B^T on the 5th-generation tensor cores: tcgen05.mma kind::f16
//                   from shared memory, FP32 accumulators in TMEM drained every 256-512
//                   reduction steps into FP32 registers, three products
//                   hi*hi + hi*lo + lo*hi per k-step (the dropped lo*lo is below 2^-22 of the
//                   product), operands staged by TMA (128-byte swizzled K-major layout), one
//                   thread issues the MMAs and commits them to an mbarrier per stage; the
//                   epilogue undoes the operands' scales exactly;
//                   Gram:  S_bar3 = Et Et^T w/N (upper-triangle 128 x 128 tiles, mirrored,
//                          three 64 KB stages);
//                   W:     W^T = (2/N) G E^T  as  E G^T with a transposed epilogue (128 x 256
//                          tiles, two 96 KB stages);
//   g3_split_kernel G = w * gscale * (D3 - D3_des) symmetrised (or the upstream gradient),
//                   scaled by the power of two that brings max |G| (g3_absmax_kernel) into
//                   [1/2, 1), split like E;
//   s3_gather_kernel g_y = sum_r 1/2 [W(r, y) f'(a_y(r)) + W(r, y - r) f'(a_{y-r}(r))]
//                   (weight 1 at r = 0), the two ends of every shift vector.
// Every wait on an mbarrier is bounded; a timeout sets an error flag that the host reads.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "common.cuh"

namespace dmcr {

// C = scale * A B^T on the tensor cores (see tc_gemm_kernel): operands as TMA tensor maps
struct GemmArgs {
    CUtensorMap ta_hi, ta_lo, tb_hi, tb_lo;
    int M, N, K;
    float scale;
    const float* amaxA;     // operand scale sources (null: unscaled); C *= 2^(eA + eB)
    const float* amaxB;
    float* C;
    int64_t ldc;
    int mode;               // 1 symmetric Gram (upper tiles, mirrored), 2 C[n][m]
    int Mvalid, Nvalid;
    const int* done;
    int* err;
};

// the same with plain device pointers (host side)
struct GemmOperands {
    const uint16_t *Ah, *Al, *Bh, *Bl;   // FP16 bit patterns
    int64_t lda, ldb;
    int M, N, K;
    float scale;
    const float* amaxA;
    const float* amaxB;
    float* C;
    int64_t ldc;
    int mode;
    int Mvalid, Nvalid;
    const int* done;
    int* err;
};

namespace {

// Tiles of GM x BN outputs, BN = 128 or 256 (kernel template); GK reduction steps per stage.
constexpr int GM = 128, GK = 64;
constexpr int A_TILE = GM * GK * 2;                    // one FP16 A tile (128 rows of 128 bytes), 16 KB
template <int BN>
struct GemmShape {
    static constexpr int B_TILE = BN * GK * 2;                   // one FP16 B tile
    static constexpr int STAGE_BYTES = 2 * A_TILE + 2 * B_TILE;  // A hi, A lo, B hi, B lo
    static constexpr int STAGES = BN == 128 ? 3 : 2;             // 192 KB of stages
    static constexpr int EPI_WARPS = BN / 32;                    // 128 columns of one lane quadrant each
    static constexpr int THREADS = 32 * (EPI_WARPS + 2);         // epilogue warps, then TMA, then MMA
    // 128-wide tiles keep the small cross terms hi*lo + lo*hi in an accumulator of their own
    // (FLUSH 8 k-blocks: 32 MMAs per accumulator); 256-wide tiles add all three products into
    // one accumulator (TMEM holds two buffers of 256 columns) and drain twice as often
    static constexpr bool SPLIT = BN == 128;
    static constexpr int FLUSH = SPLIT ? 8 : 4;
    static constexpr uint32_t BUF_COLS = SPLIT ? 2 * BN : BN;     // one buffer: main (+ cross)
    static constexpr uint32_t TMEM_COLS = 2 * BUF_COLS;          // 512 columns, 128 lanes
    // instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B F16 (bits 7-9, 10-12 = 0),
    // both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
    static constexpr uint32_t IDESC = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(GM >> 4) << 24);
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
};
// The tensor core adds into its FP32 accumulator without round-to-nearest: over a long
// reduction the error is biased toward zero (~4e-8 relative per accumulation measured on
// GB300).  So TMEM accumulates at most FLUSH k-blocks (GemmShape) before the partial sums are
// added, rounded to nearest, into FP32 registers.
constexpr uint32_t WAIT_LIMIT = 1u << 22;


__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// 2-D tiled TMA load of one box into shared memory, completion counted on an mbarrier
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// bounded wait for the completion of the mbarrier phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t addr = smem_u32(bar);
    for (uint32_t i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// whole warp: allocate TMEM columns, address written to shared memory
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// shared-memory matrix descriptor, K-major with the 128-byte swizzle: each operand row is
// one 128-byte line (64 FP16) whose 16-byte chunks are stored at chunk ^ (row % 8); atoms of
// 8 rows (1024 bytes, 1024-byte aligned) follow each other at SBO = 1024; LBO is unused by
// this layout (encoded 1); descriptor version 1, layout type 2 (SWIZZLE_128B).  A k-step of
// 16 FP16 starts 32 bytes further into the line.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 lanes x 16 columns of 32 bits: thread i of the warp gets lane (lane base + i)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// x = hi + lo to 22 significant bits (both FP16, round to nearest)
__device__ __forceinline__ void split_f16(float x, uint16_t& hi, uint16_t& lo) {
    const __half h = __float2half_rn(x);
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
}

// exponent e of the scale 2^-e that maps max |x| = *amax into [1/2, 1); 0 without a source,
// for 0 and for non-finite maxima
__device__ __forceinline__ int scale_exp(const float* amax) {
    if (amax == nullptr) return 0;
    const float a = *amax;
    if (!(a > 0.f) || !isfinite(a)) return 0;
    int e;
    frexpf(a, &e);
    return e;
}

}  // namespace

// ------------------------------------------------------------------------- GEMM

// C = scale 2^(eA + eB) A B^T with A (M x K) and B (N x K) row-major (K contiguous), each given
// as FP16 hi + lo through four TMA tensor maps (boxes 64 x 128 for A, 64 x BN for B, 128-byte
// swizzle).  M a multiple of 128, N of BN, K of 64.  Tiles are 128 x BN.  mode 1 (Gram, A = B,
// square tiles, BN = 128): only tiles bn >= bm, written to C[m][n] and C[n][m]; mode 2:
// C[n][m].  Entries with m >= Mvalid or n >= Nvalid are not written.
//
// The single issuing thread spends about 400 cycles per stage besides the MMAs (barrier
// wait, commit, loop): 128 x 256 tiles (twice the MMA work per stage) keep the tensor pipe
// fed where the grid is large (the W GEMM); the Gram, whose upper triangle holds few tiles,
// keeps 128 x 128 tiles so that it fills the SMs.
//
// Warp roles: warp EPI (one lane) loads the stages with TMA; warp EPI + 1 (one lane) issues
// the MMAs and commits them; warps 0 .. EPI - 1 drain the TMEM accumulators every FLUSH
// k-blocks into FP32 registers (warp w reads TMEM lanes 32 (w % 4) .. + 31 and columns
// 128 (w / 4) .. + 127; TMEM is double-buffered, two periods of BN columns) and write the
// tile.  Barriers: full[s] (TMA bytes landed), empty[s] (MMAs done reading stage s),
// tfull[b] (period finished in TMEM buffer b), tempty[b] (buffer b read).
template <int BN>
__global__ void __launch_bounds__(GemmShape<BN>::THREADS, 1) tc_gemm_kernel(const __grid_constant__ GemmArgs g) {
    using S = GemmShape<BN>;
    constexpr int GN = BN, GSTAGES = S::STAGES, STAGE_BYTES = S::STAGE_BYTES, B_TILE = S::B_TILE;
    constexpr int EPI_WARPS = S::EPI_WARPS, FLUSH = S::FLUSH;
    constexpr uint32_t TMEM_COLS = S::TMEM_COLS;
    if (g.done != nullptr && *g.done) return;
    extern __shared__ __align__(1024) uint8_t gsm_raw[];
    // the swizzle atoms need 1024-byte aligned tiles
    uint8_t* gsm = gsm_raw + ((1024 - (smem_u32(gsm_raw) & 1023)) & 1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(gsm + GSTAGES * STAGE_BYTES);
    uint64_t* empty = full + GSTAGES;
    uint64_t* tfull = empty + GSTAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* mdone = tempty + 2;   // every MMA of this CTA finished (the last commit)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mdone + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tilesM = g.M / GM, tilesN = g.N / GN;
    int bm, bn;
    if (g.mode == 1) {
        // the upper triangle in square tiles (the launcher takes BN = GM), row by row: (bm, bn >= bm)
        int t = (int)blockIdx.x;
        bm = 0;
        while (t >= tilesN - bm) {
            t -= tilesN - bm;
            ++bm;
        }
        bn = bm + t;
    } else {
        // B tiles fastest: the CTAs in flight share a few A row blocks and sweep the whole of
        // B (the W GEMM's G, Kpad x Kpad, stays in L2), so A streams from DRAM once
        bn = (int)(blockIdx.x % tilesN);
        bm = (int)(blockIdx.x / tilesN);
    }
    if (tid == 0) {
        for (int s = 0; s < GSTAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], EPI_WARPS * 32);
        }
        mbar_init(mdone, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == EPI_WARPS + 1) tmem_alloc(tslot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const int nk = g.K / GK;
    const int nper = (nk + FLUSH - 1) / FLUSH;
    bool ok = true;

    if (warp == EPI_WARPS) {
        // ---- TMA producer
        if (lane == 0) {
            int issued = 0;   // stages whose copies were started
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % GSTAGES;
                if (kb >= GSTAGES) ok = mbar_wait(&empty[s], ((kb / GSTAGES) - 1) & 1);
                if (!ok) break;
                uint8_t* st = gsm + s * STAGE_BYTES;
                mbar_expect_tx(&full[s], STAGE_BYTES);
                const int k0 = kb * GK;
                tma_load_2d(st, &g.ta_hi, k0, bm * GM, &full[s]);
                tma_load_2d(st + A_TILE, &g.ta_lo, k0, bm * GM, &full[s]);
                tma_load_2d(st + 2 * A_TILE, &g.tb_hi, k0, bn * GN, &full[s]);
                tma_load_2d(st + 2 * A_TILE + B_TILE, &g.tb_lo, k0, bn * GN, &full[s]);
                issued = kb + 1;
            }
            // no copy of this CTA may still be in flight when it exits, after a give-up as
            // well: wait (bounded) for the bytes of the stages it actually started.  Each
            // stage's barrier has begun no phase after the one waited on here, so the
            // parity is unambiguous.
            for (int kb = issued > GSTAGES ? issued - GSTAGES : 0; kb < issued; ++kb)
                if (!mbar_wait(&full[kb % GSTAGES], (kb / GSTAGES) & 1)) ok = false;
        }
        __syncwarp();
    } else if (warp == EPI_WARPS + 1) {
        // ---- MMA issuer
        if (lane == 0) {
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % GSTAGES;
                const int p = kb / FLUSH, buf = p & 1;
                // TMEM buffer buf was last used by period p - 2: wait until it was read
                if (kb % FLUSH == 0 && p >= 2) ok = mbar_wait(&tempty[buf], ((p / 2) - 1) & 1);
                if (ok) ok = mbar_wait(&full[s], (kb / GSTAGES) & 1);
                if (!ok) break;
                tc_fence_after();
                const uint32_t st = smem_u32(gsm + s * STAGE_BYTES);
                const uint32_t t_acc = tmem + (uint32_t)buf * S::BUF_COLS;
                const uint32_t t_cross = S::SPLIT ? t_acc + GN : t_acc;
#pragma unroll
                for (int ks = 0; ks < GK / 16; ++ks) {
                    const uint32_t off = ks * 32;   // 16 FP16 = 32 bytes per k-step
                    const uint64_t ah = smem_desc_sw128(st + off);
                    const uint64_t al = smem_desc_sw128(st + A_TILE + off);
                    const uint64_t bh = smem_desc_sw128(st + 2 * A_TILE + off);
                    const uint64_t bl = smem_desc_sw128(st + 2 * A_TILE + B_TILE + off);
                    const uint32_t more = (kb % FLUSH != 0) || ks != 0;
                    mma_f16(t_acc, ah, bh, S::IDESC, more);
                    mma_f16(t_cross, ah, bl, S::IDESC, S::SPLIT ? more : 1u);
                    mma_f16(t_cross, al, bh, S::IDESC, 1);
                }
                mma_commit(&empty[s]);
                if (kb % FLUSH == FLUSH - 1 || kb == nk - 1) mma_commit(&tfull[buf]);
            }
            // TMEM is freed below: first every MMA issued above (all of them, also after a
            // give-up of this thread or of another role) must have finished writing it.  A
            // commit tracks every earlier tcgen05 operation of this thread.
            mma_commit(mdone);
            if (!mbar_wait(mdone, 0)) ok = false;
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp w owns TMEM lanes 32 (w % 4) .. + 31 (tile rows) and the 128
        // columns from 128 (w / 4)
        constexpr int EC = 128;
        const int quad = warp & 3, half = warp >> 2;
        float acc[EC];
#pragma unroll
        for (int c = 0; c < EC; ++c) acc[c] = 0.f;
        for (int p = 0; p < nper; ++p) {
            const int buf = p & 1;
            // warp-uniform decision: tcgen05.ld below is .sync.aligned
            ok = __all_sync(0xffffffffu, mbar_wait(&tfull[buf], (p / 2) & 1));
            if (!ok) break;
            tc_fence_after();
            const uint32_t t_acc =
                tmem + (uint32_t)buf * S::BUF_COLS + (uint32_t)(EC * half) + ((uint32_t)(32 * quad) << 16);
#pragma unroll
            for (int c = 0; c < EC; c += 16) {
                float v[16];
                tmem_ld16(t_acc + (uint32_t)c, v);
                if (S::SPLIT) {
                    float w[16];
                    tmem_ld16(t_acc + GN + (uint32_t)c, w);
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc[c + j] += v[j] + w[j];
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc[c + j] += v[j];
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty[buf]);
        }
        const int m = bm * GM + 32 * quad + lane;
        // undo the operands' power-of-two scales together with the output scale (exact)
        const float scale = ldexpf(g.scale, scale_exp(g.amaxA) + scale_exp(g.amaxB));
        if (ok && m < g.Mvalid) {
#pragma unroll
            for (int c = 0; c < EC; ++c) {
                const int n = bn * GN + EC * half + c;
                if (n >= g.Nvalid) continue;
                const float x = scale * acc[c];
                if (g.mode == 2) {
                    g.C[(int64_t)n * g.ldc + m] = x;
                } else {
                    // Gram: a diagonal tile holds both halves; the others are mirrored
                    g.C[(int64_t)m * g.ldc + n] = x;
                    if (bm != bn) g.C[(int64_t)n * g.ldc + m] = x;
                }
            }
        }
    }
    if (!ok && g.err != nullptr) atomicExch(g.err, 1);
    // the MMA issuer reaches this barrier only after its last commit arrived (or its bounded
    // wait for it ran out), and the epilogue warps after their last TMEM read
    tc_fence_before();
    __syncthreads();
    if (warp == EPI_WARPS + 1) tmem_dealloc(tmem, TMEM_COLS);
}

// ------------------------------------------------------------------------- ensemble

// shift k of the canonical half window -> (rz, ry, rx); inverse of canon_index (32-bit: the
// half window holds at most 2^14 shifts here)
__device__ __forceinline__ void decode_shift(const LevelGeom& g, int k, int& rz, int& ry, int& rx) {
    const int Px = g.P[2], Py = g.P[1];
    const int wx = 2 * Px + 1, wy = 2 * Py + 1;
    if (k <= Px) {
        rz = 0; ry = 0; rx = k;
        return;
    }
    k -= Px + 1;
    if (k < Py * wx) {
        rz = 0; ry = 1 + k / wx; rx = k % wx - Px;
        return;
    }
    k -= Py * wx;
    rz = 1 + k / (wy * wx);
    k %= wy * wx;
    ry = k / wx - Py;
    rx = k % wx - Px;
}

// position coordinates of a level (z, y, c), 32-bit (levels hold < 2^31 positions)
struct Pos3 {
    int z, y, c;
};

__device__ __forceinline__ Pos3 pos_of(const LevelGeom& g, int64_t x) {
    const int n12 = (int)(g.n[1] * g.n[2]), n2 = (int)g.n[2];
    const int xi = (int)x;
    Pos3 p;
    p.z = xi / n12;
    const int r = xi - p.z * n12;
    p.y = r / n2;
    p.c = r - p.y * n2;
    return p;
}

// v + d wrapped into [0, n) for |d| <= n (windows never exceed half a level)
__device__ __forceinline__ int wrap_add(int v, int d, int n) {
    int w = v + d;
    w = w >= n ? w - n : w;
    return w < 0 ? w + n : w;
}

// linear index of p + (rz, ry, rx), periodic
__device__ __forceinline__ int64_t partner(const LevelGeom& g, const Pos3& p, int rz, int ry, int rx) {
    const int n0 = (int)g.n[0], n1 = (int)g.n[1], n2 = (int)g.n[2];
    return ((int64_t)wrap_add(p.z, rz, n0) * n1 + wrap_add(p.y, ry, n1)) * n2 + wrap_add(p.c, rx, n2);
}

// s = sigma(alpha (a - 0.75)) for a = (u + v) / 2, exact form (any finite range)
__device__ __forceinline__ float sig_pair(const ThreshConst& tc, float u, float v) {
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(fmaf(-tc.kappa, u + v, tc.cexp)));
    float s;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(e + 1.0f));
    return s;
}

// one block: 64 positions x 32 shifts.  Thread (tx, ty) owns positions x0 + 2 tx and
// x0 + 2 tx + 1 and shifts k0 + ty + 8 i (i = 0..3).  E^T rows (shift-major) are written as
// pairs of positions, one 32-bit word per thread (128-byte lines per warp); E rows
// (position-major) go through a shared transpose and are written as pairs of shifts.
// Padding entries are 0.
__global__ void __launch_bounds__(256) ens_kernel(S3Job j, ThreshConst tc) {
    if (j.done != nullptr && *j.done) return;
    __shared__ uint16_t th[64][34], tl[64][34];
    __shared__ int3 shifts[32];
    const LevelGeom& g = j.g;
    // f(x) = x: e is bounded by max |M|, scaled into [-1, 1); the soft f is bounded by ~1.03
    const float sE = ldexpf(1.f, -(tc.identity ? scale_exp(j.amax + 1) : 0));
    const int64_t x0 = (int64_t)(blockIdx.x % (j.Npad / 64)) * 64;
    const int64_t k0 = (int64_t)(blockIdx.x / (j.Npad / 64)) * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    if (threadIdx.x < 32 && k0 + threadIdx.x < j.K) {
        int rz, ry, rx;
        decode_shift(g, (int)(k0 + threadIdx.x), rz, ry, rx);
        shifts[threadIdx.x] = make_int3(rz, ry, rx);
    }
    __syncthreads();
    const int64_t xa = x0 + 2 * tx;
    const bool ina = xa < g.N, inb = xa + 1 < g.N;
    const Pos3 pa = pos_of(g, ina ? xa : 0), pb = pos_of(g, inb ? xa + 1 : 0);
    const float ua = ina ? j.field[xa] : 0.f, ub = inb ? j.field[xa + 1] : 0.f;
    uint32_t* Eth = reinterpret_cast<uint32_t*>(j.Eth);
    uint32_t* Etl = reinterpret_cast<uint32_t*>(j.Etl);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int kk = ty + 8 * i;
        const int64_t k = k0 + kk;
        float ea = 0.f, eb = 0.f;
        if (k < j.K) {
            const int3 r = shifts[kk];
            if (ina) {
                const float v = j.field[partner(g, pa, r.x, r.y, r.z)];
                ea = tc.identity ? 0.5f * (ua + v) : fmaf(tc.c1, sig_pair(tc, ua, v), tc.c3);
            }
            if (inb) {
                const float v = j.field[partner(g, pb, r.x, r.y, r.z)];
                eb = tc.identity ? 0.5f * (ub + v) : fmaf(tc.c1, sig_pair(tc, ub, v), tc.c3);
            }
        }
        uint16_t ha, la, hb, lb;
        split_f16(ea * sE, ha, la);
        split_f16(eb * sE, hb, lb);
        // the lower address holds the lower 16 bits (little endian)
        Eth[(k * j.Npad + xa) / 2] = (uint32_t)ha | ((uint32_t)hb << 16);
        Etl[(k * j.Npad + xa) / 2] = (uint32_t)la | ((uint32_t)lb << 16);
        th[2 * tx][kk] = ha;
        th[2 * tx + 1][kk] = hb;
        tl[2 * tx][kk] = la;
        tl[2 * tx + 1][kk] = lb;
    }
    __syncthreads();
    // E rows: 64 positions x 16 words of shift pairs
    uint32_t* Eh = reinterpret_cast<uint32_t*>(j.Eh);
    uint32_t* El = reinterpret_cast<uint32_t*>(j.El);
    const int w = threadIdx.x & 15;
    for (int pp = threadIdx.x >> 4; pp < 64; pp += 16) {
        const int64_t o = ((x0 + pp) * j.Kpad + k0) / 2 + w;
        Eh[o] = (uint32_t)th[pp][2 * w] | ((uint32_t)th[pp][2 * w + 1] << 16);
        El[o] = (uint32_t)tl[pp][2 * w] | ((uint32_t)tl[pp][2 * w + 1] << 16);
    }
}

// G(a, b) = w * gscale * sym(D3 - D3_des) on the level's K x K block; d<G, E^T E>/dE =
// E (G + G^T), so G is symmetrised (the loss gradient already is symmetric).  A block holds
// a 32 x 32 tile; the transposed entries come through shared memory, so both reads are
// coalesced.  Returns v(a0 + i, b0 + tx) for i = ty, ty + 8, ... in v[4] (0 outside K x K).
__device__ __forceinline__ float g3_delta(const S3Job& j, int64_t a, int64_t b) {
    return j.src[a * j.K + b] - (j.sub != nullptr ? j.sub[a * j.K + b] : 0.f);
}

__device__ __forceinline__ void g3_tile(const S3Job& j, int64_t a0, int64_t b0, float (&v)[4]) {
    __shared__ float tt[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int i = ty; i < 32; i += 8) {
        const int64_t b = b0 + i, a = a0 + tx;
        tt[tx][i] = (a < j.K && b < j.K) ? g3_delta(j, b, a) : 0.f;   // tt[a - a0][b - b0] = d(b, a)
    }
    __syncthreads();
    const float sc = j.weight * (j.sc != nullptr ? j.sc->gscale : 1.f);
    for (int q = 0; q < 4; ++q) {
        const int i = ty + 8 * q;
        const int64_t a = a0 + i, b = b0 + tx;
        v[q] = (a < j.K && b < j.K) ? sc * 0.5f * (g3_delta(j, a, b) + tt[i][tx]) : 0.f;
    }
}

// max |v| of a block's values into *out (non-negative floats order like their bit patterns;
// *out starts at 0)
__device__ __forceinline__ void block_absmax(float m, float* out) {
    __shared__ float sh[8];
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, sh[w]);
        atomicMax(reinterpret_cast<int*>(out), __float_as_int(m));
    }
}

// one 32 x 32 tile of G per block
__global__ void __launch_bounds__(256) g3_absmax_kernel(S3Job j) {
    if (j.done != nullptr && *j.done) return;
    const int64_t tiles = (j.K + 31) / 32;
    float v[4];
    g3_tile(j, (blockIdx.x / tiles) * 32, (blockIdx.x % tiles) * 32, v);
    float m = 0.f;
    for (int q = 0; q < 4; ++q) m = fmaxf(m, fabsf(v[q]));
    block_absmax(m, j.amax);
}

// f(x) = x: max |M| of the level's field, the bound of |e|
__global__ void __launch_bounds__(256) field_absmax_kernel(S3Job j) {
    if (j.done != nullptr && *j.done) return;
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < j.g.N; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(j.field[i]));
    block_absmax(m, j.amax + 1);
}

// G scaled by 2^-eG (max |G| into [1/2, 1)) and split into FP16 hi + lo, one 32 x 32 tile of
// Kpad x Kpad per block (zero padding)
__global__ void __launch_bounds__(256) g3_split_kernel(S3Job j) {
    if (j.done != nullptr && *j.done) return;
    const int64_t tiles = j.Kpad / 32;
    const int64_t a0 = (blockIdx.x / tiles) * 32, b0 = (blockIdx.x % tiles) * 32;
    float v[4];
    g3_tile(j, a0, b0, v);
    const int eG = scale_exp(j.amax);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int q = 0; q < 4; ++q) {
        const int64_t i = (a0 + ty + 8 * q) * j.Kpad + b0 + tx;
        uint16_t hi, lo;
        split_f16(ldexpf(v[q], -eG), hi, lo);
        j.Gh[i] = hi;
        j.Gl[i] = lo;
    }
}

// g_y = sum_k c_k [W(k, y) f'(a_y(r_k)) + W(k, y - r_k) f'(a_{y - r_k}(r_k))], c_0 = 1/2 (the two
// terms coincide at r = 0), c_k = 1/2 otherwise; f' = c1 alpha s (1 - s), or 1 for f(x) = x.
// Block (position block, shift chunk of S3_SHIFTS): per-chunk partials, summed in a fixed order
// by the gradient assembly.
__global__ void __launch_bounds__(256) s3_gather_kernel(S3Job j, ThreshConst tc) {
    if (j.done != nullptr && *j.done) return;
    const LevelGeom& g = j.g;
    const int64_t y = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= g.N) return;
    const int64_t kA = (int64_t)blockIdx.y * S3_SHIFTS;
    const int64_t kB = min(kA + (int64_t)S3_SHIFTS, j.K);
    const float c1a = tc.c1 * tc.alpha;
    const float my = j.field[y];
    const Pos3 py = pos_of(g, y);
    float acc = 0.f;
    // the chunk's shifts in canonical order: rx fastest, then ry, then rz (decoded once); the
    // partner indices y + r and y - r are stepped along rx and rebuilt when (rz, ry) changes;
    // four shifts per step, their loads issued together
    int rz, ry, rx;
    decode_shift(g, (int)kA, rz, ry, rx);
    const float* __restrict__ field = j.field;
    const float* __restrict__ W = j.W;
    const int n0 = (int)g.n[0], n1 = (int)g.n[1], n2 = (int)g.n[2];
    int64_t rowp = 0, rowm = 0;
    int cp = 0, cm = 0;
    auto rows = [&]() {
        rowp = ((int64_t)wrap_add(py.z, rz, n0) * n1 + wrap_add(py.y, ry, n1)) * n2;
        rowm = ((int64_t)wrap_add(py.z, -rz, n0) * n1 + wrap_add(py.y, -ry, n1)) * n2;
    };
    rows();
    cp = wrap_add(py.c, rx, n2);
    cm = wrap_add(py.c, -rx, n2);
    constexpr int U = 4;
    for (int64_t k0 = kA; k0 < kB; k0 += U) {
        int64_t ym[U];
        float vp[U], vm[U], w1[U], w2[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool in = k0 + u < kB;
            const int64_t k = in ? k0 + u : kA;
            const int64_t yp = rowp + cp;                       // y + r
            ym[u] = rowm + cm;                                  // y - r
            vp[u] = field[yp];
            vm[u] = field[ym[u]];
            w1[u] = in ? W[k * j.Npad + y] : 0.f;
            w2[u] = in ? W[k * j.Npad + ym[u]] : 0.f;
            if (++rx > g.P[2]) {
                rx = -g.P[2];
                if (++ry > g.P[1]) {
                    ry = -g.P[1];
                    ++rz;
                }
                rows();
                cp = wrap_add(py.c, rx, n2);
                cm = wrap_add(py.c, -rx, n2);
            } else {
                cp = cp + 1 == n2 ? 0 : cp + 1;
                cm = cm == 0 ? n2 - 1 : cm - 1;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float d1 = 1.f, d2 = 1.f;
            if (!tc.identity) {
                const float s1 = sig_pair(tc, my, vp[u]);
                const float s2 = sig_pair(tc, vm[u], my);
                d1 = c1a * s1 * (1.f - s1);
                d2 = c1a * s2 * (1.f - s2);
            }
            acc = fmaf(0.5f * w1[u], d1, acc);
            acc = fmaf(0.5f * w2[u], d2, acc);
        }
    }
    j.part[(int64_t)blockIdx.y * g.N + y] = acc;
}

// ------------------------------------------------------------------------- launchers

size_t gemm_smem_bytes() { return std::max(GemmShape<128>::SMEM, GemmShape<256>::SMEM); }

void set_gram_attributes() {
    cudaFuncSetAttribute(tc_gemm_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GemmShape<128>::SMEM);
    cudaFuncSetAttribute(tc_gemm_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GemmShape<256>::SMEM);
}

__global__ void set_flag_kernel(int* flag, int v) {
    if (flag != nullptr) *flag = v;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// rows x cols FP16 row-major (row stride ld elements), boxes of box_rows rows x 64 columns
bool make_map(CUtensorMap* m, const uint16_t* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (enc == nullptr) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(uint16_t)};
    const cuuint32_t box[2] = {(cuuint32_t)GK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<uint16_t*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool gram_ready() { return tensor_map_encoder() != nullptr; }

// BN = 128 for the Gram (mode 1), 256 otherwise
void launch_tc_gemm(const GemmOperands& o, cudaStream_t s) {
    const int BN = o.mode == 1 ? 128 : 256;
    const int64_t tm = o.M / GM, tn = o.N / BN;
    int64_t blocks = tm * tn;
    if (o.mode == 1) blocks = tm * (tm + 1) / 2;   // square tiles: BN = 128, M = N
    if (blocks <= 0) return;
    GemmArgs a{};
    const bool ok = make_map(&a.ta_hi, o.Ah, o.M, o.K, o.lda, GM) && make_map(&a.ta_lo, o.Al, o.M, o.K, o.lda, GM) &&
                    make_map(&a.tb_hi, o.Bh, o.N, o.K, o.ldb, BN) && make_map(&a.tb_lo, o.Bl, o.N, o.K, o.ldb, BN);
    if (!ok) {
        // no valid tensor map: never launch TMA on it; report through the error word
        set_flag_kernel<<<1, 1, 0, s>>>(o.err, 2);
        return;
    }
    a.M = o.M; a.N = o.N; a.K = o.K;
    a.scale = o.scale;
    a.amaxA = o.amaxA;
    a.amaxB = o.amaxB;
    a.C = o.C;
    a.ldc = o.ldc;
    a.mode = o.mode;
    a.Mvalid = o.Mvalid; a.Nvalid = o.Nvalid;
    a.done = o.done;
    a.err = o.err;
    if (BN == 128)
        tc_gemm_kernel<128><<<(unsigned)blocks, GemmShape<128>::THREADS, GemmShape<128>::SMEM, s>>>(a);
    else
        tc_gemm_kernel<256><<<(unsigned)blocks, GemmShape<256>::THREADS, GemmShape<256>::SMEM, s>>>(a);
}

constexpr int ABSMAX_BLOCKS = 512;

// E and E^T of one level (f(x) = x: after the bound of |e|)
void launch_ensemble(const S3Job& j, const ThreshConst& tc, cudaStream_t s) {
    if (tc.identity) {
        set_flag_kernel<<<1, 1, 0, s>>>(reinterpret_cast<int*>(j.amax + 1), 0);
        const int64_t blocks = std::min<int64_t>(ABSMAX_BLOCKS, (j.g.N + 255) / 256);
        field_absmax_kernel<<<(unsigned)blocks, 256, 0, s>>>(j);
    }
    ens_kernel<<<(unsigned)((j.Npad / 64) * (j.Kpad / 32)), 256, 0, s>>>(j, tc);
}

void launch_s3_forward(const S3Job& j, const ThreshConst& tc, int* err, cudaStream_t s) {
    launch_ensemble(j, tc, s);
    GemmOperands a{};
    a.Ah = j.Eth; a.Al = j.Etl; a.Bh = j.Eth; a.Bl = j.Etl;
    a.amaxA = a.amaxB = tc.identity ? j.amax + 1 : nullptr;
    a.lda = a.ldb = j.Npad;
    a.M = a.N = (int)j.Kpad;
    a.K = (int)j.Npad;
    a.scale = (float)((double)j.weight / (double)j.g.N);
    a.C = j.desc;
    a.ldc = j.K;
    a.mode = 1;
    a.Mvalid = a.Nvalid = (int)j.K;
    a.done = j.done;
    a.err = err;
    launch_tc_gemm(a, s);
}

void launch_s3_backward(const S3Job& j, const ThreshConst& tc, int* err, cudaStream_t s) {
    if (j.ens) launch_ensemble(j, tc, s);
    set_flag_kernel<<<1, 1, 0, s>>>(reinterpret_cast<int*>(j.amax), 0);
    const int64_t tk = (j.K + 31) / 32;
    g3_absmax_kernel<<<(unsigned)(tk * tk), 256, 0, s>>>(j);
    g3_split_kernel<<<(unsigned)((j.Kpad / 32) * (j.Kpad / 32)), 256, 0, s>>>(j);
    GemmOperands a{};
    a.Ah = j.Eh; a.Al = j.El; a.Bh = j.Gh; a.Bl = j.Gl;
    a.amaxA = tc.identity ? j.amax + 1 : nullptr;
    a.amaxB = j.amax;
    a.lda = j.Kpad;
    a.ldb = j.Kpad;
    a.M = (int)j.Npad;
    a.N = (int)j.Kpad;
    a.K = (int)j.Kpad;
    a.scale = (float)(2.0 / (double)j.g.N);
    a.C = j.W;
    a.ldc = j.Npad;
    a.mode = 2;
    a.Mvalid = (int)j.Npad;
    a.Nvalid = (int)j.Kpad;
    a.done = j.done;
    a.err = err;
    launch_tc_gemm(a, s);
    const dim3 grid((unsigned)((j.g.N + 255) / 256), (unsigned)((j.K + S3_SHIFTS - 1) / S3_SHIFTS));
    s3_gather_kernel<<<grid, 256, 0, s>>>(j, tc);
}

}  // namespace dmcr
