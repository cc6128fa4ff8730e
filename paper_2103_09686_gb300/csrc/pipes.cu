// Pipe-rate microbenchmark of the benchmark's roofline (not part of the dmcr C ABI; built
// as libdmcr_pipes.so and loaded by bench.py --pipes).  Measures, in operations per SM per
// clock, the instructions the correlation kernels are built from:
//   0 MUFU reciprocal (rcp.approx.ftz), 1 MUFU exp2, 2 MUFU tanh, 3 MUFU log2,
//   4 FP32 FFMA, 5 FP32 FFMA2 (lane operations: two per instruction),
//   6 the adjoint's pair arithmetic held in registers (pairs per SM per clock),
//   7 the forward's pair arithmetic held in registers (pairs per SM per clock),
//   8 FP64 DFMA (the FFT path's arithmetic).
// Every thread runs many independent chains (no chain waits on another), as many CTAs of
// 256 threads as fit on an SM at once (all resident together, so each CTA's cycle count
// spans the concurrent run), and each loop iteration carries at least 64 operations so the
// loop's own instructions are a few percent of the stream.  Cycles come from clock64
// inside the kernel, so the rates do not depend on the clock the GPU runs at.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int ITERS = 1024;

__device__ __forceinline__ float p_rcp(float x) { float y; asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float p_ex2(float x) { float y; asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float p_tanh(float x) { float y; asm volatile("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float p_lg2(float x) { float y; asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }

// operations per chain step counted by the host, per op kind
__host__ __device__ constexpr int chains(int op) {
    return op == 4 ? 32 : (op == 5 ? 16 : (op == 8 ? 16 : (op >= 6 ? 8 : 16)));
}

template <int OP>
__global__ void __launch_bounds__(256) pipe_kernel(float* out, long long* cyc, float seed) {
    constexpr int CH = chains(OP);
    float r[CH];
    float2 q[CH];
    double dq[OP == 8 ? CH : 1];
#pragma unroll
    for (int i = 0; i < CH; ++i) {
        r[i] = seed + 0.01f * i + 1e-6f * threadIdx.x;
        q[i] = make_float2(r[i], r[i] + 0.5f);
        if (OP == 8) dq[i] = (double)r[i];
    }
    const float2 a2 = make_float2(0.999f, 0.998f), b2 = make_float2(0.001f, 0.002f);
    const float2 one2 = make_float2(1.f, 1.f);
    const long long t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < ITERS; ++it) {
        if (OP <= 3) {
#pragma unroll
            for (int rep = 0; rep < 4; ++rep)
#pragma unroll
                for (int i = 0; i < CH; ++i) {
                    if (OP == 0) r[i] = p_rcp(r[i] + 1.0f);   // FADD keeps rcp(rcp(x)) from folding
                    else if (OP == 1) r[i] = p_ex2(-r[i]);
                    else if (OP == 2) r[i] = p_tanh(r[i]);
                    else r[i] = p_lg2(fabsf(r[i]));
                }
        } else if (OP == 4) {
#pragma unroll
            for (int rep = 0; rep < 2; ++rep)
#pragma unroll
                for (int i = 0; i < CH; ++i) r[i] = fmaf(r[i], 0.999f, 0.001f);
        } else if (OP == 5) {
#pragma unroll
            for (int rep = 0; rep < 4; ++rep)
#pragma unroll
                for (int i = 0; i < CH; ++i) q[i] = __ffma2_rn(q[i], a2, b2);
        } else if (OP == 6) {
            // per packed pair (two pairs): d = x y + 1, then either two reciprocals or a
            // shared one (product, rcp, FMUL2), then the Horner cubic with accumulation --
            // 4 of 8 positions of each kind, as in the adjoint kernel
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const float2 d = __ffma2_rn(q[i], a2, one2);
                float2 s;
                if (i < CH / 2) {
                    s = make_float2(p_rcp(d.y), p_rcp(d.x));
                } else {
                    const float rr = p_rcp(d.x * d.y);
                    s = __fmul2_rn(d, make_float2(rr, rr));
                }
                float2 h = __ffma2_rn(a2, s, b2);
                h = __ffma2_rn(h, s, a2);
                q[i] = __ffma2_rn(h, s, q[i]);
            }
        } else if (OP == 8) {
#pragma unroll
            for (int rep = 0; rep < 4; ++rep)
#pragma unroll
                for (int i = 0; i < CH; ++i) dq[i] = fma(dq[i], 0.999, 0.001);
        } else {
            // forward: d, shared reciprocal, u = s + beta, acc += u^2
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const float2 d = __ffma2_rn(q[i], a2, one2);
                const float rr = p_rcp(d.x * d.y);
                const float2 u = __ffma2_rn(d, make_float2(rr, rr), b2);
                q[i] = __ffma2_rn(u, u, q[i]);
            }
        }
    }
    const long long t1 = clock64();
    float s = 0.f;
    for (int i = 0; i < CH; ++i) s += r[i] + q[i].x + q[i].y;
    if (OP == 8)
        for (int i = 0; i < CH; ++i) s += (float)dq[i];
    if (s == 12345.f) out[0] = s;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

// operations one thread counts per loop iteration
constexpr double ops_per_iter(int op) {
    return op <= 3 ? 4.0 * 16 : (op == 4 ? 2.0 * 32 : (op == 5 ? 4.0 * 16 * 2 : (op == 8 ? 4.0 * 16 : 8.0 * 2)));
}

}  // namespace

// rates[0..8] as listed at the top (ops, lane operations or pairs per SM per clock);
// returns 0, or a CUDA error code.  Synchronous; allocates a few bytes of device memory.
extern "C" int dmcr_bench_pipe_rates(double rates[9]) {
    int dev = 0, sms = 0;
    if (rates == nullptr) return 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const void* kern[9] = {(const void*)pipe_kernel<0>, (const void*)pipe_kernel<1>, (const void*)pipe_kernel<2>,
                           (const void*)pipe_kernel<3>, (const void*)pipe_kernel<4>, (const void*)pipe_kernel<5>,
                           (const void*)pipe_kernel<6>, (const void*)pipe_kernel<7>, (const void*)pipe_kernel<8>};
    int per_sm[9];
    for (int op = 0; op < 9 && e == cudaSuccess; ++op) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[op], kern[op], 256, 0);
        if (e == cudaSuccess && per_sm[op] < 1) e = cudaErrorInvalidConfiguration;
    }
    if (e != cudaSuccess) return (int)e;
    const int blocks_max = sms * 8;
    float* out = nullptr;
    long long* cyc = nullptr;
    if ((e = cudaMalloc(&out, 4)) != cudaSuccess) return (int)e;
    if ((e = cudaMalloc(&cyc, blocks_max * sizeof(long long))) != cudaSuccess) {
        cudaFree(out);
        return (int)e;
    }
    long long* h = new long long[blocks_max];
    for (int op = 0; op < 9 && e == cudaSuccess; ++op) {
        const int blocks = sms * (per_sm[op] < 8 ? per_sm[op] : 8);
        for (int rep = 0; rep < 2; ++rep) {   // the first launch warms up
            switch (op) {
                case 0: pipe_kernel<0><<<blocks, 256>>>(out, cyc, 0.7f); break;
                case 1: pipe_kernel<1><<<blocks, 256>>>(out, cyc, 0.7f); break;
                case 2: pipe_kernel<2><<<blocks, 256>>>(out, cyc, 0.7f); break;
                case 3: pipe_kernel<3><<<blocks, 256>>>(out, cyc, 0.7f); break;
                case 4: pipe_kernel<4><<<blocks, 256>>>(out, cyc, 0.7f); break;
                case 5: pipe_kernel<5><<<blocks, 256>>>(out, cyc, 0.7f); break;
                case 6: pipe_kernel<6><<<blocks, 256>>>(out, cyc, 0.7f); break;
                case 7: pipe_kernel<7><<<blocks, 256>>>(out, cyc, 0.7f); break;
                default: pipe_kernel<8><<<blocks, 256>>>(out, cyc, 0.7f); break;
            }
        }
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) break;
        if ((e = cudaMemcpy(h, cyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost)) != cudaSuccess) break;
        long long mx = 1;
        for (int i = 0; i < blocks; ++i) mx = h[i] > mx ? h[i] : mx;
        rates[op] = (double)blocks * 256.0 * ITERS * ops_per_iter(op) / sms / (double)mx;
    }
    delete[] h;
    cudaFree(out);
    cudaFree(cyc);
    return (int)e;
}
