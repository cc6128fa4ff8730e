// Pipe-rate probe: measured throughput of the instructions the correlation kernels are
// built from (MUFU reciprocal / exp2 / tanh / log2 and FP32 FMA), in operations per SM
// per clock.  Each thread runs 16 independent dependency chains at full occupancy; SM
// clocks are read with clock64 inside the kernel, so the rates do not depend on the clock
// the GPU happens to run at.  Used to derive the roofline peaks.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dmcr.h"

namespace {

constexpr int CH = 16;
constexpr int ITERS = 2048;

__device__ __forceinline__ float p_rcp(float x) { float y; asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float p_ex2(float x) { float y; asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float p_tanh(float x) { float y; asm volatile("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float p_lg2(float x) { float y; asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }

template <int OP>
__global__ void __launch_bounds__(256) probe_kernel(float* out, long long* cyc, float seed) {
    float r[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) r[i] = seed + 0.01f * i + 1e-6f * threadIdx.x;
    const long long t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < ITERS; ++it) {
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            if (OP == 0) r[i] = p_rcp(r[i] + 1.0f);          // FADD + MUFU.RCP
            else if (OP == 1) r[i] = p_ex2(-r[i]);            // MUFU.EX2
            else if (OP == 2) r[i] = p_tanh(r[i]);            // MUFU.TANH
            else if (OP == 3) r[i] = p_lg2(r[i] + 2.0f);      // FADD + MUFU.LG2
            else r[i] = fmaf(r[i], 0.999f, 0.001f);           // FFMA
        }
    }
    const long long t1 = clock64();
    float s = 0.f;
    for (int i = 0; i < CH; ++i) s += r[i];
    if (s == 12345.f) out[0] = s;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" dmcr_status dmcr_pipe_rates(double rates[5]) {
    int dev = 0, sms = 0;
    if (rates == nullptr) return DMCR_EINVAL;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DMCR_ECUDA;
    const int blocks = sms * 8;
    float* out = nullptr;
    long long* cyc = nullptr;
    if (cudaMalloc(&out, 4) != cudaSuccess) return DMCR_ECUDA;
    if (cudaMalloc(&cyc, blocks * sizeof(long long)) != cudaSuccess) {
        cudaFree(out);
        return DMCR_ECUDA;
    }
    long long* h = new long long[blocks];
    dmcr_status st = DMCR_OK;
    for (int op = 0; op < 5 && st == DMCR_OK; ++op) {
        for (int rep = 0; rep < 2; ++rep) {
            switch (op) {
                case 0: probe_kernel<0><<<blocks, 256>>>(out, cyc, 0.7f); break;
                case 1: probe_kernel<1><<<blocks, 256>>>(out, cyc, 0.7f); break;
                case 2: probe_kernel<2><<<blocks, 256>>>(out, cyc, 0.7f); break;
                case 3: probe_kernel<3><<<blocks, 256>>>(out, cyc, 0.7f); break;
                default: probe_kernel<4><<<blocks, 256>>>(out, cyc, 0.7f); break;
            }
        }
        if (cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(h, cyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess) {
            st = DMCR_ECUDA;
            break;
        }
        long long mx = 1;
        for (int i = 0; i < blocks; ++i) mx = h[i] > mx ? h[i] : mx;
        rates[op] = (double)blocks * 256.0 * ITERS * CH / sms / (double)mx;
    }
    delete[] h;
    cudaFree(out);
    cudaFree(cyc);
    return st;
}
