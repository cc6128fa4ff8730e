// FFT path of the descriptor (sm_103a): the periodic autocorrelation
//     C(r) = (1/N) sum_x M_x M_{x+r} = (1/N) IDFT( |DFT(M)|^2 )(r)
// gives, exactly up to rounding,
//   * the identity-threshold descriptor (f(x) = x, the ablation of Sec. 4.1):
//         S_bar(r) = ( <M^2> + C(r) ) / 2,   <M^2> = C(0);
//   * the soft-threshold descriptor of a BINARY field (App. A):
//         S_bar(r) = (1 - 2 f(1/2)^2) C(r) + 2 f(1/2)^2 C(0)  (r != 0),   S_bar(0) = C(0),
//     used to characterise binary targets;
// and the identity-threshold adjoint as one cross-correlation,
//         g(y) = ( M_y sum_r A(r) + sum_r A(r) M_{y+r} ) / 2,
//         sum_r A(r) M_{y+r} = (1/N) IDFT( DFT(M) conj(DFT(A_embedded)) )(y).
// Transforms are hand-written: mixed-radix (2, 3, 4, 5) Stockham passes over one axis per
// launch, a block transforming L lines in shared memory, in FP64 complex arithmetic (the
// descriptor needs ~1e-7 relative accuracy; an FP32 transform of 2^20 points is not there).
#include "common.cuh"

namespace dmcr {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// multiply by -i (forward radix-4) or +i (inverse)
__device__ __forceinline__ double2 mul_i(double2 a, int sign) {
    return sign < 0 ? make_double2(a.y, -a.x) : make_double2(-a.y, a.x);
}

// Line geometry of one pass: lines along `axis` of an (n0, n1, n2) grid.
struct LineMap {
    int64_t base;
    int64_t stride;
    bool valid;
};

__device__ __forceinline__ LineMap line_of(const FftPass& p, int l) {
    LineMap m;
    const int64_t n0 = p.n[0], n1 = p.n[1], n2 = p.n[2];
    if (p.axis == 2) {
        const int64_t li = (int64_t)blockIdx.x * p.L + l;
        m.valid = li < n0 * n1;
        m.base = li * n2;
        m.stride = 1;
    } else {
        const int64_t nb2 = (n2 + p.L - 1) / p.L;
        const int64_t pidx = blockIdx.x / nb2;
        const int64_t i2 = (blockIdx.x % nb2) * p.L + l;
        m.valid = i2 < n2;
        if (p.axis == 1) {
            m.base = pidx * n1 * n2 + i2;
            m.stride = n2;
        } else {
            m.base = pidx * n2 + i2;
            m.stride = n1 * n2;
        }
    }
    return m;
}

// One Stockham stage of radix R over the L lines in shared memory (src -> dst): every
// butterfly reads R values n/R apart, multiplies by the twiddles of its offset k within the
// current sub-transform length Ns, and writes R values Ns apart.  R is a template parameter so
// that the butterfly's values stay in registers.
template <int R>
__device__ __forceinline__ void fft_stage(const FftPass& p, const double2* __restrict__ src, double2* __restrict__ dst,
                                          int Ns) {
    const int n = p.len, L = p.L;
    const int nR = n / R;
    const int tstep = n / (Ns * R);
    for (int t = threadIdx.x; t < L * nR; t += blockDim.x) {
        const int l = t / nR, j = t - l * nR;
        const int k = j % Ns;
        const double2* in = src + l * n;
        double2 v[R];
        v[0] = in[j];
#pragma unroll
        for (int r = 1; r < R; ++r) {
            double2 w = p.tw[(k * r) * tstep];
            if (p.sign > 0) w.y = -w.y;
            v[r] = cmul(in[j + r * nR], w);
        }
        double2 V[R];
        if (R == 2) {
            V[0] = cadd(v[0], v[1]);
            V[1] = csub(v[0], v[1]);
        } else if (R == 4) {
            const double2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
            const double2 c = cadd(v[1], v[3]), d = mul_i(csub(v[1], v[3]), p.sign);
            V[0] = cadd(a, c);
            V[1] = cadd(b, d);
            V[2] = csub(a, c);
            V[3] = csub(b, d);
        } else {
            // radix 3 and 5: V[q] = sum_r v[r] omega^(r q),  omega = exp(sign 2 pi i / R)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                double2 acc = v[0];
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    double2 w = R == 3 ? p.om3[(r * q) % 3] : p.om5[(r * q) % 5];
                    if (p.sign > 0) w.y = -w.y;
                    acc = cadd(acc, cmul(v[r], w));
                }
                V[q] = acc;
            }
        }
        double2* out = dst + l * n + (j / Ns) * Ns * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) out[q * Ns] = V[q];
    }
}

__global__ void __launch_bounds__(256) fft_pass_kernel(FftPass p) {
    extern __shared__ __align__(16) double2 sbuf[];
    const int n = p.len, L = p.L;
    double2* src = sbuf;
    double2* dst = sbuf + (size_t)L * n;
    const int total = L * n;
    // load L lines (lanes along the contiguous axis when the lines are strided)
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int l, i;
        if (p.axis == 2) { l = e / n; i = e - l * n; }
        else { i = e / L; l = e - i * L; }
        const LineMap m = line_of(p, l);
        double2 v = make_double2(0.0, 0.0);
        if (m.valid) {
            const int64_t g = m.base + (int64_t)i * m.stride;
            v = p.real_in != nullptr ? make_double2((double)p.real_in[g], 0.0) : p.data[g];
        }
        src[l * n + i] = v;
    }
    int Ns = 1;
    for (int s = 0; s < p.nrad; ++s) {
        const int R = p.rad[s];
        __syncthreads();
        switch (R) {
            case 2: fft_stage<2>(p, src, dst, Ns); break;
            case 3: fft_stage<3>(p, src, dst, Ns); break;
            case 4: fft_stage<4>(p, src, dst, Ns); break;
            default: fft_stage<5>(p, src, dst, Ns); break;
        }
        double2* tmp = src;
        src = dst;
        dst = tmp;
        Ns *= R;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int l, i;
        if (p.axis == 2) { l = e / n; i = e - l * n; }
        else { i = e / L; l = e - i * L; }
        const LineMap m = line_of(p, l);
        if (m.valid) p.data[m.base + (int64_t)i * m.stride] = src[l * n + i];
    }
}

size_t fft_smem_bytes(int len, int L) { return (size_t)2 * L * len * sizeof(double2); }

int fft_lines_per_block(int len) {
    int L = 4096 / len;
    if (L > 16) L = 16;
    return L < 1 ? 1 : L;
}

void launch_fft_pass(const FftPass& p, cudaStream_t s) {
    int64_t blocks;
    if (p.axis == 2) blocks = (p.n[0] * p.n[1] + p.L - 1) / p.L;
    else blocks = (p.axis == 1 ? p.n[0] : p.n[1]) * ((p.n[2] + p.L - 1) / p.L);
    fft_pass_kernel<<<(unsigned)blocks, 256, fft_smem_bytes(p.len, p.L), s>>>(p);
}

// P <- |X|^2 (X is kept: the adjoint of the same call reuses the transform of the field)
__global__ void fft_power_kernel(const double2* __restrict__ X, double2* __restrict__ P, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double2 v = X[i];
    P[i] = make_double2(v.x * v.x + v.y * v.y, 0.0);
}

// H <- X conj(H)
__global__ void fft_xcorr_kernel(const double2* __restrict__ X, double2* __restrict__ H, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double2 a = X[i], b = H[i];
    H[i] = make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

__device__ __forceinline__ int64_t wrapn(int64_t v, int64_t n) {
    const int64_t m = v % n;
    return m < 0 ? m + n : m;
}

// Canonical half-window index k -> (rz, ry, rx).
__device__ __forceinline__ void canon_decode(const LevelGeom& g, int64_t k, int& rz, int& ry, int& rx) {
    const int Px = g.P[2], Py = g.P[1];
    const int64_t wx = 2 * Px + 1, wy = 2 * Py + 1;
    if (k <= Px) { rz = 0; ry = 0; rx = (int)k; return; }
    k -= Px + 1;
    if (k < (int64_t)Py * wx) { rz = 0; ry = 1 + (int)(k / wx); rx = (int)(k % wx) - Px; return; }
    k -= (int64_t)Py * wx;
    rz = 1 + (int)(k / (wy * wx));
    const int64_t rem = k % (wy * wx);
    ry = (int)(rem / wx) - Py;
    rx = (int)(rem % wx) - Px;
}

// desc[k] = w * S_bar(r_k) from the unnormalised inverse transform X = N^2 C (mode 0:
// identity threshold; mode 1: soft threshold of a binary field, App. A with fh2 = f(1/2)^2).
__global__ void fft_sample_kernel(LevelGeom g, const double2* __restrict__ X, float weight, int mode, double fh2,
                                  float* __restrict__ desc) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.Khalf) return;
    int rz, ry, rx;
    canon_decode(g, k, rz, ry, rx);
    const double invN2 = 1.0 / ((double)g.N * (double)g.N);
    const double C0 = X[0].x * invN2;
    const double Cr = X[(wrapn(rz, g.n[0]) * g.n[1] + wrapn(ry, g.n[1])) * g.n[2] + wrapn(rx, g.n[2])].x * invN2;
    double s;
    if (mode == 0) s = 0.5 * (C0 + Cr);
    else s = (k == 0) ? C0 : (1.0 - 2.0 * fh2) * Cr + 2.0 * fh2 * C0;
    desc[k] = (float)((double)weight * s);
}

// H[u] = sum of the window coefficients A(r) with r = u (mod n), gathered over the at most
// two preimages per axis (windows are at most half a period); A is plane 0 of the dense
// coefficient grid (quad layout of gcoef_kernel).
__global__ void fft_embed_kernel(LevelGeom g, const float* __restrict__ Gd, double2* __restrict__ H) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= g.N) return;
    const int64_t ux = u % g.n[2], uy = (u / g.n[2]) % g.n[1], uz = u / (g.n[1] * g.n[2]);
    const int64_t cz[2] = {uz, uz - g.n[0]}, cy[2] = {uy, uy - g.n[1]}, cx[2] = {ux, ux - g.n[2]};
    double acc = 0.0;
    const int wy = 2 * g.P[1] + 1;
    for (int a = 0; a < 2; ++a) {
        const int64_t rz = cz[a];
        if (rz < -g.P[0] || rz > g.P[0] || (a == 1 && cz[1] == cz[0])) continue;
        for (int b = 0; b < 2; ++b) {
            const int64_t ry = cy[b];
            if (ry < -g.P[1] || ry > g.P[1]) continue;
            for (int c = 0; c < 2; ++c) {
                const int64_t rx = cx[c];
                if (rx < -g.P[2] || rx > g.P[2]) continue;
                const int64_t row = (rz + g.P[0]) * wy + (ry + g.P[1]);
                const int col = (int)(rx + g.P[2]);
                const int blk = col / T, m = col % T;
                acc += (double)Gd[(row * g.NB + blk) * GBLOCK + 4 * m];
            }
        }
    }
    H[u] = make_double2(acc, 0.0);
}

// part[y] = ( M_y sum_r A(r) + Re(Z[y]) / N ) / 2,  sum_r A(r) = Re(DFT(H)[0]) read before the product.
__global__ void fft_vjp_combine_kernel(int64_t N, const float* __restrict__ M, const double2* __restrict__ Z,
                                       const double* __restrict__ sumA, float* __restrict__ part) {
    const int64_t y = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= N) return;
    part[y] = (float)(0.5 * ((double)M[y] * (*sumA) + Z[y].x / (double)N));
}

__global__ void fft_dc_kernel(const double2* __restrict__ H, double* __restrict__ out) { *out = H[0].x; }

// tw[t] = exp(-2 pi i t / len), from the library's sincospi (double)
__global__ void fft_twiddle_kernel(double2* __restrict__ tw, int len) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= len) return;
    double sv, cv;
    sincospi(2.0 * (double)t / (double)len, &sv, &cv);
    tw[t] = make_double2(cv, -sv);
}

void launch_fft_twiddles(double2* tw, int len, cudaStream_t s) {
    fft_twiddle_kernel<<<(len + 255) / 256, 256, 0, s>>>(tw, len);
}

void launch_fft_power(const double2* X, double2* P, int64_t N, cudaStream_t s) {
    fft_power_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(X, P, N);
}
void launch_fft_xcorr(const double2* X, double2* H, int64_t N, cudaStream_t s) {
    fft_xcorr_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(X, H, N);
}
void launch_fft_sample(const LevelGeom& g, const double2* X, float weight, int mode, double fh2, float* desc,
                       cudaStream_t s) {
    fft_sample_kernel<<<(unsigned)((g.Khalf + 255) / 256), 256, 0, s>>>(g, X, weight, mode, fh2, desc);
}
void launch_fft_embed(const LevelGeom& g, const float* Gd, double2* H, cudaStream_t s) {
    fft_embed_kernel<<<(unsigned)((g.N + 255) / 256), 256, 0, s>>>(g, Gd, H);
}
void launch_fft_dc(const double2* H, double* out, cudaStream_t s) { fft_dc_kernel<<<1, 1, 0, s>>>(H, out); }
void launch_fft_vjp_combine(int64_t N, const float* M, const double2* Z, const double* sumA, float* part,
                            cudaStream_t s) {
    fft_vjp_combine_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, M, Z, sumA, part);
}

void set_fft_attributes() {
    cudaFuncSetAttribute(fft_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
}

}  // namespace dmcr
