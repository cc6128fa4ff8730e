// Shared declarations of the dmcr CUDA library (kernels + C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dmcr {

constexpr int T = 8;            // shifts per thread (forward) / positions per strip (adjoint)
constexpr int TX = 32;          // tile width in positions (fastest axis)
constexpr int FWD_THREADS = 128;
constexpr int ADJ_THREADS = 128;   // 32 rows x 4 strips of 8 positions
constexpr int NPEN_BLOCKS = 256;   // fixed grid of the penalty reduction (deterministic)
constexpr int MAX_DYN_SMEM = 200 * 1024;   // dynamic shared memory limit of the correlation kernels

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
    int nChunks;
};

// Soft-threshold constants in the product form used on the device:
//   P = E'_x E_y,  E_y = 2^(-kappa M_y),  E'_x = 2^(cexp - kappa M_x)
//   s = 1/(1+P) = sigma(alpha (a - 0.75)),  f = c1 s + c3.
struct ThreshConst {
    float kappa;     // (alpha/2) log2(e)
    float cexp;      // 0.75 alpha log2(e)
    float c1, c3;
    float alpha;
    float lim;       // fast path when |kappa M| <= lim everywhere in a block
    int identity;    // f(x) = x
};

// Device-side scalars of one evaluation / reconstruction.
struct Scalars {
    float loss[6];        // E, E2, Ebc, lambda, L, rel_err
    float gscale;         // dL/dD = gscale * rho
    float pen_coef;       // penalty gradient coefficient: pen_coef * ex * dex
    float lr_t;           // Adam step size of the current iteration
    int done;             // 0 running, 1 converged, 2 non-finite loss
    int iter;             // iterations evaluated in this call
    int64_t adam_step;    // Adam steps taken (global, for bias correction)
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

// ---------------------------------------------------------------- launchers (kernels.cu)
void launch_restrict(int ndim, const int64_t nf[3], const float* fine, float* coarse,
                     const int* done, cudaStream_t s);
void launch_prolongate(int ndim, const int64_t nc[3], const float* coarse, float* fine, int mode,
                       cudaStream_t s);
void launch_corr_fwd(const LevelGeom& g, const ThreshConst& tc, const float* field, float* partial,
                     const int* done, cudaStream_t s);
void launch_fwd_reduce(const LevelGeom& g, const ThreshConst& tc, const float* partial, float weight,
                       float* desc, const int* done, cudaStream_t s);
void launch_penalty(const float* field, int64_t N, double* partials, const int* done, cudaStream_t s);
void launch_loss(const LossParams& lp, const float* desc, const float* target, const double* pen,
                 Scalars* sc, float* loss_out, float* history, cudaStream_t s);
void launch_gcoef(const LevelGeom& g, const ThreshConst& tc, const float* src, const float* sub,
                  const Scalars* sc, float weight, float* Gd, const int* done, cudaStream_t s);
void launch_corr_adj(const LevelGeom& g, const ThreshConst& tc, const float* field, const float* Gd,
                     float* part, const int* done, cudaStream_t s);
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
void launch_final(const FinalArgs& a, const int* done, cudaStream_t s);
void launch_init_uniform(float* field, int64_t count, uint64_t seed, cudaStream_t s);
void launch_scalars_init(Scalars* sc, int64_t adam_step, cudaStream_t s);
void set_kernel_attributes();
size_t fwd_smem_bytes(const LevelGeom& g);
size_t adj_smem_bytes(const LevelGeom& g);

}  // namespace dmcr
