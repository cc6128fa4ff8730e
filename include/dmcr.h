/*
 * dmcr.h -- C ABI of the GB300 (sm_103a) library for differentiable microstructure
 * characterization and reconstruction (Seibert, Ambati, Rassloff, Kaestner,
 * "Reconstructing random heterogeneous media through differentiable optimization",
 * arXiv 2103.09686).
 *
 * The library evaluates, for a relaxed (real-valued) periodic 2-D or 3-D phase field M:
 *   - the soft-thresholded two-point correlation descriptor
 *       S_bar_l(r) = (1/N_l) sum_x f( a_x(r) )^2,
 *       a_x(r) = (M_x + M_{x+r mod n}) / 2  (r != 0),  a_x(0) = M_x
 *     (Sec. 3.2.2 Eq. s3 with p=r, q=s; Sec. 3.2.3 Eq. convdef; Sec. 3.2.4
 *     Eq. softthreshold with f(0)=0, f(1)=1, f''(0.75)=0, alpha=10),
 *     on every level l of the simultaneous multigrid pyramid and concatenated as
 *     D = [w_1 S_bar_1, w_2 S_bar_2, ...] (Sec. 3.3 Eq. mg);
 *   - the loss L = E + lambda E_bc, E = ||D - D_des||_2, lambda = lambda0 E
 *     (Sec. 3.1 Eq. L_func_dMCR) and its exact gradient with respect to every pixel
 *     or voxel, back-propagated through all levels at once (Sec. 3.3);
 *   - Adam reconstructions driven by that gradient (Sec. 3, Eq. M-update; App. B).
 *
 * Conventions common to every call
 *   - Every call returns a dmcr_status.  On failure dmcr_last_error() (thread local)
 *     returns a one-line reason; nothing has been enqueued when argument validation
 *     fails (DMCR_EINVAL).
 *   - Fields are FP32, C order (n[0] slowest).  2-D fields use n[0], n[1]; 3-D fields
 *     n[0], n[1], n[2].  Shift component r_a runs along array axis a.
 *   - Every float pointer is CALLER-OWNED DEVICE memory unless stated otherwise; the
 *     library never frees caller memory and never keeps a pointer after a call returns.
 *   - Scratch memory: calls that need it take `ws`, a caller-owned device buffer of at
 *     least dmcr_workspace_size() bytes, 256-byte aligned.  The library allocates no
 *     device memory in those calls.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Work is enqueued asynchronously on it unless the call says otherwise.
 *   - Half-window layout of one level (HALF, the canonical order), with P the window:
 *       2-D: (0, 0..P1), then (1..P0, -P1..P1) row-major;
 *       3-D: (0, 0, 0..P2), (0, 1..P1, -P2..P2), (1..P0, -P1..P1, -P2..P2).
 *     K_half = (prod_a (2 P_a + 1) + 1) / 2 entries; the descriptor holds `levels`
 *     such blocks, finest level first.
 */
#ifndef DMCR_H
#define DMCR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DMCR_OK = 0,
    DMCR_EINVAL = 1,      /* invalid argument (sizes, window, levels, null pointer) */
    DMCR_ENOMEM = 2,      /* workspace too small */
    DMCR_ECUDA = 3,       /* a CUDA runtime call failed */
    DMCR_ENONFINITE = 4,  /* the loss became NaN or Inf */
    DMCR_ETIMEOUT = 5,    /* a bounded device wait ran out */
    DMCR_ENOTSUP = 6      /* combination not supported by this build */
} dmcr_status;

enum { DMCR_SOFT = 0, DMCR_IDENTITY = 1 };           /* threshold (Sec. 3.2.4; f(x)=x ablation of Sec. 4.1) */
/* Evaluation path.  DIRECT: the shift-by-shift kernels (any threshold).  FFT: the
 * autocorrelation by hand-written FP64 FFTs -- exact (up to rounding) for the identity
 * threshold, and for the soft threshold of BINARY fields through the App. A mapping
 * (descriptor only; use it to characterise binary targets).  Every level size must factor
 * into 2, 3 and 5 and be <= 4096 per axis.  AUTO: DIRECT for the soft threshold; for the
 * identity threshold the cheaper of the two per level (measured crossover). */
enum { DMCR_PATH_AUTO = 0, DMCR_PATH_DIRECT = 1, DMCR_PATH_FFT = 2 };
enum { DMCR_LOSS_NORM = 0, DMCR_LOSS_SQUARED = 1 };  /* L = E(1 + lambda0 E_bc)  |  E^2 (1 + lambda0 E_bc) */
enum { DMCR_PROLONG_ADJOINT_ACCUMULATE = 0, DMCR_PROLONG_INJECT = 1 };
/* Descriptor.  S2: the two-point S_bar2(r) on the half window, K_half floats per level
 * (Sec. 3.2.4).  S3: the full quadratic reduction of the ensemble, Eq. s3,
 * S_bar3(r_a, r_b) = (1/N) sum_x e_x(r_a) e_x(r_b) for every pair of half-window shifts: a
 * K_half x K_half matrix per level, row-major, whose diagonal is S_bar2 (the Gram matrix of
 * the ensemble, Sec. 3.4 footnote).  S3 is computed on the tensor cores (operands split
 * into two FP16 parts after a power-of-two scaling, three products, FP32 accumulation;
 * FP32-level accuracy) and needs the DIRECT or AUTO path. */
/* S2_TILDE: the corrected two-point descriptor of App. A (Eq. s2rfroms2rbar), per level
 * S_tilde(0) = S_bar(0) and S_tilde(r) = (S_bar(r) - 2 f(1/2)^2 S_bar(0)) / (1 - 2 f(1/2)^2),
 * K_half floats per level (equal to the exact S2 of binary fields); any path. */
enum { DMCR_DESC_S2 = 0, DMCR_DESC_S3 = 1, DMCR_DESC_S2_TILDE = 2 };
enum { DMCR_INIT_CALLER = 0, DMCR_INIT_UNIFORM_SEEDED = 1 };

/* Problem statement (Sec. 3.3): field size, window P_a per axis, multigrid levels. */
typedef struct {
    int ndim;                /* 2 or 3 */
    int64_t n[3];            /* finest field sizes, C order; n[a] divisible by 2^(levels-1) */
    int window[3];           /* P_a >= 0 per axis; at every level P_a <= n_a(level) / 2 */
    int levels;              /* >= 1; level l has size n / 2^(l-1), mean of 2^d children */
    int threshold;           /* DMCR_SOFT (default) or DMCR_IDENTITY */
    float alpha;             /* soft-threshold slope; the paper uses 10 */
    float level_weight_exp;  /* w_l = 2^(level_weight_exp (l-1)); <0 selects ndim/2 (2^(l-1) in 2-D); must be finite */
    int path;                /* DMCR_PATH_AUTO, DMCR_PATH_DIRECT or DMCR_PATH_FFT */
    int tune[4];             /* launch shape (0 = built-in choice): forward tile rows {2,4,8,16,32},
                                adjoint ry rows per shift chunk (1..16), adjoint chunk target
                                limit (1..64), adjoint rx blocks of 8 shifts per chunk at most
                                (1..32).  Results agree to rounding across shapes. */
    int descriptor;          /* DMCR_DESC_S2 (default), DMCR_DESC_S3 or DMCR_DESC_S2_TILDE */
    int phases;              /* phase fields (1..8; 0 means 1).  See "Several phases" below. */
} dmcr_params;

/* Several phases (the multi-phase outlook of Sec. 5; the paper defines the descriptor for
 * one field).  With phases = P > 1 every field argument is a stack of P phase fields, each
 * of the size n above, phase-major and contiguous (P x N floats; gradients, Adam moments
 * and the uniform start field likewise), and the descriptor holds, per level and per
 * ordered phase pair (a, b) in row-major order, the cross-correlation
 *     S_bar^{a->b}(r) = (1/N) sum_x f((M^a_x + M^b_{x+r}) / 2)^2
 * on the half window (K_half floats): P^2 K_half floats per level.  The block (b, a) holds
 * S_bar^{a->b}(-r), so both blocks together give the full window; (a, a) is S_bar2 of
 * phase a.  The box penalty E_bc sums the excess of every phase field, each divided by
 * the finest position count N of one field, and lambda0 < 0 selects that N.  Requires
 * descriptor = DMCR_DESC_S2 and the direct path (AUTO never picks the FFT; FFT gives
 * DMCR_ENOTSUP).  Cost: P^2 times one field's. */

/* Loss options (Sec. 3.1).  lambda = lambda0 * E (NORM) or lambda0 * E^2 (SQUARED). */
typedef struct {
    int mode;                /* DMCR_LOSS_NORM (the paper) or DMCR_LOSS_SQUARED */
    float lambda0;           /* <0 selects the finest pixel count N */
    int bc_on;               /* 0 disables the box penalty E_bc */
} dmcr_loss_opts;

/* loss_out layout written by dmcr_loss_grad / dmcr_reconstruct (6 floats) */
enum { DMCR_OUT_E = 0, DMCR_OUT_E2 = 1, DMCR_OUT_EBC = 2, DMCR_OUT_LAMBDA = 3, DMCR_OUT_L = 4,
       DMCR_OUT_REL_ERR = 5, DMCR_OUT_COUNT = 6 };

/* Reconstruction options (flow chart of Sec. 3; Adam at the TensorFlow defaults, App. B). */
typedef struct {
    int max_iters;           /* iterations (loss + gradient + Adam step) at most */
    float tol_rel;           /* stop when ||D - D_des|| / ||D_des|| < tol_rel (0: never) */
    float lr, beta1, beta2, eps;   /* 1e-3, 0.9, 0.999, 1e-7 */
    dmcr_loss_opts loss;
    int init;                /* DMCR_INIT_CALLER or DMCR_INIT_UNIFORM_SEEDED */
    uint64_t seed;           /* SplitMix64 seed for DMCR_INIT_UNIFORM_SEEDED */
    int check_every;         /* stopping test every k iterations (>= 1) */
    int report_rounded;      /* nonzero: dmcr_reconstruct(_batched) evaluates the returned field
                                rounded to 0/1 once more for report.rounded_rel_err (NaN when 0) */
} dmcr_recon_opts;

/* Adam state of one job: caller-owned device buffers, kept between calls (resume). */
typedef struct {
    float* m;                /* N floats, zero for a fresh start */
    float* v;                /* N floats, zero for a fresh start */
    int64_t step;            /* Adam steps taken so far (host value, updated on return) */
} dmcr_adam_state;

typedef struct {
    int iterations;          /* Adam steps taken in this call */
    int converged;           /* 1 if tol_rel was reached */
    float loss[DMCR_OUT_COUNT];   /* loss_out of the last evaluated iterate */
    int status;              /* dmcr_status of the run */
    float rounded_rel_err;   /* rel_err of the returned field rounded to 0/1 (M >= 1/2 -> 1; Sec. 4.1);
                                NaN unless opts.report_rounded */
} dmcr_recon_report;

/* Library version as 10000*major + 100*minor + patch. */
int dmcr_version(void);

/* Reason for the last failing call on this host thread ("" if none). */
const char* dmcr_last_error(void);

/* Descriptor length: sum_l K_half (S2, S2_TILDE), sum_l K_half^2 (S3), times phases^2.
 * Returns DMCR_EINVAL on bad params. */
dmcr_status dmcr_descriptor_length(const dmcr_params* p, int64_t* length);

/* Bytes of scratch memory (`ws`) the calls below need for these params. */
dmcr_status dmcr_workspace_size(const dmcr_params* p, size_t* bytes);

/*
 * dmcr_descriptor -- the multigrid descriptor D of `field` (Sec. 3.2, Sec. 3.3 Eq. mg).
 *   field: N floats (device, read only).  desc: dmcr_descriptor_length floats (device,
 *   written).  Also used to characterise a target: D_des = dmcr_descriptor(target).
 *   Errors: DMCR_EINVAL (params), DMCR_ENOMEM (ws_bytes too small), DMCR_ENOTSUP (a
 *   combination of descriptor, path and phases that is not provided, see above),
 *   DMCR_ECUDA.  The call is asynchronous: a bounded tensor-core wait of the three-point
 *   descriptor that gives up only marks the workspace, and the synchronous
 *   dmcr_reconstruct reports it as DMCR_ETIMEOUT.
 */
dmcr_status dmcr_descriptor(const dmcr_params* p, const float* field, float* desc,
                            void* ws, size_t ws_bytes, void* stream);

/*
 * dmcr_loss_grad -- loss and exact gradient (Sec. 3.1 Eq. L_func_dMCR; Sec. 3.3).
 *   field: N floats; target_desc: descriptor_length floats (device, read only).
 *   loss_out: DMCR_OUT_COUNT floats (device, written: E, E^2, E_bc, lambda, L, rel_err).
 *   grad: N floats (device, written) or NULL for the loss alone.
 *   desc_out: descriptor_length floats (device, written) or NULL.
 *   At E = 0 the NORM-mode gradient of E is defined as 0.
 */
dmcr_status dmcr_loss_grad(const dmcr_params* p, const dmcr_loss_opts* opts, const float* field,
                           const float* target_desc, float* loss_out, float* grad, float* desc_out,
                           void* ws, size_t ws_bytes, void* stream);

/*
 * dmcr_descriptor_vjp -- grad_field = (dD/dM)^T grad_desc for an arbitrary upstream
 *   gradient (the backward of a differentiable descriptor; Sec. 3.3: through every level).
 *   grad_desc: descriptor_length floats; grad_field: N floats (device, written).
 */
dmcr_status dmcr_descriptor_vjp(const dmcr_params* p, const float* field, const float* grad_desc,
                                float* grad_field, void* ws, size_t ws_bytes, void* stream);

/*
 * dmcr_restrict -- one multigrid coarsening (Sec. 3.3; read: each coarse cell is the mean
 *   of its 2^d children).  n_fine: sizes of `fine` (each even).  coarse: N/2^d floats.
 */
dmcr_status dmcr_restrict(int ndim, const int64_t n_fine[3], const float* fine, float* coarse,
                          void* stream);

/*
 * dmcr_prolongate -- coarse to fine (Sec. 3.3).  mode DMCR_PROLONG_ADJOINT_ACCUMULATE:
 *   fine += R^T coarse, i.e. every child gains parent / 2^d (the transpose of
 *   dmcr_restrict, used to back-propagate through the levels); DMCR_PROLONG_INJECT:
 *   fine = parent value copied to every child (coarse-to-fine warm start).
 *   n_coarse: sizes of `coarse`; fine has 2^d times as many cells.
 */
dmcr_status dmcr_prolongate(int ndim, const int64_t n_coarse[3], const float* coarse, float* fine,
                            int mode, void* stream);

/*
 * dmcr_init_uniform -- field[i] = top 24 bits of SplitMix64(seed, i) * 2^-24, the
 *   counter-based uniform[0,1) start of a reconstruction ("randomly initialized", Sec. 3).
 */
dmcr_status dmcr_init_uniform(float* field, int64_t count, uint64_t seed, void* stream);

/*
 * dmcr_reconstruct -- Adam reconstruction (flow chart of Sec. 3; Eq. M-update; App. B).
 *   Iteration t: evaluate L and dL/dM at the current field; if (t-1) % check_every == 0
 *   and rel_err < tol_rel, stop; otherwise take one Adam step.  The iteration runs as a
 *   captured CUDA graph; the stopping test is taken on the device.
 *   field_inout: N floats, the start (DMCR_INIT_CALLER) and the result.
 *   state: Adam moments (device) and step count (host), updated for resume.
 *   history: max_iters * 3 floats (device: E, L, rel_err per iteration) or NULL.
 *   SYNCHRONOUS: returns after the run, with `report` (host) filled in; report.loss is the
 *   loss of the returned field.  The graph runs on a private stream created with the
 *   priority of `stream` (so a high-priority caller stream keeps its priority).  The
 *   library keeps the 32 most recently captured iteration graphs (of this call and the
 *   batched one), keyed by their whole launch sequence, so a later call with the same
 *   arguments and options captures nothing.
 */
dmcr_status dmcr_reconstruct(const dmcr_params* p, const dmcr_recon_opts* opts,
                             const float* target_desc, float* field_inout, dmcr_adam_state* state,
                             float* history, dmcr_recon_report* report, void* ws, size_t ws_bytes,
                             void* stream);

/*
 * dmcr_adam_step -- ONE iteration of the reconstruction loop (flow chart of Sec. 3):
 *   the loss at the current field (written to loss_out, DMCR_OUT_COUNT floats, device, or
 *   NULL), its exact gradient and one Adam step (Keras form, bias correction with step
 *   state->step + 1).  Uses opts->lr, beta1, beta2, eps and opts->loss; ignores the
 *   stopping fields.  Asynchronous on `stream`; state->step is incremented on return.
 *   A non-finite loss leaves the field unchanged (check loss_out).
 *   The first call with a given set of arguments (params, the options above, every pointer,
 *   ws_bytes, the current device) captures the iteration into a CUDA graph that the library
 *   keeps (the 16 most recently used sets); a later call with the same arguments launches
 *   one small kernel with this call's step count and replays the graph, with the same
 *   results bit for bit.  While `stream` is being captured by the caller, or while the
 *   dmcr_profile timers are on, the kernels are launched directly instead.
 */
dmcr_status dmcr_adam_step(const dmcr_params* p, const dmcr_recon_opts* opts, const float* target_desc,
                           float* field, dmcr_adam_state* state, float* loss_out, void* ws, size_t ws_bytes,
                           void* stream);

/*
 * Batched calls: `count` independent instances of any sizes, windows and levels (they must
 * share the threshold and alpha), evaluated by ONE fused launch per phase -- every
 * (instance, level) is a segment of the same grid, heaviest blocks first.  Pointer
 * arguments are HOST arrays of `count` device pointers; loss_out holds count x
 * DMCR_OUT_COUNT floats (device).  Each instance gives exactly the result of the
 * corresponding single-instance call (same tiles, same summation order).
 * The workspace is dmcr_batch_workspace_size() bytes, 256-byte aligned.
 */
dmcr_status dmcr_batch_workspace_size(int count, const dmcr_params* params, size_t* bytes);
dmcr_status dmcr_descriptor_batched(int count, const dmcr_params* params, const float* const* fields,
                                    float* const* descs, void* ws, size_t ws_bytes, void* stream);
dmcr_status dmcr_loss_grad_batched(int count, const dmcr_params* params, const dmcr_loss_opts* opts,
                                   const float* const* fields, const float* const* targets, float* loss_out,
                                   float* const* grads /* NULL: loss only */, void* ws, size_t ws_bytes,
                                   void* stream);
dmcr_status dmcr_descriptor_vjp_batched(int count, const dmcr_params* params, const float* const* fields,
                                        const float* const* grad_descs, float* const* grad_fields, void* ws,
                                        size_t ws_bytes, void* stream);
/* One Adam iteration of every instance (one opts for all; states: host array of count). */
dmcr_status dmcr_adam_step_batched(int count, const dmcr_params* params, const dmcr_recon_opts* opts,
                                   const float* const* targets, float* const* fields, dmcr_adam_state* states,
                                   float* loss_out, void* ws, size_t ws_bytes, void* stream);
/*
 * Graph-captured reconstruction of every instance (opts, states, reports: host arrays of
 * count).  Instances stop independently on their own device flags (converged instances
 * cost nothing in later launches); the call returns when all have stopped.  SYNCHRONOUS.
 * report.loss is the loss of the returned field of that instance.  An instance whose loss
 * becomes non-finite stops with report.status = DMCR_ENONFINITE (its field is left at the
 * last finite iterate); the other instances are unaffected and the call returns DMCR_OK.
 */
dmcr_status dmcr_reconstruct_batched(int count, const dmcr_params* params, const dmcr_recon_opts* opts,
                                     const float* const* targets, float* const* fields, dmcr_adam_state* states,
                                     dmcr_recon_report* reports, void* ws, size_t ws_bytes, void* stream);

/*
 * Per-kernel timing with CUDA events recorded on the launching stream (host side).
 *   dmcr_profile_enable(1) starts recording every kernel the library launches outside a
 *   graph capture; dmcr_profile_reset() clears the records; dmcr_profile_read(i, ...)
 *   waits for the recorded events and returns the i-th kernel name, its summed duration
 *   in milliseconds and its launch count (DMCR_EINVAL once i is past the last entry).
 */
dmcr_status dmcr_profile_enable(int on);
dmcr_status dmcr_profile_reset(void);
dmcr_status dmcr_profile_read(int index, char* name, int name_len, double* total_ms, int64_t* launches);

/*
 * dmcr_descriptor_noalloc -- the same descriptor as dmcr_descriptor, for callers that
 *   cannot allocate device memory (no cudaMalloc, no caching allocator) at the point of
 *   the call: code running under a runtime that forbids allocation during execution, or
 *   deployments that reserve all device memory up front.  The paper has no counterpart;
 *   this is a deployment convenience of this library.
 *   Scratch comes from one fixed device array of DMCR_NOALLOC_SCRATCH_BYTES (16 MiB) in
 *   the library, held by every GPU that loads it until the process exits.  Problems whose
 *   scratch (pyramid levels plus per-tile partial sums) exceeds it are rejected with
 *   DMCR_ENOMEM and a message; use dmcr_descriptor with a workspace for those.
 *   The call allocates nothing.  Its first call on a device looks up the array's device
 *   address (cudaGetSymbolAddress) with that device current; make that first call before
 *   any stream capture.  All calls share the one array and every call overwrites what the
 *   previous one left there, so calls that can overlap on the GPU (different streams,
 *   threads or graphs without ordering between them) race: serialise them.
 *   field: N floats, desc: dmcr_descriptor_length floats (device).  Asynchronous on `stream`.
 */
#define DMCR_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
dmcr_status dmcr_descriptor_noalloc(const dmcr_params* p, const float* field, float* desc, void* stream);


#ifdef __cplusplus
}
#endif

#endif /* DMCR_H */
