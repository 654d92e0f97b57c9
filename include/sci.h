/*
 * libsci -- GAP-TV / ADMM-TV reconstruction for video snapshot compressive
 * imaging (SCI) on one NVIDIA GB300 (sm_103a).
 *
 * Method: X. Yuan, "Various Total Variation for Snapshot Video Compressive
 * Imaging", arXiv 2005.08028.  Equation numbers count the paper's numbered
 * displays in order (Eq. 3: Y = sum_k X_k . C_k + G; Eqs. 21-22: GAP;
 * Eqs. 24-26: ADMM; Eqs. 29-32: the ITV2D/ITV3D dual projections);
 * "Algorithm 1" is the paper's GAP-ATV-Clip/Cham/FGP listing.
 *
 * Conventions for every call below
 * --------------------------------
 *  - Layout: a video (x, theta, u) is float32 [B][nx][ny], frame-major then
 *    row-major; element (k, i, j) is at k*nx*ny + i*ny + j.  i < nx is the
 *    vertical index (difference operator D_v), j < ny the horizontal one (D_h).
 *    A measurement y is float32 [nx][ny].
 *  - Masks: binary masks C_k in {0,1} (B <= 32) are passed bit-packed as
 *    uint32 [nx][ny]; bit k of word (i, j) is C_k(i, j).  sci_masks_pack
 *    builds this from a dense uint8 [B][nx][ny] array.
 *  - Pointers: all array pointers are DEVICE pointers owned by the caller,
 *    unless a comment says "host".  The library never frees or keeps them
 *    beyond the call (the solver's CUDA-graph cache remembers their values;
 *    see sci_graph_cache_clear).
 *  - Scratch: calls that need scratch take (work, work_bytes), a caller-owned
 *    device buffer of at least the size that the matching *_workspace query
 *    returns, aligned to 256 bytes.  The library allocates no device memory.
 *  - Streams: every call is asynchronous on `stream` (a cudaStream_t; NULL is
 *    the legacy default stream).  Argument errors are detected on the host and
 *    returned before anything is enqueued.  SCI_ERR_CUDA reports a failed
 *    launch (cudaGetLastError after the enqueue); errors raised while the
 *    kernels run surface at the caller's next synchronisation.
 *  - No exceptions cross this interface.
 */
#ifndef SCI_H_
#define SCI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* sci_stream_t; /* identical to cudaStream_t */

typedef enum {
    SCI_OK = 0,
    SCI_ERR_ARG = 1,        /* null pointer, non-positive size, bad enum, lambda <= 0, ... */
    SCI_ERR_SHAPE = 2,      /* B > 32, or sizes whose element count overflows */
    SCI_ERR_CUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    SCI_ERR_NONFINITE = 4,  /* non-finite scalar argument, or non-finite input data when
                               sci_params.check_input = 1 */
    SCI_ERR_TIMEOUT = 5,    /* reserved: a bounded device-side wait gave up */
    SCI_ERR_WORKSPACE = 6   /* work == NULL, misaligned, or work_bytes too small */
} sci_status;

typedef enum { SCI_TV_ATV = 0, SCI_TV_ITV2D = 1, SCI_TV_VTV = 2 } sci_tv_type;
typedef enum { SCI_F32 = 0, SCI_BF16 = 1, SCI_F16 = 2 } sci_dtype;

/* TVdenoise dual solver (Algorithm 1's boxes, Sec. 2.3).  FGP: the ATV-FGP
 * box, accelerated with the nu recursion.  CHAM: the ATV-Cham box with
 * delta t = 1/8 and the max(1, |.|) denominator the paper states it used,
 * reading its D^T as the divergence (minus the adjoint; with the adjoint the
 * printed update ascends).  It is then the same projected dual step as FGP
 * without momentum (nu = 1 throughout), and the ITV2D / VTV forms take the
 * paper's norms for ITV2D-Cham and the ITV3D dual (Eqs. 29-32).  CLIP: the
 * ATV-Clip box (iterative clipping; ATV only): theta_h = x - D_h^T w_h,
 * theta_v = x - D_v^T w_v, w = clip(w + (1/alpha) D theta_dir, T), output
 * x - D_h^T w_h - D_v^T w_v from the final duals, with alpha = 4 (the bound
 * on the 1-D difference operator's largest eigenvalue; the box leaves alpha
 * undefined) and T = lambda (the prox scale of the other boxes; the printed
 * 2 lambda matches a fidelity without the factor 1/2).  The two directions
 * do not interact: on a frame constant along one axis the converged box is
 * that axis's exact 1-D TV prox. */
typedef enum { SCI_DUAL_FGP = 0, SCI_DUAL_CHAM = 1, SCI_DUAL_CLIP = 2 } sci_dual_solver;

/* Solver parameters (Algorithm 1; Sec. 2.2). */
typedef struct {
    int tv;           /* sci_tv_type: ATV (Eq. 8), ITV2D (Eq. 9) or VTV = ITV3D (Eq. 10) */
    float lambda;     /* TV weight lambda > 0 of TVdenoise = prox of lambda*TV */
    float rho;        /* ADMM penalty rho >= 0 (Eq. 24); ignored by sci_gap_tv */
    int outer_iters;  /* T >= 0 outer iterations */
    int inner_iters;  /* S >= 1 FGP dual updates per TVdenoise */
    int storage;      /* sci_dtype of the library's internal fields; math is FP32 */
    int fuse_k;       /* FGP dual updates per temporally blocked launch: 0 = library
                         choice, k >= 1 = at most k (clamped to what the tile's halo
                         allows), -1 = one launch per update (no temporal blocking) */
    int init;         /* 1: start from theta = Phi^T y (and u = 0); 0: resume from theta (and u) */
    int use_graph;    /* 1: run the T iterations as one cached CUDA graph; 0: plain launches */
    int dual;         /* sci_dual_solver of TVdenoise; 0 (FGP) when zero-initialised;
                         SCI_DUAL_CLIP needs tv = SCI_TV_ATV and is not run by the
                         batched driver */
    int warm_start;   /* 1: dual warm start -- each TVdenoise call starts from the dual w
                         the previous call ended with (Algorithm 1 initialises w once,
                         before the outer loop; nu is still reset inside the box); 0 (the
                         default): w = 0 at every call, so TVdenoise is a pure function.
                         sci_gap_tv and sci_admm_tv on the temporally blocked path only
                         (SCI_ERR_ARG with fuse_k = -1, VTV with B > 24, FISTA or TwIST).
                         The carried w lives in the workspace in the storage type: init = 1
                         starts it at 0, init = 0 resumes from what the previous call on
                         the same workspace left there. */
    int check_input;  /* 1: before enqueueing the solve, count the non-finite entries of y
                         (and of theta, u when init = 0) on the device, synchronise
                         `stream`, and return SCI_ERR_NONFINITE if there are any (so the
                         call blocks; SCI_ERR_ARG while `stream` is capturing).  0: no
                         check (NaN or Inf in y then propagates into the outputs and the
                         FP64 residual history). */
    int tile;         /* tile class of the temporally blocked kernel: 0 = library choice;
                         otherwise one that sci_tile_classes lists for the TV form and
                         frame count: 1 = one-frame 64 x 128 pixels (512 threads, each
                         a 4 x 4 pixel block), 2 = one-frame 32 x 64 (256 threads, each
                         8 rows of a column), 3 = one-frame 64 x 128 (512 threads, each
                         16 rows of a column), 4 = one-frame 32 x 64 (256 threads, each a
                         2 x 4 block), 8 / 10 = VTV 32 x 32 for
                         up to 8 / 10 frames, 16 / 24 = VTV 32 x 16 for up to 16 / 24
                         frames (SCI_ERR_ARG otherwise; the batched driver takes 0 only).
                         With FP32 storage every class gives the same bits. */
} sci_params;

/* Human-readable name of a status code (static string). */
const char* sci_status_str(sci_status s);

/* Library version, major*10000 + minor*100 + patch. */
int sci_version(void);

/*
 * Pack dense binary masks into the bit layout above (storage only; Eq. 2's
 * D_k = diag(vec C_k)).  masks: uint8 [B][nx][ny] with values 0 or 1.
 * bits: uint32 [nx][ny] (output).  bad_count: optional device int that the
 * kernel increments once per entry that is neither 0 nor 1 (such entries are
 * packed as 1); pass NULL to skip the check.  1 <= B <= 32.
 */
sci_status sci_masks_pack(const uint8_t* masks, int nx, int ny, int B, uint32_t* bits,
                          int* bad_count, sci_stream_t stream);

/* Forward operator y = Phi x = sum_k C_k . X_k (Eq. 3 without noise). */
sci_status sci_forward(const float* x, const uint32_t* bits, int nx, int ny, int B,
                       float* y, sci_stream_t stream);

/* Adjoint x = Phi^T y: X_k = C_k . Y (Phi = [D_1..D_B], Eq. 2). */
sci_status sci_adjoint(const float* y, const uint32_t* bits, int nx, int ny, int B,
                       float* x, sci_stream_t stream);

/*
 * rho == 0: GAP projection x = theta + Phi^T (Phi Phi^T)^+ (y - Phi theta)
 * (Eq. 21), with Phi Phi^T = diag(R), R = sum_k C_k^2, and R^+ = 0 where R = 0.
 * rho > 0: ADMM x-update (Eq. 24), x = v + Phi^T ((y - Phi v) / (R + rho)),
 * v = theta - u.  u may be NULL (treated as 0).  1/(R + rho) is formed in
 * FP64 and rounded to FP32.  x may alias neither theta nor u.
 */
sci_status sci_project(const float* theta, const float* u, const float* y,
                       const uint32_t* bits, int nx, int ny, int B, float rho, float* x,
                       sci_stream_t stream);

/* Bytes of scratch sci_tv_prox needs. */
size_t sci_tv_prox_workspace(int nx, int ny, int B, int tv);

/*
 * TVdenoise by FGP (Algorithm 1, ATV-FGP box; Eqs. 29-32 for ITV2D / VTV):
 * inner_iters dual updates from w = p = 0, nu = 1, step 1/(8 lambda), then
 * theta = x - lambda (D_h^T p_h + D_v^T p_v).  x, theta: float32 [B][nx][ny]
 * (may not alias).  D_h, D_v are forward differences without wrap-around.
 */
sci_status sci_tv_prox(const float* x, int nx, int ny, int B, int tv, float lambda,
                       int inner_iters, float* theta, void* work, size_t work_bytes,
                       sci_stream_t stream);

/*
 * TVdenoise by Chambolle's dual projection (Algorithm 1, ATV-Cham box, with
 * the reading stated at sci_dual_solver): inner_iters dual updates from
 * w = 0, w <- proj(w + (1/(8 lambda)) D theta) with theta = x - lambda D^T w,
 * then theta = x - lambda D^T w.  Same arguments, layouts, workspace
 * (sci_tv_prox_workspace) and errors as sci_tv_prox.
 */
sci_status sci_tv_prox_cham(const float* x, int nx, int ny, int B, int tv, float lambda,
                            int inner_iters, float* theta, void* work, size_t work_bytes,
                            sci_stream_t stream);

/*
 * TVdenoise by the ATV-Clip box (Algorithm 1, ATV-Clip; see SCI_DUAL_CLIP):
 * inner_iters clipping updates from w = 0, then theta = x - D_h^T w_h -
 * D_v^T w_v.  tv must be SCI_TV_ATV (SCI_ERR_ARG otherwise).  Same arguments,
 * layouts, workspace (sci_tv_prox_workspace) and errors as sci_tv_prox.
 */
sci_status sci_tv_prox_clip(const float* x, int nx, int ny, int B, int tv, float lambda,
                            int inner_iters, float* theta, void* work, size_t work_bytes,
                            sci_stream_t stream);

/* Bytes of scratch sci_gap_tv / sci_admm_tv / sci_fista_tv / sci_twist_tv need for these sizes and params. */
size_t sci_solver_workspace(int nx, int ny, int B, const sci_params* params);

/*
 * GAP-TV (Eqs. 21-22, Algorithm 1): T outer iterations of
 *   x = projection of theta onto {Phi x = y};  theta = TVdenoise(x).
 * theta: in/out float32 [B][nx][ny] (input ignored when params->init = 1).
 * x_out: float32 [B][nx][ny], receives x^(T) (theta^(0) when T = 0); may be NULL.
 * resid: optional device double array; when resid_every > 0 it receives
 *   ||y - Phi theta^(t)||_2^2 (FP64 accumulation) for t = resid_every,
 *   2*resid_every, ... <= T, at index t/resid_every - 1.
 */
sci_status sci_gap_tv(const float* y, const uint32_t* bits, int nx, int ny, int B,
                      const sci_params* params, float* theta, float* x_out,
                      double* resid, int resid_every, void* work, size_t work_bytes,
                      sci_stream_t stream);

/*
 * FISTA-TV (Sec. 2.2, FISTA steps), with L = ||Phi||^2 = max_ij R_ij and
 * tau_1 = 1: T iterations of
 *   z = theta + (1/L) Phi^T (y - Phi theta);  x = TVdenoise(z);
 *   theta = x + ((tau_t - 1)/tau_{t+1}) (x - x_prev).
 * TVdenoise takes params->lambda (the same plug-in strength as GAP), so a
 * fixed point minimises 1/2||y - Phi x||^2 + lambda L TV(x).  The printed
 * momentum indices are garbled; this is standard FISTA.  Same arguments,
 * workspace (sci_solver_workspace) and errors as sci_gap_tv.  params->init = 1
 * starts from theta = Phi^T y; 0 starts from the given theta with the momentum
 * restarted.  On return theta and x_out (if not NULL) hold the estimate x^(T).
 * resid (if resid_every > 0) records ||y - Phi x^(t)||^2.
 */
sci_status sci_fista_tv(const float* y, const uint32_t* bits, int nx, int ny, int B,
                        const sci_params* params, float* theta, float* x_out,
                        double* resid, int resid_every, void* work, size_t work_bytes,
                        sci_stream_t stream);

/*
 * TwIST-TV (Sec. 2.2, TwIST steps).  The printed unit gradient step needs
 * ||Phi|| <= 1, so the steps run on Phi / sqrt(L), y / sqrt(L) with L = max_ij
 * R_ij (as for FISTA): T iterations of
 *   z = x + (1/L) Phi^T (y - Phi x);  theta = TVdenoise(z);
 *   x_next = theta (first iteration: one plain step)
 *   x_next = (1 - alpha) x_prev + (alpha - beta) x + beta theta (later ones).
 * alpha, beta follow TwIST's rule for the eigenvalue bounds of the normalised
 * A^T A: xi_m = 1, xi_1 = min_{R > 0} R / max R (the nullspace's zero
 * eigenvalues are left to the TV term): rho = (1 - sqrt(xi_1)) / (1 +
 * sqrt(xi_1)), alpha = 1 + rho^2, beta = 2 alpha / (1 + xi_1); they are
 * formed in FP64 on the device from the mask counts.  TVdenoise takes
 * params->lambda (as FISTA).  params->init = 1 starts from x = Phi^T y, 0
 * from the given theta (the two-step recursion restarts).  On return theta
 * and x_out (if not NULL) hold x^(T); resid (if resid_every > 0) records
 * ||y - Phi x^(t)||^2 for t = resid_every, 2 resid_every, ...  Same
 * arguments, workspace (sci_solver_workspace) and errors as sci_gap_tv.
 */
sci_status sci_twist_tv(const float* y, const uint32_t* bits, int nx, int ny, int B,
                        const sci_params* params, float* theta, float* x_out,
                        double* resid, int resid_every, void* work, size_t work_bytes,
                        sci_stream_t stream);

/*
 * ADMM-TV (Eqs. 24-26): T iterations of
 *   x = ADMM x-update (rho = params->rho);  theta = TVdenoise(u + x);  u = u + x - theta.
 * TVdenoise uses params->lambda (Eq. 25 carries no rho).  theta, u: in/out
 * float32 [B][nx][ny] (inputs ignored when params->init = 1: theta = Phi^T y, u = 0).
 * Other arguments as sci_gap_tv.
 */
sci_status sci_admm_tv(const float* y, const uint32_t* bits, int nx, int ny, int B,
                       const sci_params* params, float* theta, float* u, float* x_out,
                       double* resid, int resid_every, void* work, size_t work_bytes,
                       sci_stream_t stream);

/* One measurement of a batched reconstruction. */
typedef struct {
    int nx, ny, B;          /* frame size and frame count (B <= 32; VTV: B <= 24) */
    const float* y;         /* measurement, float32 [nx][ny] */
    const uint32_t* bits;   /* packed masks, uint32 [nx][ny] */
    float* theta;           /* in/out float32 [B][nx][ny] (input used when params->init = 0) */
    float* x_out;           /* optional float32 [B][nx][ny]: x^(T) */
} sci_problem;

/* Bytes of scratch sci_gap_tv_batched needs for these problems (0: invalid). */
size_t sci_gap_tv_batched_workspace(const sci_problem* problems, int count, const sci_params* params);

/*
 * GAP-TV (Algorithm 1) on `count` independent measurements of any mix of
 * sizes, all with the same params.  problems: HOST array of descriptors
 * (device pointers inside).  Each launch covers every measurement: the pixel
 * kernels walk a table of 256-pixel blocks and the temporally blocked FGP
 * kernel a table of tiles (largest measurements first), so the T iterations
 * are about 2 + ceil(S/K) launches each, captured once as a CUDA graph and
 * replayed on later identical calls.  The tables are copied from host memory
 * at every call, so this call must not be made while `stream` is capturing
 * (SCI_ERR_ARG).  VTV problems need B <= 24 (SCI_ERR_SHAPE otherwise).
 * Results equal those of sci_gap_tv on each measurement.
 */
sci_status sci_gap_tv_batched(const sci_problem* problems, int count, const sci_params* params,
                              void* work, size_t work_bytes, sci_stream_t stream);

/* Kernels enqueued by this thread's most recent sci_gap_tv_batched call. */
long long sci_last_batch_launches(void);

/* Release every CUDA graph cached by sci_gap_tv_batched. */
void sci_batch_graph_cache_clear(void);

/* ---------------------------------------------------------------------------
 * Learned TV prox (no counterpart in the paper, whose Sec. 4 points at
 * plug-and-play reconstruction as future work): theta = x + f(x), f a
 * 4-layer 3x3x3 convolutional network 1 -> 32 -> 32 -> 32 -> 1 with ReLU
 * between layers and zero padding over (frame, row, column).  BF16 weights
 * and activations, FP32 accumulation; the 32 -> 32 layers run on the tensor
 * cores (tcgen05).  It stands in for S FGP dual updates inside GAP-TV.
 *
 * params: FP32 [sci_lprox_param_count()] = w1 [27][32][1], b1 [32],
 *   w2 [27][32][32], b2 [32], w3 [27][32][32], b3 [32], w4 [27][1][32], b4 [1];
 *   tap = (dz+1)*9 + (dy+1)*3 + (dx+1);
 *   out[v][o] = b[o] + sum_tap sum_i w[tap][o][i] in[v + (dz,dy,dx)][i].
 * x, theta, target: float32 [count][B][nx][ny] (count volumes).
 * ------------------------------------------------------------------------- */
size_t sci_lprox_param_count(void);

/* Scratch bytes for sci_lprox_apply (training = 0) or the training calls (1). */
size_t sci_lprox_workspace(int nx, int ny, int B, int count, int training);

/* theta = x + f(x) for `count` volumes. */
sci_status sci_lprox_apply(const float* params, const float* x, int nx, int ny, int B, int count,
                           float* theta, void* work, size_t work_bytes, sci_stream_t stream);

/*
 * One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; `step`
 * counts from 1) on the mean squared error between x + f(x) and target.
 * params, adam_m, adam_v: FP32 [param_count], updated in place.  loss:
 * optional device double receiving the sum of squared errors (before the step).
 */
sci_status sci_lprox_train_step(float* params, float* adam_m, float* adam_v, int step, float lr,
                                const float* x, const float* target, int nx, int ny, int B, int count,
                                double* loss, void* work, size_t work_bytes, sci_stream_t stream);

/* Gradient of that loss with respect to params (FP32 [param_count]), no update. */
sci_status sci_lprox_grads(const float* params, const float* x, const float* target, int nx, int ny,
                           int B, int count, float* grad, double* loss, void* work, size_t work_bytes,
                           sci_stream_t stream);

/* Scratch bytes for sci_gap_tv_lprox. */
size_t sci_gap_tv_lprox_workspace(int nx, int ny, int B, int count, const sci_params* plain);

/*
 * GAP-TV with the learned prox in place of FGP: T iterations of
 *   x = GAP projection of theta (Eq. 21);  theta = x + f(x)
 * on `count` measurements of the same size (y, bits: [count][nx][ny];
 * theta, x_out: [count][B][nx][ny]; init = 1 starts from Phi^T y).
 * Fallback: when check_every > 0, after every check_every iterations the
 * residual ||y - Phi theta||^2 of each measurement (written to resid_out,
 * host [count][ceil(T/check_every)], nullable) is compared with
 * fallback_ratio x resid_limit[c] (host, the plain method's residual at the
 * same checkpoint, e.g. from a calibration run; nullable = never fall back).
 * A measurement that exceeds it restarts from its last checkpoint with plain
 * GAP-TV (params `plain`, e.g. FGP with S = 10) for the remaining iterations;
 * fell_back (host [count], nullable) reports which did.  With check_every >
 * 0 this call synchronises `stream` at every checkpoint.
 */
sci_status sci_gap_tv_lprox(const float* params, const float* y, const uint32_t* bits, int nx, int ny, int B,
                            int count, int outer_iters, int init, float* theta, float* x_out, int check_every,
                            const double* resid_limit, float fallback_ratio, const sci_params* plain,
                            int* fell_back, double* resid_out, void* work, size_t work_bytes,
                            sci_stream_t stream);

/* Device int in `work` that the tensor-core kernel sets to 1 if a bounded wait
 * gave up (cleared at the start of each call above); read after a sync. */
sci_status sci_lprox_error_word(void* work, size_t work_bytes, int nx, int ny, int B, int count,
                                int training, int** out);

/*
 * The tensor-core building block: a 3x3x3 convolution with 32 input and 32
 * output channels over channels-last BF16 activations [nvol][D][H][W][32]
 * (zero padding), weights BF16 [27][32 out][32 in], FP32 accumulation,
 * output BF16 (relu != 0: + bias[32], then ReLU).  act, w 16-byte aligned.
 * err: device int set to 1 if a bounded wait inside the kernel gave up.
 */
sci_status sci_conv3d_c32_bf16(const void* act, const void* w, const float* bias, int relu, int nvol,
                               int D, int H, int W, void* out, int* err, sci_stream_t stream);

/* Release every CUDA graph the solver has cached (call before freeing buffers
 * whose addresses an earlier solve used, if the same addresses may be reused
 * with different contents sizes or parameters; safe at any time). */
void sci_graph_cache_clear(void);

/* Number of CUDA kernels the calling thread's most recent sci_gap_tv /
 * sci_admm_tv call enqueued (as graph nodes or launches); for accounting. */
long long sci_last_solve_launches(void);

/* FGP dual updates per temporally blocked launch that the solver and
 * sci_tv_prox use for this TV, frame count and params->fuse_k (0: the
 * one-launch-per-update kernels serve; -1: invalid arguments). */
int sci_fused_updates(int tv, int B, int inner_iters, int fuse_k);

/* Tile classes (sci_params.tile) that can run this TV form and frame count,
 * the library's default first: written to out[0..max), the number that fit
 * returned (0 for VTV with B > 24, which runs the per-update kernels). */
int sci_tile_classes(int tv, int B, int* out, int max);

/* sci_fused_updates for a given tile class (0: the default class); -1 for a
 * class that does not fit. */
int sci_fused_updates_tile(int tv, int B, int inner_iters, int fuse_k, int tile);

/* Outer loop that sci_tune_fuse times. */
typedef enum { SCI_ALGO_GAP = 0, SCI_ALGO_ADMM = 1, SCI_ALGO_FISTA = 2 } sci_algo;

/*
 * Fuse-depth autotuner (no counterpart in the paper; it picks the launch
 * shape of its FGP box).  For each of the n_candidates values k in
 * `candidates` (HOST array, each >= -1, as params->fuse_k), runs a solve of
 * probe_iters outer iterations (sci_gap_tv, sci_admm_tv or sci_fista_tv by
 * algo; params->init = 1 and use_graph = 0 are forced) once untimed, then
 * `reps` times, each bracketed by CUDA events recorded on `stream`, and
 * writes the median milliseconds per solve to ms[i] (HOST float array of
 * n_candidates).  *best (HOST int) receives the first candidate with the
 * smallest median.  With FP32 storage every fuse depth gives bit-identical
 * results, so the choice only changes speed; with 16-bit storage the duals
 * carried from one fused launch to the next are rounded to 16 bits, so the
 * depth moves those roundings.  The other arguments are those of the timed
 * solver (u: ADMM only, else ignored); theta (and u) are overwritten with
 * the probe solve's output.  Blocks the calling thread (it synchronises on
 * the events); SCI_ERR_ARG while `stream` is capturing, for
 * 1 <= n_candidates <= 64, 1 <= reps <= 100, 1 <= probe_iters <= 1000 not
 * met, or a NULL host pointer; the timed solver's errors otherwise.
 */
sci_status sci_tune_fuse(int algo, const float* y, const uint32_t* bits, int nx, int ny, int B,
                         const sci_params* params, float* theta, float* u, void* work,
                         size_t work_bytes, const int* candidates, int n_candidates,
                         int probe_iters, int reps, float* ms, int* best, sci_stream_t stream);

/*
 * Launch-shape autotuner: as sci_tune_fuse, over n_candidates pairs
 * (fuse_ks[i], tiles[i]) (HOST arrays; each pair as params->fuse_k and
 * params->tile).  ms[i] receives pair i's median milliseconds per solve and
 * *best (HOST int) the index of the fastest pair.  Same limits and errors as
 * sci_tune_fuse.
 */
sci_status sci_tune_launch(int algo, const float* y, const uint32_t* bits, int nx, int ny, int B,
                           const sci_params* params, float* theta, float* u, void* work, size_t work_bytes,
                           const int* fuse_ks, const int* tiles, int n_candidates, int probe_iters, int reps,
                           float* ms, int* best, sci_stream_t stream);

/*
 * The same for sci_gap_tv_batched: one K for every tile class of the batch
 * (k <= 0 selects the library's default there).  Each problem's theta and
 * x_out are overwritten.  Same limits and errors as sci_tune_fuse.
 */
sci_status sci_tune_fuse_batched(const sci_problem* problems, int count, const sci_params* params,
                                 void* work, size_t work_bytes, const int* candidates,
                                 int n_candidates, int probe_iters, int reps, float* ms, int* best,
                                 sci_stream_t stream);

/* Scratch for the FP64 reductions below: at least this many bytes. */
size_t sci_reduce_workspace(void);

/*
 * out[0] = sum_i (a[i] - b[i])^2 with FP64 accumulation in a fixed order
 * (deterministic).  b may be NULL (then sum a[i]^2).  out: device double.
 * PSNR = 10 log10(peak^2 * n / out[0]) is formed by the caller.
 */
sci_status sci_sqdiff_f64(const float* a, const float* b, size_t n, double* out,
                          void* work, size_t work_bytes, sci_stream_t stream);

/* out[0] = ||y - Phi theta||_2^2 with FP64 accumulation (deterministic). */
sci_status sci_residual_f64(const float* theta, const float* y, const uint32_t* bits,
                            int nx, int ny, int B, double* out, void* work,
                            size_t work_bytes, sci_stream_t stream);

/*
 * sci_tv_prox_noalloc -- the same FGP TV prox as sci_tv_prox, for callers
 * that cannot hand the library any device memory for scratch.  (The paper
 * has no counterpart: this is an interface convenience of this library.)
 *
 * Who needs it: code that must not call cudaMalloc or any allocator at the
 * point of use -- a plugin living inside a host framework that owns all
 * device memory, a latency-critical streaming loop where cudaFree's implicit
 * device synchronisation is unacceptable, or a fixed-budget embedded pipeline
 * that reserves all memory up front.  Such callers still pass x and theta.
 *
 * Scratch: a fixed array of 48 MiB compiled into libsci (three rotating FP32
 * dual buffers, 24 bytes per voxel), so B*nx*ny may be at most
 * sci_tv_prox_noalloc_max_voxels() = 2,097,152 (e.g. 512 x 512 x 8); larger
 * sizes return SCI_ERR_SHAPE before anything is enqueued.  Every GPU that
 * loads the library keeps this array until the process exits.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  The call allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine.
 *
 * All calls share the one array and it keeps the last call's contents; the
 * first dual update overwrites every entry it later reads, so nothing needs
 * clearing.  Calls whose execution overlaps on the GPU (different streams, or
 * different host threads without ordering) race on the array: serialise them.
 * Other arguments, layout and results are exactly those of sci_tv_prox.
 */
sci_status sci_tv_prox_noalloc(const float* x, int nx, int ny, int B, int tv, float lambda,
                               int inner_iters, float* theta, sci_stream_t stream);

/* Largest B*nx*ny that sci_tv_prox_noalloc accepts. */
long long sci_tv_prox_noalloc_max_voxels(void);

#ifdef __cplusplus
}
#endif

#endif /* SCI_H_ */
