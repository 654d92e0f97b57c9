// Internal launchers shared by the libsci translation units (not exported).
#pragma once

#include "sci_common.cuh"

namespace sci {

// ---- measurement-model kernels (sci_ops.cu) ----
void launch_pack(const uint8_t* masks, Geo g, uint32_t* bits, int* bad, cudaStream_t s);
void launch_forward(const float* x, const uint32_t* bits, Geo g, float* y, cudaStream_t s);
template <typename T>
void launch_adjoint(const float* y, const uint32_t* bits, Geo g, T* x, cudaStream_t s);
void launch_rinv(const uint32_t* bits, Geo g, float rho, float* rinv, cudaStream_t s);
// FISTA (Sec. 2.2): rinv = 1/L in every pixel, L = max mask count (lmax: one
// device word of scratch); theta_next = x + beta (x - x_prev), x_prev = x.
void launch_fista_step(const uint32_t* bits, Geo g, unsigned* lmax, float* rinv, cudaStream_t s);
template <typename T>
void launch_fista_momentum(const T* x, T* x_prev, T* theta_next, long long n, float beta, cudaStream_t s);
// TwIST (Sec. 2.2): counts[0] = max mask count (launch_fista_step), counts[1]
// = smallest nonzero count; w3 = (1 - alpha, alpha - beta, beta) on the device.
// The step overwrites x_prev with x_next.
void launch_twist_coef(const uint32_t* bits, Geo g, unsigned* counts, float* w3, cudaStream_t s);
template <typename T>
void launch_twist_step(T* x_prev, const T* x, const T* theta, const float* w3, long long n, bool first,
                       cudaStream_t s);
template <typename T>
void launch_residual_field(const T* theta, const T* u, const float* y, const uint32_t* bits,
                           const float* rinv, Geo g, float* r, cudaStream_t s);
void launch_project(const float* theta, const float* u, const float* y, const uint32_t* bits,
                    Geo g, float rho, float* x, cudaStream_t s);
template <typename Tin, typename Tout>
void launch_cast(const Tin* in, Tout* out, long long count, cudaStream_t s);
void launch_zero(void* p, size_t bytes, cudaStream_t s);
// *count += number of NaN / Inf entries of a[0..n)
void launch_count_nonfinite(const float* a, long long n, unsigned* count, cudaStream_t s);
// x = xt (sub = false) or x = xt - x (sub = true), xt in the given storage type.
void launch_xt_minus(const void* xt, int storage, float* x, long long N, bool sub, cudaStream_t s);

// FP64 reductions: partials has room for kReduceParts doubles.
constexpr int kReduceParts = 1024;
void launch_sqdiff(const float* a, const float* b, long long n, double* partials,
                   double* out, cudaStream_t s);
template <typename T>
void launch_residual_norm(const T* theta, const float* y, const uint32_t* bits, Geo g,
                          double* partials, double* out, cudaStream_t s);

// ---- FGP TV prox kernels (sci_fgp.cu) ----
enum class OuterMode : int { Prox = 0, Gap = 1, Admm = 2 };

// Kernel code for the ATV-Clip box (Algorithm 1), passed where the dual-update
// kernels take a sci_tv_type.  With the duals scaled by the threshold lambda
// (|w| <= 1), the box is the ATV dual step without momentum, step
// 1/(alpha lambda), whose horizontal gradient reads theta_h = xt - lambda
// D_h^T w_h and vertical one theta_v = xt - lambda D_v^T w_v; its output is
// the FGP box's, xt - lambda D^T w.
constexpr int kTvClip = 3;
constexpr double kClipAlpha = 4.0;

struct FgpFields {
    void* xt;      // x-tilde, the prox input, storage type [B][nx][ny]
    void* p[3];    // three rotating dual buffers, each holds h then v: 2*N elements
};

// First dual update (w = p = 0).  In Prox mode x-tilde is read from `xin`
// (FP32) and not written; otherwise x-tilde = theta + c_k * r is formed,
// written to fields.xt, and used.
template <typename T>
void launch_fgp_first(int tv, OuterMode mode, const float* xin, const T* theta,
                      const float* r, const uint32_t* bits, Geo g, float lambda,
                      T* xt, T* p_out, cudaStream_t s);
// Dual update s >= 1: w = p + coef (p - q); q may be null (then w = p).
template <typename T>
void launch_fgp_iter(int tv, const T* xt, const T* p, const T* q, float coef, Geo g,
                     float lambda, T* p_out, cudaStream_t s);
// One dual update streamed through 32x8 shared-memory halo tiles
// (sci_stream.cu): first = 1 starts from w = 0 and forms x-tilde (Prox: from
// xin; otherwise theta + c_k r, written to xt); later updates read xt and
// w = p + coef (p - q) (q may be null).
template <typename T>
void launch_fgp_stream(int tv, OuterMode mode, int first, const float* xin, const T* theta, const float* r,
                       const uint32_t* bits, Geo g, float lambda, float coef, T* xt, const T* p, const T* q,
                       T* pout, cudaStream_t s);
// Output theta = xt - lambda D^T p and the outer-loop epilogue.
struct OutArgs {
    OuterMode mode;
    const float* xin;       // Prox mode: FP32 x-tilde
    float* theta_f32;       // Prox mode: FP32 output
    const float* y;
    const uint32_t* bits;
    const float* rinv;      // 1/R (GAP) or 1/(R + rho) (ADMM)
    float* r_next;          // residual field for the next projection (may be null)
    float* x_out;           // FP32 x^(t+1) (may be null)
    double* resid_partials; // per-block partials of ||y - Phi theta||^2 (may be null)
};
template <typename T>
void launch_fgp_out(const OutArgs& a, const T* xt, const T* p, Geo g, float lambda,
                    T* theta, T* u, cudaStream_t s);
void launch_sum_partials(const double* partials, int count, double* out, cudaStream_t s);
int out_partial_count(Geo g);

// ---- temporally blocked FGP (sci_fused.cuh, instantiated by sci_fused_{f32,f16,bf16}.cu) ----
constexpr int kMaxFuse = 32;  // dual updates per fused launch
struct FusedArgs {
    Geo g;
    OuterMode mode;
    int K;                  // dual updates in this launch
    int halo;               // top / left tile halo, >= K + 1 (bottom / right: halo - 1)
    int first;              // 1: w = p = 0 and x-tilde formed here (from theta, r or xin)
    int last;               // 1: write theta (and u, x_out); 0: carry p, w (and x-tilde)
    int warm;               // dual warm start: the first launch starts from w = warm_in (p = 0),
                            // the last one also writes its final w to warm_out
    int cls;                // tile class to launch (0: the library's choice for the TV form and B)
    float lambda, step;     // lambda and 1/(8 lambda)
    float coef[kMaxFuse];   // momentum coefficients of this launch's updates
    const float* xin;       // Prox mode: the prox input
    float* theta_f32;       // Prox mode: the prox output
    const uint32_t* bits;   // Gap / Admm: packed masks
    const float* r;         // Gap / Admm: residual field
    float* x_out;           // optional FP32 x^(t+1) (last launch only)
    // Gap / Admm, last launch of a VTV tile (all frames of a pixel in one
    // thread): the next projection's residual field r_next = rinv (y - sum_k
    // c_k (theta'_k - u'_k)) at the tile's interior pixels (null: not formed)
    float* r_next;
    const float* y;
    const float* rinv;
};
// Buffers of one fused launch.  A CTA reads its whole extended tile but
// writes only its interior, so whatever a launch reads from a neighbour's
// interior must not be written by the same launch: theta and the carried dual
// state (p_h, p_v, w_h, w_v) therefore ping-pong between two buffers.
template <typename T>
struct FusedBufs {
    const T* theta_in;  // Gap / Admm: theta^(t) (read with halos by the first launch)
    const T* u_in;      // Admm: u^(t) (read at the thread's own voxels by the last launch)
    T* theta_out;       // must not alias theta_in
    T* u_out;           // may alias u_in (the same thread reads, then writes)
    T* xt;              // x-tilde, written by the first launch, read by later ones
    const T* st_in[4];  // carried p_h, p_v, w_h, w_v (read by non-first launches)
    T* st_out[4];       // must not alias st_in (written by non-last launches)
    const T* warm_in[2];  // dual warm start: w_h, w_v the previous TVdenoise ended with
    T* warm_out[2];       // w_h, w_v this TVdenoise ends with (must not alias warm_in)
};
// One problem of a batched launch (device-resident table entry).
template <typename T>
struct BatchItem {
    Geo g;
    int cls;                 // tile configuration class (fused_class)
    int tiles_x, tiles_y;    // tile grid per frame (one-frame classes) or per problem
    int cta_begin;           // first fused work item of this problem
    int pix_begin;           // first 256-pixel block of this problem (pixel kernels)
    const float* y;
    const uint32_t* bits;
    float* rinv;             // 1/R (pseudo-inverse)
    float* r;                // residual field
    float* x_out;            // optional FP32 x^(T)
    float* theta_user;       // the caller's FP32 theta
    T* theta[2];             // ping-pong theta buffers
    T* xt;
    T* st[2][4];             // ping-pong carried duals (p_h, p_v, w_h, w_v)
};
// Default dual updates per fused launch for this TV form (sci_batch.cu).
int default_fuse(int tv);

// Interior rows (columns) of a fused tile of `extent` rows (columns) whose
// top (left) halo is `halo` and bottom (right) halo is halo - 1.
__host__ __device__ inline int fused_interior(int extent, int halo) { return extent - 2 * halo + 1; }

// Largest halo the fused kernel supports for this TV / frame count (0: none).
int fused_max_halo(int tv, int B);
// Tile classes: 1 = one-frame 64 x 128 (512 threads x 16 rows), 2 = one-frame
// 32 x 64 (256 x 8), 8 / 10 = VTV 32 x 32 for up to 8 / 10 frames, 16 / 24 =
// VTV 32 x 16 for up to 16 / 24 frames.  Whether a class runs this TV form
// and frame count, and the largest halo its tile allows.
bool fused_class_fits(int tv, int B, int cls);
int fused_class_max_halo(int cls);
// Tile configuration class for this TV / frame count (0: none) and its tile size.
int fused_class(int tv, int B);
void fused_class_dims(int cls, int* EH, int* EW);
// One launch over every tile of the problems items[0..nitems) (all of class cls).
template <typename T>
bool launch_fgp_fused_batched(int tv, int cls, const FusedArgs& a, const BatchItem<T>* items, int nitems,
                              int total, int tpar, int spar, int want_x, cudaStream_t s);
template <typename T>
bool launch_fgp_fused(int tv, const FusedArgs& a, const FusedBufs<T>& b, cudaStream_t s);

}  // namespace sci
