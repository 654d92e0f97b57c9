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
template <typename T>
void launch_residual_field(const T* theta, const T* u, const float* y, const uint32_t* bits,
                           const float* rinv, Geo g, float* r, cudaStream_t s);
void launch_project(const float* theta, const float* u, const float* y, const uint32_t* bits,
                    Geo g, float rho, float* x, cudaStream_t s);
template <typename Tin, typename Tout>
void launch_cast(const Tin* in, Tout* out, long long count, cudaStream_t s);
void launch_zero(void* p, size_t bytes, cudaStream_t s);
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

}  // namespace sci
