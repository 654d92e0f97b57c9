// Measurement-model kernels: mask packing, Phi x, Phi^T y, the GAP / ADMM
// projection, the per-pixel residual field and FP64 reductions.
//
// Sec. 1 of the paper: Y = sum_k X_k . C_k + G (Eq. 3), Phi = [D_1..D_B] with
// diagonal D_k (Eq. 2), so Phi Phi^T = diag(R), R = sum_k C_k^2, and the GAP
// projection (Eq. 21) and ADMM x-update (Eq. 24) act pixel by pixel.
//
// Every kernel here gives one thread one pixel (i, j) and loops over the B
// frames, so the frame sum of a pixel stays in registers.  A warp covers 32
// consecutive columns: each frame load is one coalesced 128-byte line.
#include <algorithm>

#include <type_traits>

#include "sci_internal.cuh"

namespace sci {

__global__ void k_pack(const uint8_t* __restrict__ masks, Geo g, uint32_t* __restrict__ bits,
                       int* __restrict__ bad) {
    int i, j;
    pixel_ij(i, j);
    if (i >= g.nx || j >= g.ny) return;
    const long long pix = (long long)i * g.ny + j;
    uint32_t w = 0;
    int nbad = 0;
    for (int k = 0; k < g.B; ++k) {
        const uint8_t v = masks[k * g.n + pix];
        if (v != 0) w |= 1u << k;
        nbad += (v > 1);
    }
    bits[pix] = w;
    if (bad != nullptr && nbad) atomicAdd(bad, nbad);
}

__global__ void k_forward(const float* __restrict__ x, const uint32_t* __restrict__ bits, Geo g,
                          float* __restrict__ y) {
    int i, j;
    pixel_ij(i, j);
    if (i >= g.nx || j >= g.ny) return;
    const long long pix = (long long)i * g.ny + j;
    const uint32_t w = bits[pix];
    float acc = 0.f;
    for (int k = 0; k < g.B; ++k) acc += mask_bit(w, k) * x[k * g.n + pix];
    y[pix] = acc;
}

template <typename T>
__global__ void k_adjoint(const float* __restrict__ y, const uint32_t* __restrict__ bits, Geo g,
                          T* __restrict__ x) {
    int i, j;
    pixel_ij(i, j);
    if (i >= g.nx || j >= g.ny) return;
    const long long pix = (long long)i * g.ny + j;
    const uint32_t w = bits[pix];
    const float yv = y[pix];
    for (int k = 0; k < g.B; ++k) st<T>(x, k * g.n + pix, mask_bit(w, k) * yv);
}

// 1/(R + rho) in FP64, rounded to FP32; 0 where R + rho == 0 (pseudo-inverse).
__global__ void k_rinv(const uint32_t* __restrict__ bits, Geo g, float rho, float* __restrict__ rinv) {
    const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= g.n) return;
    const uint32_t mask = g.B >= 32 ? 0xffffffffu : ((1u << g.B) - 1u);
    const double R = (double)__popc(bits[pix] & mask) + (double)rho;
    rinv[pix] = R == 0.0 ? 0.f : (float)(1.0 / R);
}

// FISTA's step (Sec. 2.2): 1/L with L = ||Phi||^2 = max_ij R_ij.  k_mask_max
// takes the largest mask count into *lmax (zeroed by the caller); k_fill_step
// writes 1/L (0 when no pixel is measured) in every pixel of the field the
// GAP residual kernels scale by, so they form z = theta + (1/L) Phi^T (y - Phi theta).
__global__ void k_mask_max(const uint32_t* __restrict__ bits, Geo g, unsigned* __restrict__ lmax) {
    const uint32_t mask = g.B >= 32 ? 0xffffffffu : ((1u << g.B) - 1u);
    unsigned m = 0;
    for (long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x; pix < g.n;
         pix += (long long)gridDim.x * blockDim.x)
        m = max(m, (unsigned)__popc(bits[pix] & mask));
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) atomicMax(lmax, m);
}

__global__ void k_fill_step(const unsigned* __restrict__ lmax, Geo g, float* __restrict__ rinv) {
    const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= g.n) return;
    const unsigned L = *lmax;
    rinv[pix] = L == 0 ? 0.f : (float)(1.0 / (double)L);
}

// TwIST's alpha, beta (Sec. 2.2, TwIST steps) for the normalised operator
// A = Phi / sqrt(L): the eigenvalues of A^T A are 0 (its nullspace) and
// R_ij / L, so xi_m = 1 and xi_1 = min_{R > 0} R / max R.  k_mask_min_pos
// takes the smallest nonzero mask count into *cmin (set to ~0 by the
// caller); k_twist_coef then forms, in FP64 on one thread,
//   kappa = xi_1, rho = (1 - sqrt(kappa)) / (1 + sqrt(kappa)),
//   alpha = 1 + rho^2, beta = 2 alpha / (1 + xi_1)
// and stores the combination weights (1 - alpha, alpha - beta, beta) as FP32.
__global__ void k_mask_min_pos(const uint32_t* __restrict__ bits, Geo g, unsigned* __restrict__ cmin) {
    const uint32_t mask = g.B >= 32 ? 0xffffffffu : ((1u << g.B) - 1u);
    unsigned m = 0xffffffffu;
    for (long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x; pix < g.n;
         pix += (long long)gridDim.x * blockDim.x) {
        const unsigned c = (unsigned)__popc(bits[pix] & mask);
        if (c > 0) m = min(m, c);
    }
    m = __reduce_min_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) atomicMin(cmin, m);
}

__global__ void k_twist_coef(const unsigned* __restrict__ lmax, const unsigned* __restrict__ cmin,
                             float* __restrict__ w3) {
    const unsigned L = *lmax, c = *cmin;
    const double xi1 = (L == 0 || c == 0xffffffffu) ? 1.0 : (double)c / (double)L;
    const double sk = sqrt(xi1);
    const double rho = (1.0 - sk) / (1.0 + sk);
    const double alpha = 1.0 + rho * rho;
    const double beta = 2.0 * alpha / (1.0 + xi1);
    w3[0] = (float)(1.0 - alpha);
    w3[1] = (float)(alpha - beta);
    w3[2] = (float)beta;
}

// TwIST's two-step update, written over x_prev:
//   x_next = theta (first iteration: one plain step)
//   x_next = (1 - alpha) x_prev + (alpha - beta) x + beta theta   (later ones)
// as fma(beta, theta, fma(alpha - beta, x, (1 - alpha) x_prev)) in FP32.
template <typename T>
__global__ void k_twist_step(T* __restrict__ x_prev, const T* __restrict__ x, const T* __restrict__ theta,
                             const float* __restrict__ w3, long long n, int first) {
    const float c0 = w3[0], c1 = w3[1], c2 = w3[2];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float th = ld<T>(theta, i);
        const float xn = first ? th : fmaf(c2, th, fmaf(c1, ld<T>(x, i), c0 * ld<T>(x_prev, i)));
        st<T>(x_prev, i, xn);
    }
}

// FISTA momentum: theta_next = x + beta (x - x_prev), then x_prev = x.
template <typename T>
__global__ void k_fista_momentum(const T* __restrict__ x, T* __restrict__ x_prev, T* __restrict__ theta_next,
                                 long long n, float beta) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float xv = ld<T>(x, i), xp = ld<T>(x_prev, i);
        st<T>(theta_next, i, fmaf(beta, xv - xp, xv));
        st<T>(x_prev, i, xv);
    }
}

// r = rinv * (y - sum_k c_k (theta_k - u_k)); u may be null.
template <typename T>
__global__ void k_residual_field(const T* __restrict__ theta, const T* __restrict__ u,
                                 const float* __restrict__ y, const uint32_t* __restrict__ bits,
                                 const float* __restrict__ rinv, Geo g, float* __restrict__ r) {
    int i, j;
    pixel_ij(i, j);
    if (i >= g.nx || j >= g.ny) return;
    const long long pix = (long long)i * g.ny + j;
    const uint32_t w = bits[pix];
    float acc = 0.f;
    for (int k = 0; k < g.B; ++k) {
        float v = ld<T>(theta, k * g.n + pix);
        if (u != nullptr) v -= ld<T>(u, k * g.n + pix);
        acc = __fmaf_rn(mask_bit(w, k), v, acc);
    }
    r[pix] = rinv[pix] * (y[pix] - acc);
}

// The same residual for four consecutive pixels per thread, with 128-bit
// loads of the fields (64-bit for 16-bit storage), when the frame size is a
// multiple of 4 (frames then start 16-byte aligned).  Each pixel's sum runs
// over k in the same order as above.
template <typename T> struct vec4_of;
template <> struct vec4_of<float> { using type = float4; };
template <> struct vec4_of<__half> { using type = uint2; };
template <> struct vec4_of<__nv_bfloat16> { using type = uint2; };

template <typename T>
__device__ __forceinline__ void ld4(const T* p, long long i, float (&v)[4]) {
    if constexpr (std::is_same<T, float>::value) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p + i));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else {
        const uint2 a = __ldg(reinterpret_cast<const uint2*>(p + i));
        const unsigned short h[4] = {(unsigned short)(a.x & 0xffffu), (unsigned short)(a.x >> 16),
                                     (unsigned short)(a.y & 0xffffu), (unsigned short)(a.y >> 16)};
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = cvraw<T>(__uint_as_float((unsigned)h[e]));
    }
}

template <typename T>
__global__ void k_residual_field4(const T* __restrict__ theta, const T* __restrict__ u,
                                  const float* __restrict__ y, const uint32_t* __restrict__ bits,
                                  const float* __restrict__ rinv, Geo g, float* __restrict__ r) {
    const long long n4 = g.n >> 2;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n4;
         q += (long long)gridDim.x * blockDim.x) {
        const long long pix = q << 2;
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(bits + pix));
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < g.B; ++k) {
            float v[4];
            ld4<T>(theta, k * g.n + pix, v);
            if (u != nullptr) {
                float uu[4];
                ld4<T>(u, k * g.n + pix, uu);
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] -= uu[e];
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[e] = __fmaf_rn(mask_bit(ws[e], k), v[e], acc[e]);
        }
        const float4 yv = __ldg(reinterpret_cast<const float4*>(y + pix));
        const float4 ri = __ldg(reinterpret_cast<const float4*>(rinv + pix));
        *reinterpret_cast<float4*>(r + pix) =
            make_float4(ri.x * (yv.x - acc[0]), ri.y * (yv.y - acc[1]), ri.z * (yv.z - acc[2]), ri.w * (yv.w - acc[3]));
    }
}

// Number of entries of a that are NaN or +-Inf, added to *count.
__global__ void k_count_nonfinite(const float* __restrict__ a, long long n, unsigned* __restrict__ count) {
    unsigned c = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        c += isfinite(a[i]) ? 0u : 1u;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// x = v + c_k * (y - sum_k c_k v_k) / (R + rho), v = theta - u.
__global__ void k_project(const float* __restrict__ theta, const float* __restrict__ u,
                          const float* __restrict__ y, const uint32_t* __restrict__ bits, Geo g,
                          float rho, float* __restrict__ x) {
    int i, j;
    pixel_ij(i, j);
    if (i >= g.nx || j >= g.ny) return;
    const long long pix = (long long)i * g.ny + j;
    const uint32_t w = bits[pix];
    float acc = 0.f;
    for (int k = 0; k < g.B; ++k) {
        float v = theta[k * g.n + pix];
        if (u != nullptr) v -= u[k * g.n + pix];
        acc += mask_bit(w, k) * v;
    }
    const uint32_t mask = g.B >= 32 ? 0xffffffffu : ((1u << g.B) - 1u);
    const double R = (double)__popc(w & mask) + (double)rho;
    const float rinv = R == 0.0 ? 0.f : (float)(1.0 / R);
    const float rr = rinv * (y[pix] - acc);
    for (int k = 0; k < g.B; ++k) {
        float v = theta[k * g.n + pix];
        if (u != nullptr) v -= u[k * g.n + pix];
        x[k * g.n + pix] = v + mask_bit(w, k) * rr;
    }
}

template <typename Tin, typename Tout>
__global__ void k_cast(const Tin* __restrict__ in, Tout* __restrict__ out, long long count) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < count;
         idx += (long long)gridDim.x * blockDim.x)
        st<Tout>(out, idx, ld<Tin>(in, idx));
}

// ---- FP64 reductions (fixed order: per-thread strided sums, warp shuffle,
// per-block tree, then one block sums the partials in index order) ----
__global__ void k_sqdiff_partial(const float* __restrict__ a, const float* __restrict__ b,
                                 long long n, double* __restrict__ partials) {
    double acc = 0.0;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const double d = (double)a[idx] - (b != nullptr ? (double)b[idx] : 0.0);
        acc += d * d;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

template <typename T>
__global__ void k_resid_partial(const T* __restrict__ theta, const float* __restrict__ y,
                                const uint32_t* __restrict__ bits, Geo g,
                                double* __restrict__ partials) {
    double acc = 0.0;
    for (long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x; pix < g.n;
         pix += (long long)gridDim.x * blockDim.x) {
        const uint32_t w = bits[pix];
        float s = 0.f;
        for (int k = 0; k < g.B; ++k) s += mask_bit(w, k) * ld<T>(theta, k * g.n + pix);
        const double d = (double)y[pix] - (double)s;
        acc += d * d;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void k_sum_partials(const double* __restrict__ partials, int count, double* __restrict__ out) {
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < count; idx += blockDim.x) acc += partials[idx];
    acc = block_sum(acc);
    if (threadIdx.x == 0) out[0] = acc;
}

// x_out = xt (GAP) or xt - x_out (ADMM: x_out holds u_old in FP32), for 16-bit storage.
template <typename T>
__global__ void k_xt_minus(const T* __restrict__ xt, float* __restrict__ x, long long N, bool sub) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = ld<T>(xt, i);
        x[i] = sub ? v - x[i] : v;
    }
}
void launch_xt_minus(const void* xt, int storage, float* x, long long N, bool sub, cudaStream_t s) {
    const int blocks = 152 * 8;
    if (storage == SCI_BF16)
        k_xt_minus<__nv_bfloat16><<<blocks, 256, 0, s>>>((const __nv_bfloat16*)xt, x, N, sub);
    else if (storage == SCI_F16)
        k_xt_minus<__half><<<blocks, 256, 0, s>>>((const __half*)xt, x, N, sub);
    else
        k_xt_minus<float><<<blocks, 256, 0, s>>>((const float*)xt, x, N, sub);
}

// ---------------------------------------------------------------- launchers

void launch_pack(const uint8_t* masks, Geo g, uint32_t* bits, int* bad, cudaStream_t s) {
    k_pack<<<pixel_grid(g.nx, g.ny), pixel_block(), 0, s>>>(masks, g, bits, bad);
}

void launch_forward(const float* x, const uint32_t* bits, Geo g, float* y, cudaStream_t s) {
    k_forward<<<pixel_grid(g.nx, g.ny), pixel_block(), 0, s>>>(x, bits, g, y);
}

template <typename T>
void launch_adjoint(const float* y, const uint32_t* bits, Geo g, T* x, cudaStream_t s) {
    k_adjoint<T><<<pixel_grid(g.nx, g.ny), pixel_block(), 0, s>>>(y, bits, g, x);
}

void launch_rinv(const uint32_t* bits, Geo g, float rho, float* rinv, cudaStream_t s) {
    const int threads = 256;
    const long long blocks = (g.n + threads - 1) / threads;
    k_rinv<<<(unsigned)blocks, threads, 0, s>>>(bits, g, rho, rinv);
}

void launch_fista_step(const uint32_t* bits, Geo g, unsigned* lmax, float* rinv, cudaStream_t s) {
    const int threads = 256;
    const long long blocks = (g.n + threads - 1) / threads;
    cudaMemsetAsync(lmax, 0, sizeof(unsigned), s);
    k_mask_max<<<(unsigned)std::min<long long>(blocks, 152 * 8), threads, 0, s>>>(bits, g, lmax);
    k_fill_step<<<(unsigned)blocks, threads, 0, s>>>(lmax, g, rinv);
}

void launch_twist_coef(const uint32_t* bits, Geo g, unsigned* counts, float* w3, cudaStream_t s) {
    const int threads = 256;
    const long long blocks = (g.n + threads - 1) / threads;
    cudaMemsetAsync(counts + 1, 0xff, sizeof(unsigned), s);
    k_mask_min_pos<<<(unsigned)std::min<long long>(blocks, 152 * 8), threads, 0, s>>>(bits, g, counts + 1);
    k_twist_coef<<<1, 1, 0, s>>>(counts, counts + 1, w3);
}

template <typename T>
void launch_twist_step(T* x_prev, const T* x, const T* theta, const float* w3, long long n, bool first,
                       cudaStream_t s) {
    const int threads = 256;
    long long blocks = (n + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_twist_step<T><<<(unsigned)std::max(blocks, 1LL), threads, 0, s>>>(x_prev, x, theta, w3, n, first ? 1 : 0);
}
template void launch_twist_step<float>(float*, const float*, const float*, const float*, long long, bool,
                                       cudaStream_t);
template void launch_twist_step<__nv_bfloat16>(__nv_bfloat16*, const __nv_bfloat16*, const __nv_bfloat16*,
                                               const float*, long long, bool, cudaStream_t);
template void launch_twist_step<__half>(__half*, const __half*, const __half*, const float*, long long, bool,
                                        cudaStream_t);

template <typename T>
void launch_fista_momentum(const T* x, T* x_prev, T* theta_next, long long n, float beta, cudaStream_t s) {
    const int threads = 256;
    long long blocks = (n + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_fista_momentum<T><<<(unsigned)std::max(blocks, 1LL), threads, 0, s>>>(x, x_prev, theta_next, n, beta);
}
template void launch_fista_momentum<float>(const float*, float*, float*, long long, float, cudaStream_t);
template void launch_fista_momentum<__nv_bfloat16>(const __nv_bfloat16*, __nv_bfloat16*, __nv_bfloat16*, long long,
                                                   float, cudaStream_t);
template void launch_fista_momentum<__half>(const __half*, __half*, __half*, long long, float, cudaStream_t);

template <typename T>
void launch_residual_field(const T* theta, const T* u, const float* y, const uint32_t* bits,
                           const float* rinv, Geo g, float* r, cudaStream_t s) {
    // The four-pixel form moved the same bytes with a quarter of the threads
    // and measured slower on the L2-resident 512 x 512 x 10 fields (7.8 against
    // 6.5 us per launch), so it serves only fields too large for L2, where
    // fewer, wider requests keep HBM busy with fewer instructions.
    const bool aligned = ((uintptr_t)theta | (uintptr_t)y | (uintptr_t)bits | (uintptr_t)rinv | (uintptr_t)r |
                          (uintptr_t)u) % 16 == 0;
    const long long field_bytes = (long long)g.B * g.n * (long long)sizeof(T);
    if (g.n % 4 == 0 && aligned && field_bytes > (64LL << 20)) {
        const int threads = 256;
        long long blocks = (g.n / 4 + threads - 1) / threads;
        if (blocks > 152 * 16) blocks = 152 * 16;
        k_residual_field4<T><<<(unsigned)std::max(blocks, 1LL), threads, 0, s>>>(theta, u, y, bits, rinv, g, r);
        return;
    }
    k_residual_field<T><<<pixel_grid(g.nx, g.ny), pixel_block(), 0, s>>>(theta, u, y, bits, rinv, g, r);
}

void launch_project(const float* theta, const float* u, const float* y, const uint32_t* bits,
                    Geo g, float rho, float* x, cudaStream_t s) {
    k_project<<<pixel_grid(g.nx, g.ny), pixel_block(), 0, s>>>(theta, u, y, bits, g, rho, x);
}

template <typename Tin, typename Tout>
void launch_cast(const Tin* in, Tout* out, long long count, cudaStream_t s) {
    const int threads = 256;
    long long blocks = (count + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_cast<Tin, Tout><<<(unsigned)blocks, threads, 0, s>>>(in, out, count);
}

void launch_zero(void* p, size_t bytes, cudaStream_t s) { cudaMemsetAsync(p, 0, bytes, s); }

void launch_count_nonfinite(const float* a, long long n, unsigned* count, cudaStream_t s) {
    if (n <= 0) return;
    const int threads = 256;
    long long blocks = (n + threads - 1) / threads;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_count_nonfinite<<<(unsigned)blocks, threads, 0, s>>>(a, n, count);
}

static int reduce_blocks(long long n) {
    long long b = (n + 255) / 256;
    if (b > kReduceParts) b = kReduceParts;
    if (b < 1) b = 1;
    return (int)b;
}

void launch_sqdiff(const float* a, const float* b, long long n, double* partials, double* out,
                   cudaStream_t s) {
    const int blocks = reduce_blocks(n);
    k_sqdiff_partial<<<blocks, 256, 0, s>>>(a, b, n, partials);
    k_sum_partials<<<1, 1024, 0, s>>>(partials, blocks, out);
}

template <typename T>
void launch_residual_norm(const T* theta, const float* y, const uint32_t* bits, Geo g,
                          double* partials, double* out, cudaStream_t s) {
    const int blocks = reduce_blocks(g.n);
    k_resid_partial<T><<<blocks, 256, 0, s>>>(theta, y, bits, g, partials);
    k_sum_partials<<<1, 1024, 0, s>>>(partials, blocks, out);
}

void launch_sum_partials(const double* partials, int count, double* out, cudaStream_t s) {
    k_sum_partials<<<1, 1024, 0, s>>>(partials, count, out);
}

#define SCI_INST(T)                                                                           \
    template void launch_adjoint<T>(const float*, const uint32_t*, Geo, T*, cudaStream_t);    \
    template void launch_residual_field<T>(const T*, const T*, const float*, const uint32_t*, \
                                           const float*, Geo, float*, cudaStream_t);          \
    template void launch_residual_norm<T>(const T*, const float*, const uint32_t*, Geo,       \
                                          double*, double*, cudaStream_t);
SCI_INST(float)
SCI_INST(__nv_bfloat16)
SCI_INST(__half)
#undef SCI_INST
template void launch_cast<float, __nv_bfloat16>(const float*, __nv_bfloat16*, long long, cudaStream_t);
template void launch_cast<__nv_bfloat16, float>(const __nv_bfloat16*, float*, long long, cudaStream_t);
template void launch_cast<float, __half>(const float*, __half*, long long, cudaStream_t);
template void launch_cast<__half, float>(const __half*, float*, long long, cudaStream_t);

}  // namespace sci
