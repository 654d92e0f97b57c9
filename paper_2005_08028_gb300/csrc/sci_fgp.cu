// FGP TV proximal map, one dual update per launch (Algorithm 1, ATV-FGP box,
// with the ITV2D / ITV3D dual projections of Eqs. 29-32).
//
// Dual update s (w = p = 0 and nu = 1 before the first):
//   theta = xt - lambda (D_h^T w_h + D_v^T w_v)
//   a     = w + (1/(8 lambda)) (D_h theta, D_v theta)
//   p'    = a / max(1, |a|)    (|.| per entry: ATV, per voxel: ITV2D, per pixel over B frames: VTV)
//   w'    = p' + ((nu_s - 1)/nu_{s+1}) (p' - p)
// and after S updates theta = xt - lambda D^T p.
//
// Only p is stored (three rotating buffers): w at any voxel is recomputed as
// p + c (p - q) from the current and previous iterates, so one update reads
// xt, p, q and writes p' -- 28 bytes per voxel in FP32.
//
// Thread mapping: one thread per pixel (i, j), looping over the B frames (VTV
// needs the whole frame column of a pixel for its norm).  D_h, D_v are forward
// differences without wrap-around; the padded dual entries (last column of
// w_h, last row of w_v) are 0 and stay 0.
#include "sci_internal.cuh"

namespace sci {

template <typename T>
__device__ __forceinline__ float round_trip(float v) {
    T tmp;
    st<T>(&tmp, 0, v);
    return ld<T>(&tmp, 0);
}

// w at linear index idx of one dual component.
template <typename T>
__device__ __forceinline__ float w_at(const T* __restrict__ p, const T* __restrict__ q, bool has_q,
                                      float c, long long idx) {
    const float pv = ld<T>(p, idx);
    if (!has_q) return pv;
    return fmaf(c, pv - ld<T>(q, idx), pv);
}

// theta = xt - lambda (D^T w) at (k, ii, jj); base = k*n + ii*ny + jj.
template <typename T>
__device__ __forceinline__ float theta_at(const T* __restrict__ xt, const T* __restrict__ p,
                                          const T* __restrict__ q, bool has_q, float c, Geo g,
                                          long long N, int ii, int jj, long long base, float lambda) {
    float div = 0.f;
    if (jj >= 1) div += w_at(p, q, has_q, c, base - 1);
    if (jj < g.ny - 1) div -= w_at(p, q, has_q, c, base);
    if (ii >= 1) div += w_at(p + N, q + (has_q ? N : 0), has_q, c, base - g.ny);
    if (ii < g.nx - 1) div -= w_at(p + N, q + (has_q ? N : 0), has_q, c, base);
    return ld<T>(xt, base) - lambda * div;
}

// ---- dual projection helpers ----
__device__ __forceinline__ void proj_atv(float& ah, float& av) {
    ah = fminf(fmaxf(ah, -1.f), 1.f);
    av = fminf(fmaxf(av, -1.f), 1.f);
}
__device__ __forceinline__ void proj_itv(float& ah, float& av) {
    const float den = fmaxf(1.f, sqrtf(ah * ah + av * av));
    ah = ah / den;
    av = av / den;
}

// x-tilde at (k, ii, jj) for the first update.
template <typename T>
__device__ __forceinline__ float xt_first(OuterMode mode, const float* __restrict__ xin,
                                          const T* __restrict__ theta, const float* __restrict__ r,
                                          const uint32_t* __restrict__ bits, Geo g, int k,
                                          long long pix) {
    if (mode == OuterMode::Prox) return xin[k * g.n + pix];
    return round_trip<T>(ld<T>(theta, k * g.n + pix) + mask_bit(bits[pix], k) * r[pix]);
}

// First update: w = 0, so theta = xt and a = (D xt)/(8 lambda).
template <typename T, int TV>
__global__ void k_fgp_first(OuterMode mode, const float* __restrict__ xin, const T* __restrict__ theta,
                            const float* __restrict__ r, const uint32_t* __restrict__ bits, Geo g,
                            float lambda, float step, T* __restrict__ xt, T* __restrict__ pout) {
    int i, j;
    pixel_ij(i, j);
    if (i >= g.nx || j >= g.ny) return;
    const long long N = (long long)g.B * g.n;
    const long long pix = (long long)i * g.ny + j;
    const bool hr = j < g.ny - 1, hd = i < g.nx - 1;
    float nrm2 = 0.f;
    for (int pass = 0; pass < (TV == SCI_TV_VTV ? 2 : 1); ++pass) {
        const float scale = (TV == SCI_TV_VTV && pass == 1) ? 1.f / fmaxf(1.f, sqrtf(nrm2)) : 1.f;
        for (int k = 0; k < g.B; ++k) {
            const float x0 = xt_first<T>(mode, xin, theta, r, bits, g, k, pix);
            const float xr = hr ? xt_first<T>(mode, xin, theta, r, bits, g, k, pix + 1) : x0;
            const float xd = hd ? xt_first<T>(mode, xin, theta, r, bits, g, k, pix + g.ny) : x0;
            float ah = (xr - x0) * step;
            float av = (xd - x0) * step;
            if (TV == SCI_TV_ATV) proj_atv(ah, av);
            else if (TV == SCI_TV_ITV2D) proj_itv(ah, av);
            else if (pass == 0) { nrm2 += ah * ah + av * av; continue; }
            else { ah *= scale; av *= scale; }
            const long long idx = k * g.n + pix;
            if (mode != OuterMode::Prox && pass == (TV == SCI_TV_VTV ? 1 : 0)) st<T>(xt, idx, x0);
            st<T>(pout, idx, ah);
            st<T>(pout, N + idx, av);
        }
    }
}

// Dual update s >= 1 from p = p^(s), q = p^(s-1) (null: w = p), c = (nu_{s-1}-1)/nu_s.
template <typename T, int TV>
__global__ void k_fgp_iter(const T* __restrict__ xt, const T* __restrict__ p, const T* __restrict__ q,
                           float c, Geo g, float lambda, float step, T* __restrict__ pout) {
    int i, j;
    pixel_ij(i, j);
    if (i >= g.nx || j >= g.ny) return;
    const long long N = (long long)g.B * g.n;
    const long long pix = (long long)i * g.ny + j;
    const bool has_q = q != nullptr;
    const bool hr = j < g.ny - 1, hd = i < g.nx - 1;
    float nrm2 = 0.f;
    for (int pass = 0; pass < (TV == SCI_TV_VTV ? 2 : 1); ++pass) {
        const float scale = (TV == SCI_TV_VTV && pass == 1) ? 1.f / fmaxf(1.f, sqrtf(nrm2)) : 1.f;
        for (int k = 0; k < g.B; ++k) {
            const long long base = k * g.n + pix;
            const float t0 = theta_at(xt, p, q, has_q, c, g, N, i, j, base, lambda);
            const float tr = hr ? theta_at(xt, p, q, has_q, c, g, N, i, j + 1, base + 1, lambda) : t0;
            const float td = hd ? theta_at(xt, p, q, has_q, c, g, N, i + 1, j, base + g.ny, lambda) : t0;
            const float wh = hr ? w_at(p, q, has_q, c, base) : 0.f;
            const float wv = hd ? w_at(p + N, q + (has_q ? N : 0), has_q, c, base) : 0.f;
            float ah = fmaf(tr - t0, step, wh);
            float av = fmaf(td - t0, step, wv);
            if (TV == SCI_TV_ATV) proj_atv(ah, av);
            else if (TV == SCI_TV_ITV2D) proj_itv(ah, av);
            else if (pass == 0) { nrm2 += ah * ah + av * av; continue; }
            else { ah *= scale; av *= scale; }
            st<T>(pout, base, ah);
            st<T>(pout, N + base, av);
        }
    }
}

// theta = xt - lambda D^T p, plus the outer-loop epilogue:
//   GAP : x^(t+1) = xt; next residual r = rinv (y - sum_k c_k theta_k)
//   ADMM: u' = xt - theta (= u + x - theta); x^(t+1) = xt - u;
//         next residual r = rinv (y - sum_k c_k (theta_k - u'_k))
//   Prox: theta written as FP32 only.
template <typename T>
__global__ void k_fgp_out(OutArgs a, const T* __restrict__ xt, const T* __restrict__ p, Geo g,
                          float lambda, T* __restrict__ theta, T* __restrict__ u) {
    int i, j;
    pixel_ij(i, j);
    const bool inside = i < g.nx && j < g.ny;
    double d2 = 0.0;
    if (inside) {
        const long long N = (long long)g.B * g.n;
        const long long pix = (long long)i * g.ny + j;
        const uint32_t word = a.bits != nullptr ? a.bits[pix] : 0u;
        float acc = 0.f, acc_theta = 0.f;
        for (int k = 0; k < g.B; ++k) {
            const long long base = k * g.n + pix;
            // D^T p grouped as (p_h left - p_h) + (p_v up - p_v), the order the
            // dual-update kernels use, so both FGP paths round alike
            const float pl = j >= 1 ? ld<T>(p, base - 1) : 0.f;
            const float ph = j < g.ny - 1 ? ld<T>(p, base) : 0.f;
            const float pu = i >= 1 ? ld<T>(p + N, base - g.ny) : 0.f;
            const float pv = i < g.nx - 1 ? ld<T>(p + N, base) : 0.f;
            const float x0 = a.mode == OuterMode::Prox ? a.xin[base] : ld<T>(xt, base);
            const float th = __fmaf_rn(-lambda, (pl - ph) + (pu - pv), x0);
            if (a.mode == OuterMode::Prox) {
                a.theta_f32[base] = th;
                continue;
            }
            st<T>(theta, base, th);
            const float thr = round_trip<T>(th);
            const float ck = mask_bit(word, k);
            acc_theta += ck * thr;
            if (a.mode == OuterMode::Gap) {
                acc = __fmaf_rn(ck, thr, acc);
                if (a.x_out != nullptr) a.x_out[base] = x0;
            } else {
                const float u_old = ld<T>(u, base);
                const float u_new = round_trip<T>(x0 - thr);
                st<T>(u, base, u_new);
                acc = __fmaf_rn(ck, thr - u_new, acc);
                if (a.x_out != nullptr) a.x_out[base] = x0 - u_old;
            }
        }
        if (a.mode != OuterMode::Prox) {
            const float yv = a.y[pix];
            if (a.r_next != nullptr) a.r_next[pix] = a.rinv[pix] * (yv - acc);
            const double d = (double)yv - (double)acc_theta;
            d2 = d * d;
        }
    }
    if (a.resid_partials != nullptr) {
        d2 = block_sum(d2);
        if (threadIdx.x == 0) a.resid_partials[blockIdx.y * gridDim.x + blockIdx.x] = d2;
    }
}

// ---------------------------------------------------------------- launchers

template <typename T>
void launch_fgp_first(int tv, OuterMode mode, const float* xin, const T* theta, const float* r,
                      const uint32_t* bits, Geo g, float lambda, T* xt, T* p_out, cudaStream_t s) {
    const float step = (float)(1.0 / (8.0 * (double)lambda));
    const dim3 grid = pixel_grid(g.nx, g.ny), block = pixel_block();
    switch (tv) {
        case SCI_TV_ATV:
            k_fgp_first<T, SCI_TV_ATV><<<grid, block, 0, s>>>(mode, xin, theta, r, bits, g, lambda, step, xt, p_out);
            break;
        case SCI_TV_ITV2D:
            k_fgp_first<T, SCI_TV_ITV2D><<<grid, block, 0, s>>>(mode, xin, theta, r, bits, g, lambda, step, xt, p_out);
            break;
        default:
            k_fgp_first<T, SCI_TV_VTV><<<grid, block, 0, s>>>(mode, xin, theta, r, bits, g, lambda, step, xt, p_out);
            break;
    }
}

template <typename T>
void launch_fgp_iter(int tv, const T* xt, const T* p, const T* q, float coef, Geo g, float lambda,
                     T* p_out, cudaStream_t s) {
    const float step = (float)(1.0 / (8.0 * (double)lambda));
    const dim3 grid = pixel_grid(g.nx, g.ny), block = pixel_block();
    switch (tv) {
        case SCI_TV_ATV:
            k_fgp_iter<T, SCI_TV_ATV><<<grid, block, 0, s>>>(xt, p, q, coef, g, lambda, step, p_out);
            break;
        case SCI_TV_ITV2D:
            k_fgp_iter<T, SCI_TV_ITV2D><<<grid, block, 0, s>>>(xt, p, q, coef, g, lambda, step, p_out);
            break;
        default:
            k_fgp_iter<T, SCI_TV_VTV><<<grid, block, 0, s>>>(xt, p, q, coef, g, lambda, step, p_out);
            break;
    }
}

int out_partial_count(Geo g) {
    const dim3 grid = pixel_grid(g.nx, g.ny);
    return (int)(grid.x * grid.y);
}

template <typename T>
void launch_fgp_out(const OutArgs& a, const T* xt, const T* p, Geo g, float lambda, T* theta, T* u,
                    cudaStream_t s) {
    k_fgp_out<T><<<pixel_grid(g.nx, g.ny), pixel_block(), 0, s>>>(a, xt, p, g, lambda, theta, u);
}

#define SCI_INST(T)                                                                             \
    template void launch_fgp_first<T>(int, OuterMode, const float*, const T*, const float*,     \
                                      const uint32_t*, Geo, float, T*, T*, cudaStream_t);       \
    template void launch_fgp_iter<T>(int, const T*, const T*, const T*, float, Geo, float, T*,  \
                                     cudaStream_t);                                             \
    template void launch_fgp_out<T>(const OutArgs&, const T*, const T*, Geo, float, T*, T*,     \
                                    cudaStream_t);
SCI_INST(float)
SCI_INST(__nv_bfloat16)
SCI_INST(__half)
#undef SCI_INST

}  // namespace sci
