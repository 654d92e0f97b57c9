// One FGP dual update per launch, streamed through shared-memory halo tiles
// (Algorithm 1, ATV-FGP box; Eqs. 29-32 for ITV2D / VTV).
//
// A CTA owns a 32 x 8 pixel tile (one pixel per thread).  For each frame it
// stages, with a one-pixel halo, the momentum point w = p + c (p - q) and
// x-tilde in shared memory, forms theta = xt - lambda D^T w on the tile plus
// its right column and bottom row, then each thread forms
// a = w + (1/(8 lambda)) D theta for its pixel.  ATV / ITV2D project and
// store per frame (frames are independent: blockIdx.z picks one).  VTV keeps
// a for all frames of the pixel in registers, takes the norm over frames and
// stores once.  Every value is read from global memory about once per update
// (halo re-reads: 1.33x for w, 1.16x for xt), so the kernel streams at the
// memory system's rate; it needs little on-chip state, which keeps many
// warps resident and suits frame counts too large for the temporally blocked
// kernel.
#include "sci_internal.cuh"

namespace sci {

namespace {

constexpr int TW = 32, TH = 8;

template <typename T>
__device__ __forceinline__ float rt_s(float v) {
    T tmp;
    st<T>(&tmp, 0, v);
    return ld<T>(&tmp, 0);
}

struct StreamArgs {
    Geo g;
    int first;            // 1: w = p = 0, x-tilde formed here
    OuterMode mode;       // Prox: x-tilde read from xin; Gap / Admm: theta + c_k r
    float lambda, step, c;  // c: momentum coefficient of w = p + c (p - q)
    const float* xin;
    const uint32_t* bits;
    const float* r;
};

template <typename T>
__device__ __forceinline__ float xt_at(const StreamArgs& a, const T* theta, const T* xt, int f, long long pix) {
    const long long idx = (long long)f * a.g.n + pix;
    if (a.mode == OuterMode::Prox) return a.xin[idx];
    if (a.first) return rt_s<T>(ld<T>(theta, idx) + mask_bit(a.bits[pix], f) * a.r[pix]);
    return ld<T>(xt, idx);
}

template <typename T, int TV, int FMAX>
__global__ void __launch_bounds__(256) k_fgp_stream(StreamArgs a, const T* __restrict__ theta, T* xt,
                                                    const T* __restrict__ p, const T* __restrict__ q,
                                                    T* __restrict__ pout) {
    __shared__ float s_wh[TH + 2][TW + 2], s_wv[TH + 2][TW + 2];  // rows -1..TH, cols -1..TW
    __shared__ float s_x[TH + 1][TW + 1], s_th[TH + 1][TW + 1];   // rows 0..TH, cols 0..TW
    constexpr bool CLIP = TV == kTvClip;                             // s_th: theta_h, s_tv: theta_v
    __shared__ float s_tv[CLIP ? TH + 1 : 1][CLIP ? TW + 1 : 1];
    const Geo g = a.g;
    const long long N = (long long)g.B * g.n;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int i0 = blockIdx.y * TH, j0 = blockIdx.x * TW;
    const int gi = i0 + ty, gj = j0 + tx;
    const bool in = gi < g.nx && gj < g.ny;
    const long long mypix = in ? (long long)gi * g.ny + gj : 0;
    const bool mh = in && gj < g.ny - 1, mv = in && gi < g.nx - 1;
    const int nfr = (TV == SCI_TV_VTV) ? g.B : 1;
    const int fbase = (TV == SCI_TV_VTV) ? 0 : blockIdx.z;
    const bool has_q = q != nullptr;

    float ah_r[FMAX], av_r[FMAX];
    // VTV norm: the frames of each parity accumulate separately and the two
    // sums are added at the end (the order the temporally blocked kernel's
    // packed frame pairs follow)
    float n2e = 0.f, n2o = 0.f;
#pragma unroll
    for (int ff = 0; ff < FMAX; ++ff) {
        if (ff >= nfr) break;
        const int f = fbase + ff;
        // ---- stage w (one-pixel halo) and x-tilde (plus right column and bottom row) ----
        for (int e = threadIdx.x; e < (TH + 2) * (TW + 2); e += 256) {
            const int rr = e / (TW + 2), cc = e % (TW + 2);
            const int ii = i0 - 1 + rr, jj = j0 - 1 + cc;
            float wh = 0.f, wv = 0.f;
            if (!a.first && ii >= 0 && ii < g.nx && jj >= 0 && jj < g.ny) {
                const long long idx = (long long)f * g.n + (long long)ii * g.ny + jj;
                const float ph = ld<T>(p, idx), pv = ld<T>(p, N + idx);
                if (has_q) {
                    wh = fmaf(a.c, ph - ld<T>(q, idx), ph);
                    wv = fmaf(a.c, pv - ld<T>(q, N + idx), pv);
                } else {
                    wh = ph;
                    wv = pv;
                }
            }
            s_wh[rr][cc] = wh;
            s_wv[rr][cc] = wv;
        }
        for (int e = threadIdx.x; e < (TH + 1) * (TW + 1); e += 256) {
            const int rr = e / (TW + 1), cc = e % (TW + 1);
            const int ii = i0 + rr, jj = j0 + cc;
            s_x[rr][cc] = (ii < g.nx && jj < g.ny) ? xt_at<T>(a, theta, xt, f, (long long)ii * g.ny + jj) : 0.f;
        }
        __syncthreads();
        // ---- theta on the tile, its right column and its bottom row ----
        for (int e = threadIdx.x; e < (TH + 1) * (TW + 1); e += 256) {
            const int rr = e / (TW + 1), cc = e % (TW + 1);
            float th = s_x[rr][cc];
            if (CLIP) {
                const float x0 = th;
                if (!a.first) {
                    th = __fmaf_rn(-a.lambda, s_wh[rr + 1][cc] - s_wh[rr + 1][cc + 1], x0);
                    s_tv[CLIP ? rr : 0][CLIP ? cc : 0] =
                        __fmaf_rn(-a.lambda, s_wv[rr][cc + 1] - s_wv[rr + 1][cc + 1], x0);
                } else {
                    s_tv[CLIP ? rr : 0][CLIP ? cc : 0] = x0;
                }
            } else if (!a.first) {
                th = __fmaf_rn(-a.lambda,
                               (s_wh[rr + 1][cc] - s_wh[rr + 1][cc + 1]) + (s_wv[rr][cc + 1] - s_wv[rr + 1][cc + 1]), th);
            }
            s_th[rr][cc] = th;
        }
        __syncthreads();
        // ---- a = w + step D theta at this thread's pixel ----
        const float t0 = s_th[ty][tx];
        const float ah = mh ? fmaf(s_th[ty][tx + 1] - t0, a.step, s_wh[ty + 1][tx + 1]) : 0.f;
        float av;
        if (CLIP) {
            const float v0 = s_tv[CLIP ? ty : 0][CLIP ? tx : 0];
            av = mv ? fmaf(s_tv[CLIP ? ty + 1 : 0][CLIP ? tx : 0] - v0, a.step, s_wv[ty + 1][tx + 1]) : 0.f;
        } else {
            av = mv ? fmaf(s_th[ty + 1][tx] - t0, a.step, s_wv[ty + 1][tx + 1]) : 0.f;
        }
        if (a.first && a.mode != OuterMode::Prox && in) st<T>(xt, (long long)f * g.n + mypix, s_x[ty][tx]);
        if (TV == SCI_TV_VTV) {
            ah_r[ff] = ah;
            av_r[ff] = av;
            if (ff & 1) n2o = fmaf(ah, ah, fmaf(av, av, n2o));
            else n2e = fmaf(ah, ah, fmaf(av, av, n2e));
        } else if (in) {
            float nh = ah, nv = av;
            if (TV == SCI_TV_ATV || CLIP) {
                nh = fminf(fmaxf(nh, -1.f), 1.f);
                nv = fminf(fmaxf(nv, -1.f), 1.f);
            } else {
                const float sc = fminf(1.f, rsqrtf(fmaf(nh, nh, nv * nv)));
                nh *= sc;
                nv *= sc;
            }
            const long long idx = (long long)f * g.n + mypix;
            st<T>(pout, idx, nh);
            st<T>(pout, N + idx, nv);
        }
        __syncthreads();  // the next frame reuses the shared tiles
    }
    if (TV == SCI_TV_VTV && in) {
        const float sc = fminf(1.f, rsqrtf(n2e + n2o));
#pragma unroll
        for (int ff = 0; ff < FMAX; ++ff) {
            if (ff >= nfr) break;
            const long long idx = (long long)ff * g.n + mypix;
            st<T>(pout, idx, ah_r[ff] * sc);
            st<T>(pout, N + idx, av_r[ff] * sc);
        }
    }
}

template <typename T, int TV, int FMAX>
void launch_t(const StreamArgs& a, const T* theta, T* xt, const T* p, const T* q, T* pout, cudaStream_t s) {
    const dim3 grid((unsigned)((a.g.ny + TW - 1) / TW), (unsigned)((a.g.nx + TH - 1) / TH),
                    (unsigned)(TV == SCI_TV_VTV ? 1 : a.g.B));
    k_fgp_stream<T, TV, FMAX><<<grid, 256, 0, s>>>(a, theta, xt, p, q, pout);
}

}  // namespace

// One dual update: first = 1 starts from w = 0 and forms x-tilde (Prox mode:
// from xin; Gap / Admm: theta + c_k r, written to xt); later updates read
// x-tilde from xt and w = p + coef (p - q) (q may be null).
template <typename T>
void launch_fgp_stream(int tv, OuterMode mode, int first, const float* xin, const T* theta, const float* r,
                       const uint32_t* bits, Geo g, float lambda, float coef, T* xt, const T* p, const T* q,
                       T* pout, cudaStream_t s) {
    StreamArgs a{};
    a.g = g;
    a.first = first;
    a.mode = mode;
    a.lambda = lambda;
    a.step = (float)(1.0 / ((tv == kTvClip ? kClipAlpha : 8.0) * (double)lambda));
    a.c = coef;
    a.xin = xin;
    a.bits = bits;
    a.r = r;
    switch (tv) {
        case SCI_TV_ATV: launch_t<T, SCI_TV_ATV, 1>(a, theta, xt, p, q, pout, s); break;
        case SCI_TV_ITV2D: launch_t<T, SCI_TV_ITV2D, 1>(a, theta, xt, p, q, pout, s); break;
        case kTvClip: launch_t<T, kTvClip, 1>(a, theta, xt, p, q, pout, s); break;
        default:
            if (g.B <= 16) launch_t<T, SCI_TV_VTV, 16>(a, theta, xt, p, q, pout, s);
            else launch_t<T, SCI_TV_VTV, 32>(a, theta, xt, p, q, pout, s);
            break;
    }
}

#define SCI_INST(T)                                                                                          \
    template void launch_fgp_stream<T>(int, OuterMode, int, const float*, const T*, const float*, const uint32_t*, \
                                       Geo, float, float, T*, const T*, const T*, T*, cudaStream_t);
SCI_INST(float)
SCI_INST(__nv_bfloat16)
SCI_INST(__half)
#undef SCI_INST

}  // namespace sci
