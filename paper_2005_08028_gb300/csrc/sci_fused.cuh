// Temporally blocked FGP: K dual updates per launch on a shared-memory tile
// with a halo (Algorithm 1, ATV-FGP box; Eqs. 29-32 for ITV2D / VTV).
//
// A CTA owns an "extended" tile of EH x EW pixels (its interior plus a halo)
// for F frames.  One dual update moves information by one pixel in each
// direction (theta needs w at the left/up neighbours, the gradient of theta
// needs the right/down ones), so after K updates p is exact K pixels in from
// every tile edge.  The output theta = xt - lambda D^T p also reads p at the
// left/up neighbour, so the halo is H = K + 1 pixels on the top and left
// sides and H - 1 = K on the bottom and right (fused_interior).
//
// Thread mapping: the tile is cut into NS = NT/EW horizontal strips of Q
// rows; thread t owns column t % EW of strip t / EW -- Q vertically adjacent
// pixels -- and all F frames of each.  F = 1 for ATV / ITV2D, whose frames
// are independent (blockIdx.z picks the frame); F >= B for VTV, whose dual
// projection couples the B frames of a pixel -- the norm is then a register
// sum inside one thread.  A warp covers 32 consecutive columns of one strip,
// so global accesses are coalesced and the row tests below are warp-uniform.
//
// State: p, w (and, when registers allow, x-tilde and theta) of the owned
// slots live in registers.  Vertical neighbours inside a strip are register
// reads; shared memory carries only what other threads read: theta and w_h
// of every slot (left/right neighbours) and w_v of each strip's last row.
// No global memory is touched between the updates of one launch.  Where it
// pays (see the configurations), rows whose results can no longer reach the
// interior are skipped: the band that matters shrinks by one row per update.
//
// This header holds the implementation; sci_fused_f32.cu, sci_fused_f16.cu and
// sci_fused_bf16.cu each instantiate it for one storage type (SCI_FUSED_STORAGE),
// so the three compile in parallel.  The f32 unit also defines the tile-class
// queries (SCI_FUSED_COMMON).
#pragma once

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "sci_internal.cuh"

namespace sci {

namespace {

template <typename T>
__device__ __forceinline__ float rt(float v) {
    T tmp;
    st<T>(&tmp, 0, v);
    return ld<T>(&tmp, 0);
}

// 1/sqrt(x) by the hardware approximation (relative error below 2^-22),
// flushing subnormal inputs to zero: only min(1, 1/|a|) is formed from it,
// which is 1 for every |a| <= 1 either way.
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <typename T> __device__ __forceinline__ float ldg(const T* p, long long i);
template <> __device__ __forceinline__ float ldg<float>(const float* p, long long i) { return __ldg(p + i); }
// 16-bit fields are read as raw unsigned shorts through the compiler's own
// read-only load, which the scheduler can batch like any other load (the
// __half / __nv_bfloat16 overloads of __ldg are inline assembly, and their
// loads were waited on one at a time).
template <> __device__ __forceinline__ float ldg<__nv_bfloat16>(const __nv_bfloat16* p, long long i) {
    return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short*>(p) + i)));
}
template <> __device__ __forceinline__ float ldg<__half>(const __half* p, long long i) {
    return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p) + i)));
}


// Compile-time tile configuration.
template <int NT_, int Q_, int F_, int EW_LOG2_, bool REG_, bool SKIP_>
struct FusedCfg {
    static constexpr int NT = NT_;            // threads per CTA
    static constexpr int Q = Q_;              // rows per strip (pixels per thread)
    static constexpr int F = F_;              // frames held per CTA
    static constexpr int EW_LOG2 = EW_LOG2_;
    static constexpr int EW = 1 << EW_LOG2;   // tile width (columns)
    static constexpr int NS = NT / EW;        // strips
    static constexpr int EH = NS * Q;         // tile height (rows)
    static constexpr bool REG = REG_;         // x-tilde and theta of owned slots in registers
    static constexpr bool SKIP = SKIP_;       // skip rows that can no longer reach the interior
    // Slot arrays (theta, w_h, and x-tilde unless REG) store each frame as one
    // leading pad word followed by EH rows of EW slots and a trailing pad word:
    // slot (r, c) sits at 1 + r * LD + c, so its left neighbour at c = 0 and its
    // right neighbour at c = EW - 1 are pad words, which hold zero.
    static constexpr int LD = EW + 1;
    static constexpr int FPP = EH * LD + 1;
    // shared memory: slot arrays [F][FPP]; w_v [F][NS][EW]
    static constexpr size_t SMEM = ((size_t)F * FPP * (REG ? 2 : 3) + (size_t)F * NS * EW) * sizeof(float);
    static_assert(NT % EW == 0, "a CTA must cover whole rows");
    static_assert(EW % 32 == 0, "a warp must stay inside one strip row");
};

// Problem views for fused_tile: a single problem read from the kernel's
// parameter space, or one entry of a device-resident batch table.
template <typename T>
struct SingleProb {
    const FusedArgs* a;
    const FusedBufs<T>* b;
    __device__ Geo g() const { return a->g; }
    __device__ const uint32_t* bits() const { return a->bits; }
    __device__ const float* r() const { return a->r; }
    __device__ float* x_out() const { return a->x_out; }
    __device__ const float* xin() const { return a->xin; }
    __device__ float* theta_f32() const { return a->theta_f32; }
    __device__ const T* theta_in() const { return b->theta_in; }
    __device__ T* theta_out() const { return b->theta_out; }
    __device__ const T* u_in() const { return b->u_in; }
    __device__ T* u_out() const { return b->u_out; }
    __device__ T* xt() const { return b->xt; }
    __device__ const T* st_in(int i) const { return b->st_in[i]; }
    __device__ T* st_out(int i) const { return b->st_out[i]; }
};
template <typename T>
struct BatchProb {
    const BatchItem<T>* it;
    int tpar, spar, want_x;
    __device__ Geo g() const { return it->g; }
    __device__ const uint32_t* bits() const { return it->bits; }
    __device__ const float* r() const { return it->r; }
    __device__ float* x_out() const { return want_x ? it->x_out : nullptr; }
    __device__ const float* xin() const { return nullptr; }
    __device__ float* theta_f32() const { return nullptr; }
    __device__ const T* theta_in() const { return it->theta[tpar]; }
    __device__ T* theta_out() const { return it->theta[tpar ^ 1]; }
    __device__ const T* u_in() const { return nullptr; }
    __device__ T* u_out() const { return nullptr; }
    __device__ T* xt() const { return it->xt; }
    __device__ const T* st_in(int i) const { return it->st[spar][i]; }
    __device__ T* st_out(int i) const { return it->st[spar ^ 1][i]; }
};

// One tile (bx, by) of frame bz (one-frame tiles) of one problem.  `a`
// carries the launch-wide settings (K, halo, first/last, lambda, momentum),
// `p` the problem's geometry and buffers.
template <typename T, int TV, class Cfg, class Prob>
__device__ __forceinline__ void fused_tile(const FusedArgs& a, const Prob& p, int bx, int by, int bz,
                                           float* smem) {
    constexpr int Q = Cfg::Q, F = Cfg::F, EW = Cfg::EW, EH = Cfg::EH, NS = Cfg::NS;
    constexpr bool REG = Cfg::REG, SKIP = Cfg::SKIP;
    constexpr int LD = Cfg::LD, FP = Cfg::FPP;  // row stride, frame stride (padded)
    float* s_th = smem;                      // [F][FPP]
    float* s_wh = s_th + F * FP;             // [F][FPP]
    float* s_wv = s_wh + F * FP;             // [F][NS][EW]: last row of each strip
    float* s_xt = s_wv + F * NS * EW;        // [F][FPP] (only when !REG)

    const Geo g = p.g();
    const int H = a.halo;
    const int TI = fused_interior(EH, H), TJ = fused_interior(EW, H);  // interior size
    const int gi0 = by * TI - H, gj0 = bx * TJ - H;
    const int nfr = (F == 1) ? 1 : g.B;          // frames this CTA updates
    const int f0 = (F == 1) ? bz : 0;            // global frame of slot f = 0
    const int tid = threadIdx.x;
    const int col = tid & (EW - 1);
    const int strip = tid >> Cfg::EW_LOG2;
    const int r0 = strip * Q;                    // first row of the strip
    const int gj = gj0 + col;
    const bool col_in = gj >= 0 && gj < g.ny;
    const bool col_int = col >= H && col < EW - H + 1;
    const int gi_top = gi0 + r0;

    // per-row flags as bit masks (bit q: row r0 + q)
    unsigned in_m = 0, ah_m = 0, av_m = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int gi = gi_top + q;
        const bool in = col_in && gi >= 0 && gi < g.nx;
        in_m |= (unsigned)in << q;
        ah_m |= (unsigned)(in && gj < g.ny - 1) << q;
        av_m |= (unsigned)(in && gi < g.nx - 1) << q;
    }
    // Strips whose rows all lie inside the image and above its last row need
    // no row masks (warp-uniform): the column conditions fold into per-thread
    // steps, zero where the gradient component is defined as zero.  w stays
    // zero there (it starts at zero and a = w + 0 * (difference) projects to
    // zero), so the masked and unmasked forms agree.
    const bool rows_inner = gi_top >= 0 && gi_top + Q - 1 < g.nx - 1;
    const float step_h = (col_in && gj < g.ny - 1) ? a.step : 0.f;
    const float step_v = col_in ? a.step : 0.f;

    float ph[F][Q], pv[F][Q], wh[F][Q], wv[F][Q];
    float xr[REG ? F : 1][REG ? Q : 1], thr[REG ? F : 1][REG ? Q : 1];

    // ---- load x-tilde (and the carried duals) for the whole extended tile ----
    // Every load is issued unconditionally -- a pixel outside the image reads
    // pixel 0 of its frame and is zeroed afterwards -- and none is consumed
    // before all are issued, so a thread's loads are in flight together
    // rather than one row at a time.
    const long long pix_top = (long long)gi_top * g.ny + gj;
    auto pix_of = [&](int q) -> long long { return ((in_m >> q) & 1u) ? pix_top + (long long)q * g.ny : 0; };
    if (!a.first) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long pix = pix_of(q);
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                const long long gidx = (long long)(f0 + f) * g.n + pix;
                ph[f][q] = ldraw<T>(p.st_in(0), gidx);
                pv[f][q] = ldraw<T>(p.st_in(1), gidx);
                wh[f][q] = ldraw<T>(p.st_in(2), gidx);
                wv[f][q] = ldraw<T>(p.st_in(3), gidx);
            }
        }
    }
    // x-tilde as loaded: straight into the x-tilde registers of REG tiles,
    // into staging registers otherwise
    float xs[REG ? 1 : F][REG ? 1 : Q];
    auto xq = [&](int f, int q) -> float& { return REG ? xr[REG ? f : 0][REG ? q : 0] : xs[REG ? 0 : f][REG ? 0 : q]; };
    if (a.mode == OuterMode::Prox) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long pix = pix_of(q);
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                xq(f, q) = __ldg(p.xin() + (long long)(f0 + f) * g.n + pix);
            }
        }
    } else if (a.first) {
        uint32_t word[Q];
        float rv[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long pix = pix_of(q);
            word[q] = __ldg(p.bits() + pix);
            rv[q] = __ldg(p.r() + pix);
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                xq(f, q) = ldraw<T>(p.theta_in(), (long long)(f0 + f) * g.n + pix);
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                xq(f, q) = rt<T>(cvraw<T>(xq(f, q)) + mask_bit(word[q], f0 + f) * rv[q]);
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long pix = pix_of(q);
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                xq(f, q) = ldraw<T>(p.xt(), (long long)(f0 + f) * g.n + pix);
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                xq(f, q) = cvraw<T>(xq(f, q));
            }
        }
    }
    if (!a.first) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                ph[f][q] = cvraw<T>(ph[f][q]);
                pv[f][q] = cvraw<T>(pv[f][q]);
                wh[f][q] = cvraw<T>(wh[f][q]);
                wv[f][q] = cvraw<T>(wv[f][q]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const bool in = (in_m >> q) & 1u;
#pragma unroll
        for (int f = 0; f < F; ++f) {
            if (f >= nfr) break;
            const float x = in ? xq(f, q) : 0.f;
            if (a.first || !in) {
                ph[f][q] = 0.f;
                pv[f][q] = 0.f;
                wh[f][q] = 0.f;
                wv[f][q] = 0.f;
            }
            const int o = f * FP + 1 + (r0 + q) * LD + col;
            if (REG) xr[REG ? f : 0][REG ? q : 0] = x;
            else s_xt[o] = x;
            s_wh[o] = wh[f][q];
            if (q == Q - 1) s_wv[(f * NS + strip) * EW + col] = wv[f][q];
        }
    }
    for (int e = tid; e < F * (EH + 1); e += Cfg::NT) {  // pad words
        const int f = e / (EH + 1), k = e - f * (EH + 1);
        s_th[f * FP + k * LD] = 0.f;
        s_wh[f * FP + k * LD] = 0.f;
    }
    __syncthreads();

    const float lam = a.lambda, step = a.step;
    // Two updates per loop trip let the compiler alternate registers instead
    // of copying the loop-carried duals (measured: VTV tiles of up to 10
    // frames -6%, ITV2D -3%).  The one-frame ATV tile gains nothing, and the
    // 16- and 24-frame VTV tiles, already near the register limit, lose.
    constexpr int kUnroll = ((TV == SCI_TV_ATV && F == 1) || F > 10) ? 1 : 2;
#pragma unroll kUnroll
    for (int s = 0; s < a.K; ++s) {
        // rows whose p stays exact after this update: [1 + s, EH - 1 - s);
        // theta is needed on those rows and the one below
        const int rlo = 1 + s, rhi = EH - 1 - s;
        const int qlo = SKIP ? max(rlo - r0, 0) : 0;
        const int qhi_p = SKIP ? min(rhi - r0, Q) : Q, qhi_t = SKIP ? min(rhi + 1 - r0, Q) : Q;
        const bool skip_theta = a.first && s == 0;  // w = 0 there: theta = xt
        // ---- theta = xt - lambda (D^T w) ----
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (q < qlo || q >= qhi_t) continue;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                const int o = f * FP + 1 + (r0 + q) * LD + col;
                float th = REG ? xr[REG ? f : 0][REG ? q : 0] : s_xt[o];
                if (!skip_theta) {
                    const float wl = s_wh[o - 1];
                    float wu;
                    if (q > 0) wu = wv[f][q > 0 ? q - 1 : 0];
                    else wu = strip > 0 ? s_wv[(f * NS + strip - 1) * EW + col] : 0.f;
                    th = th - lam * ((wl - wh[f][q]) + (wu - wv[f][q]));
                }
                if (REG) thr[REG ? f : 0][REG ? q : 0] = th;
                s_th[o] = th;
            }
        }
        __syncthreads();
        // ---- a = w + step * D theta (kept in the w registers), projection, momentum ----
        const float c = a.coef[s];
        auto dual_step = [&](auto masked_c) {
            constexpr bool MASKED = decltype(masked_c)::value;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                if (q < qlo || q >= qhi_p) continue;
                const bool mh = (ah_m >> q) & 1u, mv = (av_m >> q) & 1u;
                float n2 = 0.f;
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    if (f >= nfr) break;
                    const int o = f * FP + 1 + (r0 + q) * LD + col;
                    const float t0 = REG ? thr[REG ? f : 0][REG ? q : 0] : s_th[o];
                    const float tr = s_th[o + 1];
                    float td;
                    if (q < Q - 1) td = REG ? thr[REG ? f : 0][REG && q < Q - 1 ? q + 1 : 0] : s_th[o + LD];
                    else td = (r0 + q < EH - 1) ? s_th[o + LD] : t0;
                    float ah, av;
                    if (MASKED) {
                        ah = mh ? fmaf(tr - t0, step, wh[f][q]) : 0.f;
                        av = mv ? fmaf(td - t0, step, wv[f][q]) : 0.f;
                    } else {
                        ah = fmaf(tr - t0, step_h, wh[f][q]);
                        av = fmaf(td - t0, step_v, wv[f][q]);
                    }
                    wh[f][q] = ah;
                    wv[f][q] = av;
                    if (TV == SCI_TV_VTV) n2 = fmaf(ah, ah, fmaf(av, av, n2));
                }
                const float vscale = (TV == SCI_TV_VTV) ? fminf(1.f, rsqrt_ftz(n2)) : 1.f;
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    if (f >= nfr) break;
                    float nh = wh[f][q], nv = wv[f][q];
                    if (TV == SCI_TV_ATV) {
                        nh = fminf(fmaxf(nh, -1.f), 1.f);
                        nv = fminf(fmaxf(nv, -1.f), 1.f);
                    } else if (TV == SCI_TV_ITV2D) {
                        // a / max(1, |a|) = a * min(1, 1/|a|); 1/sqrt(0) = inf gives 1
                        const float sc = fminf(1.f, rsqrt_ftz(fmaf(nh, nh, nv * nv)));
                        nh *= sc;
                        nv *= sc;
                    } else {
                        nh *= vscale;
                        nv *= vscale;
                    }
                    const float wnh = fmaf(c, nh - ph[f][q], nh);
                    const float wnv = fmaf(c, nv - pv[f][q], nv);
                    ph[f][q] = nh;
                    pv[f][q] = nv;
                    wh[f][q] = wnh;
                    wv[f][q] = wnv;
                    s_wh[f * FP + 1 + (r0 + q) * LD + col] = wnh;
                    if (q == Q - 1) s_wv[(f * NS + strip) * EW + col] = wnv;
                }
            }
        };
        if (rows_inner) dual_step(std::false_type{});
        else dual_step(std::true_type{});
        __syncthreads();
    }

    // ---- epilogue ----
    if (!a.last) {
        // carry x-tilde (first launch of a solve), p and w of the interior
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int r = r0 + q;
            if (!((in_m >> q) & 1u) || !col_int || r < H || r >= EH - H + 1) continue;
            const long long pix = (long long)(gi_top + q) * g.ny + gj;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                const long long gidx = (long long)(f0 + f) * g.n + pix;
                if (a.first && a.mode != OuterMode::Prox)
                    st<T>(p.xt(), gidx, REG ? xr[REG ? f : 0][REG ? q : 0] : s_xt[f * FP + 1 + r * LD + col]);
                st<T>(p.st_out(0), gidx, ph[f][q]);
                st<T>(p.st_out(1), gidx, pv[f][q]);
                st<T>(p.st_out(2), gidx, wh[f][q]);
                st<T>(p.st_out(3), gidx, wv[f][q]);
            }
        }
        return;
    }
    // theta = xt - lambda D^T p needs p_h of the left neighbour and p_v of the
    // row above: stage them where w_h / w_v were (the loop ended with a barrier).
#pragma unroll
    for (int q = 0; q < Q; ++q) {
#pragma unroll
        for (int f = 0; f < F; ++f) {
            if (f >= nfr) break;
            s_wh[f * FP + 1 + (r0 + q) * LD + col] = ph[f][q];
            if (q == Q - 1) s_wv[(f * NS + strip) * EW + col] = pv[f][q];
        }
    }
    // x^(t+1) = xt - u^(t) for ADMM (only when x is requested): u^(t) is read
    // before u^(t+1) overwrites it.  Issue every load first (into the thread's
    // own theta slots, free now) so none waits behind a store it might alias.
    if (a.mode == OuterMode::Admm && p.x_out() != nullptr) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int r = r0 + q;
            const bool mine = ((in_m >> q) & 1u) && col_int && r >= H && r < EH - H + 1;
            const long long pix = mine ? (long long)(gi_top + q) * g.ny + gj : 0;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                s_th[f * FP + 1 + r * LD + col] = mine ? ldg<T>(p.u_in(), (long long)(f0 + f) * g.n + pix) : 0.f;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int r = r0 + q;
        if (!((in_m >> q) & 1u) || !col_int || r < H || r >= EH - H + 1) continue;
        const long long pix = (long long)(gi_top + q) * g.ny + gj;
#pragma unroll
        for (int f = 0; f < F; ++f) {
            if (f >= nfr) break;
            const int o = f * FP + 1 + r * LD + col;
            const float pl = s_wh[o - 1];
            float pu;
            if (q > 0) pu = pv[f][q > 0 ? q - 1 : 0];
            else pu = strip > 0 ? s_wv[(f * NS + strip - 1) * EW + col] : 0.f;
            const float x0 = REG ? xr[REG ? f : 0][REG ? q : 0] : s_xt[o];
            const float th = x0 - lam * ((pl - ph[f][q]) + (pu - pv[f][q]));
            const long long gidx = (long long)(f0 + f) * g.n + pix;
            if (a.mode == OuterMode::Prox) {
                p.theta_f32()[gidx] = th;
                continue;
            }
            st<T>(p.theta_out(), gidx, th);
            if (a.mode == OuterMode::Gap) {
                if (p.x_out() != nullptr) p.x_out()[gidx] = x0;
            } else {
                st<T>(p.u_out(), gidx, x0 - rt<T>(th));
                if (p.x_out() != nullptr) p.x_out()[gidx] = x0 - s_th[o];
            }
        }
    }
}

// ---------------------------------------------------------------- configurations

// One-frame tiles (16-row strips) update every row: skipping rows would idle
// whole strips and stall the others at the barriers.  The VTV tiles have
// 1- or 2-row strips, where skipping balances well and saves work.
using CfgF1 = FusedCfg<512, 16, 1, 7, true, false>;    // 128 x 64 tile, one frame
using CfgF1s = FusedCfg<256, 8, 1, 6, true, false>;    // 64 x 32 tile, one frame (small images)
using CfgV8 = FusedCfg<512, 2, 8, 5, false, true>;     // 32 x 32 tile, up to 8 frames
using CfgV10 = FusedCfg<512, 2, 10, 5, false, true>;   // 32 x 32 tile, up to 10 frames
using CfgV16 = FusedCfg<256, 2, 16, 5, false, true>;   // 32 x 16 tile, up to 16 frames
using CfgV24 = FusedCfg<256, 2, 24, 5, false, true>;   // 32 x 16 tile, up to 24 frames

template <typename T, int TV, class Cfg>
__global__ void __launch_bounds__(Cfg::NT, 1)
k_fgp_fused(const __grid_constant__ FusedArgs a, const __grid_constant__ FusedBufs<T> b) {
    extern __shared__ float smem[];
    const SingleProb<T> p{&a, &b};
    fused_tile<T, TV, Cfg>(a, p, blockIdx.x, blockIdx.y, blockIdx.z, smem);
}

// Many problems of one tile class in one launch: work item w is a tile of
// the problem whose [cta_begin, next cta_begin) range holds w.  A persistent
// grid walks the work items (largest problems first), or each CTA takes one
// work item (PERSIST = false), where the loop's own live values would push the
// tile code into spilling.
// Each class has its own kernel: one kernel holding every class's tile code
// needs more registers than an SM has and spills.
template <typename T, int TV, class Cfg, bool PERSIST>
__global__ void __launch_bounds__(Cfg::NT, 1)
k_fgp_fused_batched(const __grid_constant__ FusedArgs a, const BatchItem<T>* __restrict__ items, int nitems,
                    int total, int tpar, int spar, int want_x) {
    extern __shared__ float smem[];
    __shared__ int s_item;
    for (int w = blockIdx.x; w < total; w += (PERSIST ? gridDim.x : total)) {
        // The problem whose work-item range holds w: every thread tests a few
        // entries (one round of loads, where a binary search takes log2(nitems)
        // dependent ones before the tile's own loads can start).
        for (int i = threadIdx.x; i < nitems; i += Cfg::NT) {
            const int b = items[i].cta_begin;
            const int e = i + 1 < nitems ? items[i + 1].cta_begin : total;
            if (b <= w && w < e) s_item = i;
        }
        __syncthreads();
        const BatchItem<T>* it = items + s_item;
        const int local = w - it->cta_begin;
        const int tiles_x = it->tiles_x, per_frame = tiles_x * it->tiles_y;
        const int bz = local / per_frame, rem = local - bz * per_frame;
        const int by = rem / tiles_x, bx = rem - by * tiles_x;
        const BatchProb<T> p{it, tpar, spar, want_x};
        fused_tile<T, TV, Cfg>(a, p, bx, by, bz, smem);
        if (!PERSIST) break;
        __syncthreads();  // shared memory is reused by the next work item
    }
}

std::atomic<unsigned long long> g_attr_done[64];

template <typename T, int TV, class Cfg>
bool launch_cfg(int slot, const FusedArgs& a, const FusedBufs<T>& b, cudaStream_t s) {
    const int TI = fused_interior(Cfg::EH, a.halo), TJ = fused_interior(Cfg::EW, a.halo);
    if (TI < 1 || TJ < 1 || a.halo < a.K + 1 || a.K < 1 || a.K > kMaxFuse) return false;
    const dim3 grid((unsigned)((a.g.ny + TJ - 1) / TJ), (unsigned)((a.g.nx + TI - 1) / TI),
                    (unsigned)(Cfg::F == 1 ? a.g.B : 1));
    if (grid.y > 65535u || grid.z > 65535u) return false;
    auto kern = k_fgp_fused<T, TV, Cfg>;
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(g_attr_done[slot].load() & bit)) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM) !=
            cudaSuccess)
            return false;
        g_attr_done[slot].fetch_or(bit);
    }
    kern<<<grid, Cfg::NT, Cfg::SMEM, s>>>(a, b);
    return true;
}

// One "attribute set" flag word per (storage type, TV, configuration).
template <typename T>
constexpr int type_slot(int tv, int cfg) {
    return (std::is_same<T, float>::value ? 0 : (std::is_same<T, __half>::value ? 1 : 2)) * 21 + tv * 7 + cfg;
}

template <typename T, int TV>
bool launch_tv(const FusedArgs& a, const FusedBufs<T>& b, cudaStream_t s) {
    // if constexpr: each TV form instantiates only the tiles it can launch
    if constexpr (TV != SCI_TV_VTV) {
        if (a.halo <= 8 && (long long)a.g.nx * a.g.ny < 192LL * 192)
            return launch_cfg<T, TV, CfgF1s>(type_slot<T>(TV, 1), a, b, s);
        return launch_cfg<T, TV, CfgF1>(type_slot<T>(TV, 0), a, b, s);
    } else {
        if (a.g.B <= 8) return launch_cfg<T, TV, CfgV8>(type_slot<T>(TV, 2), a, b, s);
        if (a.g.B <= 10) return launch_cfg<T, TV, CfgV10>(type_slot<T>(TV, 3), a, b, s);
        if (a.g.B <= 16) return launch_cfg<T, TV, CfgV16>(type_slot<T>(TV, 4), a, b, s);
        if (a.g.B <= 24) return launch_cfg<T, TV, CfgV24>(type_slot<T>(TV, 5), a, b, s);
        return false;
    }
}

template <class Cfg>
void dims_of(int& EH, int& EW) {
    EH = Cfg::EH;
    EW = Cfg::EW;
}

}  // namespace

#ifdef SCI_FUSED_COMMON
int fused_max_halo(int tv, int B) {
    if (tv != SCI_TV_VTV) return 20;
    if (B <= 10) return 8;
    if (B <= 24) return 4;
    return 0;  // no fused kernel: the per-update kernels serve
}

int fused_class(int tv, int B) {
    if (tv != SCI_TV_VTV) return 1;
    if (B <= 8) return 8;
    if (B <= 10) return 10;
    if (B <= 16) return 16;
    if (B <= 24) return 24;
    return 0;
}

void fused_class_dims(int cls, int* EH, int* EW) {
    int h = 0, w = 0;
    switch (cls) {
        case 1: dims_of<CfgF1>(h, w); break;
        case 8: dims_of<CfgV8>(h, w); break;
        case 10: dims_of<CfgV10>(h, w); break;
        case 16: dims_of<CfgV16>(h, w); break;
        default: dims_of<CfgV24>(h, w); break;
    }
    *EH = h;
    *EW = w;
}
#endif  // SCI_FUSED_COMMON

namespace {
std::atomic<unsigned long long> g_battr_done[64];

// VTV tiles run one work item per CTA: with the persistent loop their
// kernels spill (the 24-frame tile by about 0.8 KB a thread); one-frame tiles
// spill less with it.
template <class Cfg>
constexpr bool batched_persist() {
    return Cfg::F == 1;
}

template <typename T, int TV, class Cfg>
bool launch_batched_cfg(int slot, const FusedArgs& a, const BatchItem<T>* items, int nitems, int total,
                        int tpar, int spar, int want_x, cudaStream_t s) {
    constexpr bool persist = batched_persist<Cfg>();
    auto k = k_fgp_fused_batched<T, TV, Cfg, persist>;
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(g_battr_done[slot].load() & bit)) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM) != cudaSuccess)
            return false;
        g_battr_done[slot].fetch_or(bit);
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = persist ? std::max(1, std::min(sms, total)) : std::max(1, total);
    k<<<grid, Cfg::NT, Cfg::SMEM, s>>>(a, items, nitems, total, tpar, spar, want_x);
    return true;
}

template <typename T, int TV>
bool launch_batched_tv(int cls, const FusedArgs& a, const BatchItem<T>* items, int nitems, int total, int tpar,
                       int spar, int want_x, cudaStream_t s) {
    if constexpr (TV != SCI_TV_VTV) {
        return launch_batched_cfg<T, TV, CfgF1>(type_slot<T>(TV, 0), a, items, nitems, total, tpar, spar, want_x,
                                                s);
    } else {
        switch (cls) {
            case 8: return launch_batched_cfg<T, TV, CfgV8>(type_slot<T>(TV, 2), a, items, nitems, total, tpar, spar,
                                                            want_x, s);
            case 10: return launch_batched_cfg<T, TV, CfgV10>(type_slot<T>(TV, 3), a, items, nitems, total, tpar,
                                                              spar, want_x, s);
            case 16: return launch_batched_cfg<T, TV, CfgV16>(type_slot<T>(TV, 4), a, items, nitems, total, tpar,
                                                              spar, want_x, s);
            case 24: return launch_batched_cfg<T, TV, CfgV24>(type_slot<T>(TV, 5), a, items, nitems, total, tpar,
                                                              spar, want_x, s);
            default: return false;
        }
    }
}
}  // namespace

template <typename T>
bool launch_fgp_fused_batched(int tv, int cls, const FusedArgs& a, const BatchItem<T>* items, int nitems,
                              int total, int tpar, int spar, int want_x, cudaStream_t s) {
    switch (tv) {
        case SCI_TV_ATV: return launch_batched_tv<T, SCI_TV_ATV>(cls, a, items, nitems, total, tpar, spar, want_x, s);
        case SCI_TV_ITV2D:
            return launch_batched_tv<T, SCI_TV_ITV2D>(cls, a, items, nitems, total, tpar, spar, want_x, s);
        default: return launch_batched_tv<T, SCI_TV_VTV>(cls, a, items, nitems, total, tpar, spar, want_x, s);
    }
}

template <typename T>
bool launch_fgp_fused(int tv, const FusedArgs& a, const FusedBufs<T>& b, cudaStream_t s) {
    switch (tv) {
        case SCI_TV_ATV: return launch_tv<T, SCI_TV_ATV>(a, b, s);
        case SCI_TV_ITV2D: return launch_tv<T, SCI_TV_ITV2D>(a, b, s);
        default: return launch_tv<T, SCI_TV_VTV>(a, b, s);
    }
}

// The including translation unit names the storage type to instantiate.
template bool launch_fgp_fused_batched<SCI_FUSED_STORAGE>(int, int, const FusedArgs&,
                                                          const BatchItem<SCI_FUSED_STORAGE>*, int, int, int, int,
                                                          int, cudaStream_t);
template bool launch_fgp_fused<SCI_FUSED_STORAGE>(int, const FusedArgs&, const FusedBufs<SCI_FUSED_STORAGE>&,
                                                  cudaStream_t);

}  // namespace sci
