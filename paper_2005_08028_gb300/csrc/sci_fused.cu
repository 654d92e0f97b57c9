// Temporally blocked FGP: K dual updates per launch on a shared-memory tile
// with a halo (Algorithm 1, ATV-FGP box; Eqs. 29-32 for ITV2D / VTV).
//
// A CTA owns an "extended" tile of EH x EW pixels (its interior plus a halo
// of H pixels on every side) for F frames.  One dual update moves
// information by one pixel in each direction (theta needs w at the left/up
// neighbours, the gradient of theta needs the right/down ones), so after K
// updates the interior widened by H - K >= 1 pixels is exact; the extra pixel
// feeds D^T p in the output theta = xt - lambda D^T p.
//
// Thread mapping: thread t owns the pixels t, t + NT, ..., t + (Q-1) NT of
// the tile (one column, Q rows NT/EW apart) and all F frames of each.
// F = 1 for ATV / ITV2D, whose frames are independent (blockIdx.z picks the
// frame); F >= B for VTV, whose dual projection couples the B frames of a
// pixel -- its norm is then a register sum inside one thread.  A warp covers
// 32 consecutive columns of one row: global loads are coalesced and the row
// tests below are warp-uniform.
//
// State: p and w of the owned slots live in registers; x-tilde, theta and the
// neighbour-visible copy of w live in shared memory (16 bytes per slot).  Per
// update a slot costs 8 shared-memory accesses and ~20 FP32 operations; no
// global memory is touched between the updates of one launch.  Rows whose
// results can no longer reach the interior are skipped: the needed band
// shrinks by one row per update.
#include <atomic>

#include "sci_internal.cuh"

namespace sci {

namespace {

template <typename T>
__device__ __forceinline__ float rt(float v) {
    T tmp;
    st<T>(&tmp, 0, v);
    return ld<T>(&tmp, 0);
}

// Compile-time tile configuration.
template <int NT_, int Q_, int F_, int EW_LOG2_>
struct FusedCfg {
    static constexpr int NT = NT_;            // threads per CTA
    static constexpr int Q = Q_;              // pixels per thread
    static constexpr int F = F_;              // frames held per CTA
    static constexpr int EW_LOG2 = EW_LOG2_;
    static constexpr int EW = 1 << EW_LOG2;   // tile width (columns)
    static constexpr int P = NT * Q;          // pixels per tile
    static constexpr int EH = P / EW;         // tile height (rows)
    static constexpr int RS = NT / EW;        // row stride between a thread's pixels
    static constexpr size_t SMEM = (size_t)F * P * 4 * sizeof(float);  // xt, theta, wh, wv
    static_assert(NT % EW == 0, "a CTA must cover whole rows");
};

template <typename T, int TV, class Cfg>
__global__ void __launch_bounds__(Cfg::NT, 1)
k_fgp_fused(FusedArgs a, FusedBufs<T> b) {
    constexpr int NT = Cfg::NT, Q = Cfg::Q, F = Cfg::F, EW = Cfg::EW, EH = Cfg::EH, P = Cfg::P;
    constexpr int RS = Cfg::RS;
    extern __shared__ float smem[];
    float* s_xt = smem;              // [F][P]
    float* s_th = smem + F * P;      // [F][P]
    float* s_wh = smem + 2 * F * P;  // [F][P]
    float* s_wv = smem + 3 * F * P;  // [F][P]

    const Geo g = a.g;
    const int H = a.halo;
    const int TI = EH - 2 * H, TJ = EW - 2 * H;  // interior size
    const int gi0 = blockIdx.y * TI - H, gj0 = blockIdx.x * TJ - H;
    const int nfr = (F == 1) ? 1 : g.B;          // frames this CTA updates
    const int f0 = (F == 1) ? blockIdx.z : 0;    // global frame of slot f = 0
    const int tid = threadIdx.x;
    const int col = tid & (EW - 1);
    const int row0 = tid >> Cfg::EW_LOG2;
    const int gj = gj0 + col;
    const bool col_in = gj >= 0 && gj < g.ny;
    const bool hr = gj < g.ny - 1;
    const bool col_int = col >= H && col < EW - H;

    float ph[F][Q], pv[F][Q], wh[F][Q], wv[F][Q];

    // ---- load x-tilde (and carried duals) for the whole extended tile ----
#pragma unroll
    for (int f = 0; f < F; ++f) {
        if (f >= nfr) break;
        const long long fo = (long long)(f0 + f) * g.n;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int r = row0 + q * RS, gi = gi0 + r;
            const int o = f * P + r * EW + col;
            float x = 0.f, a_ph = 0.f, a_pv = 0.f, a_wh = 0.f, a_wv = 0.f;
            if (col_in && gi >= 0 && gi < g.nx) {
                const long long pix = (long long)gi * g.ny + gj;
                const long long gidx = fo + pix;
                if (a.mode == OuterMode::Prox) {
                    x = a.xin[gidx];
                } else if (a.first) {
                    x = rt<T>(ld<T>(b.theta_in, gidx) + mask_bit(a.bits[pix], f0 + f) * a.r[pix]);
                } else {
                    x = ld<T>(b.xt, gidx);
                }
                if (!a.first) {
                    a_ph = ld<T>(b.st_in[0], gidx);
                    a_pv = ld<T>(b.st_in[1], gidx);
                    a_wh = ld<T>(b.st_in[2], gidx);
                    a_wv = ld<T>(b.st_in[3], gidx);
                }
            }
            s_xt[o] = x;
            s_wh[o] = a_wh;
            s_wv[o] = a_wv;
            ph[f][q] = a_ph;
            pv[f][q] = a_pv;
            wh[f][q] = a_wh;
            wv[f][q] = a_wv;
        }
    }
    __syncthreads();

    const float lam = a.lambda, step = a.step;
    for (int s = 0; s < a.K; ++s) {
        const int m = H - 1 - s;                       // margin still exact after this update
        const int rlo_p = H - m, rhi_p = EH - H + m;   // rows whose p is updated
        const bool skip_theta = a.first && s == 0;     // w = 0 there: theta = xt
        // ---- theta = xt - lambda (D^T w) on rows [rlo_p, rhi_p] ----
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int r = row0 + q * RS;
            if (r < rlo_p || r > rhi_p) continue;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                const int o = f * P + r * EW + col;
                float th = s_xt[o];
                if (!skip_theta) {
                    const float wl = col > 0 ? s_wh[o - 1] : 0.f;
                    const float wu = r > 0 ? s_wv[o - EW] : 0.f;
                    th = th - lam * ((wl - wh[f][q]) + (wu - wv[f][q]));
                }
                s_th[o] = th;
            }
        }
        __syncthreads();
        // ---- a = w + step * D theta (kept in the w registers), projection, momentum ----
        const float c = a.coef[s];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int r = row0 + q * RS, gi = gi0 + r;
            if (r < rlo_p || r >= rhi_p) continue;
            const bool in = col_in && gi >= 0 && gi < g.nx;
            const bool hd = gi < g.nx - 1;
            float n2 = 0.f;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                const int o = f * P + r * EW + col;
                const float t0 = s_th[o];
                const float tr = col < EW - 1 ? s_th[o + 1] : t0;
                const float td = r < EH - 1 ? s_th[o + EW] : t0;
                const float ah = (in && hr) ? fmaf(tr - t0, step, wh[f][q]) : 0.f;
                const float av = (in && hd) ? fmaf(td - t0, step, wv[f][q]) : 0.f;
                wh[f][q] = ah;
                wv[f][q] = av;
                if (TV == SCI_TV_VTV) n2 += ah * ah + av * av;
            }
            const float vscale = (TV == SCI_TV_VTV) ? fminf(1.f, rsqrtf(n2)) : 1.f;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                float nh = wh[f][q], nv = wv[f][q];
                if (TV == SCI_TV_ATV) {
                    nh = fminf(fmaxf(nh, -1.f), 1.f);
                    nv = fminf(fmaxf(nv, -1.f), 1.f);
                } else if (TV == SCI_TV_ITV2D) {
                    // a / max(1, |a|) = a * min(1, 1/|a|); rsqrtf(0) = inf gives 1
                    const float sc = fminf(1.f, rsqrtf(fmaf(nh, nh, nv * nv)));
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
                const int o = f * P + r * EW + col;
                s_wh[o] = wnh;
                s_wv[o] = wnv;
            }
        }
        __syncthreads();
    }

    // ---- epilogue ----
    if (!a.last) {
        // carry x-tilde (first launch of a solve), p and w of the interior
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int r = row0 + q * RS, gi = gi0 + r;
            if (!col_int || r < H || r >= EH - H || !col_in || gi >= g.nx) continue;
            const long long pix = (long long)gi * g.ny + gj;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                const long long gidx = (long long)(f0 + f) * g.n + pix;
                if (a.first && a.mode != OuterMode::Prox) st<T>(b.xt, gidx, s_xt[f * P + r * EW + col]);
                st<T>(b.st_out[0], gidx, ph[f][q]);
                st<T>(b.st_out[1], gidx, pv[f][q]);
                st<T>(b.st_out[2], gidx, wh[f][q]);
                st<T>(b.st_out[3], gidx, wv[f][q]);
            }
        }
        return;
    }
    // theta = xt - lambda D^T p needs p at the left / up neighbours: stage p
    // in the w slots (the update loop ended with a barrier).
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int r = row0 + q * RS;
#pragma unroll
        for (int f = 0; f < F; ++f) {
            if (f >= nfr) break;
            const int o = f * P + r * EW + col;
            s_wh[o] = ph[f][q];
            s_wv[o] = pv[f][q];
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int r = row0 + q * RS, gi = gi0 + r;
        if (!col_int || r < H || r >= EH - H || !col_in || gi >= g.nx) continue;
        const long long pix = (long long)gi * g.ny + gj;
#pragma unroll
        for (int f = 0; f < F; ++f) {
            if (f >= nfr) break;
            const int o = f * P + r * EW + col;
            const float pl = col > 0 ? s_wh[o - 1] : 0.f;
            const float pu = r > 0 ? s_wv[o - EW] : 0.f;
            const float x0 = s_xt[o];
            const float th = x0 - lam * ((pl - ph[f][q]) + (pu - pv[f][q]));
            const long long gidx = (long long)(f0 + f) * g.n + pix;
            if (a.mode == OuterMode::Prox) {
                a.theta_f32[gidx] = th;
                continue;
            }
            st<T>(b.theta_out, gidx, th);
            if (a.mode == OuterMode::Gap) {
                if (a.x_out != nullptr) a.x_out[gidx] = x0;
            } else {
                const float u_old = ld<T>(b.u_in, gidx);
                st<T>(b.u_out, gidx, x0 - rt<T>(th));
                if (a.x_out != nullptr) a.x_out[gidx] = x0 - u_old;
            }
        }
    }
}

// ---------------------------------------------------------------- configurations

using CfgF1 = FusedCfg<512, 16, 1, 7>;   // 128 x 64 tile, one frame
using CfgF1s = FusedCfg<256, 8, 1, 6>;   // 64 x 32 tile, one frame (small images)
using CfgV8 = FusedCfg<512, 2, 8, 5>;    // 32 x 32 tile, up to 8 frames
using CfgV10 = FusedCfg<512, 2, 10, 5>;  // 32 x 32 tile, up to 10 frames
using CfgV16 = FusedCfg<256, 2, 16, 5>;  // 32 x 16 tile, up to 16 frames

std::atomic<unsigned long long> g_attr_done[48];

template <typename T, int TV, class Cfg>
bool launch_cfg(int slot, const FusedArgs& a, const FusedBufs<T>& b, cudaStream_t s) {
    const int TI = Cfg::EH - 2 * a.halo, TJ = Cfg::EW - 2 * a.halo;
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
    return (std::is_same<T, float>::value ? 0 : (std::is_same<T, __half>::value ? 1 : 2)) * 15 + tv * 5 + cfg;
}

template <typename T, int TV>
bool launch_tv(const FusedArgs& a, const FusedBufs<T>& b, cudaStream_t s) {
    if (TV != SCI_TV_VTV) {
        if (a.halo <= 8 && (long long)a.g.nx * a.g.ny < 192LL * 192)
            return launch_cfg<T, TV, CfgF1s>(type_slot<T>(TV, 1), a, b, s);
        return launch_cfg<T, TV, CfgF1>(type_slot<T>(TV, 0), a, b, s);
    }
    if (a.g.B <= 8) return launch_cfg<T, TV, CfgV8>(type_slot<T>(TV, 2), a, b, s);
    if (a.g.B <= 10) return launch_cfg<T, TV, CfgV10>(type_slot<T>(TV, 3), a, b, s);
    if (a.g.B <= 16) return launch_cfg<T, TV, CfgV16>(type_slot<T>(TV, 4), a, b, s);
    return false;
}

}  // namespace

int fused_max_halo(int tv, int B) {
    if (tv != SCI_TV_VTV) return 20;
    if (B <= 10) return 8;
    if (B <= 16) return 4;
    return 0;  // no fused kernel: the per-update kernels serve
}

template <typename T>
bool launch_fgp_fused(int tv, const FusedArgs& a, const FusedBufs<T>& b, cudaStream_t s) {
    switch (tv) {
        case SCI_TV_ATV: return launch_tv<T, SCI_TV_ATV>(a, b, s);
        case SCI_TV_ITV2D: return launch_tv<T, SCI_TV_ITV2D>(a, b, s);
        default: return launch_tv<T, SCI_TV_VTV>(a, b, s);
    }
}

template bool launch_fgp_fused<float>(int, const FusedArgs&, const FusedBufs<float>&, cudaStream_t);
template bool launch_fgp_fused<__nv_bfloat16>(int, const FusedArgs&, const FusedBufs<__nv_bfloat16>&,
                                              cudaStream_t);
template bool launch_fgp_fused<__half>(int, const FusedArgs&, const FusedBufs<__half>&, cudaStream_t);

}  // namespace sci
