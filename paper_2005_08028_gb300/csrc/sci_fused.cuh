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
// reads; horizontal neighbours are adjacent lanes of a warp and cross by
// shuffles; shared memory carries what crosses between strips (theta of a
// strip's first row, w_v of its last row).  No global memory is touched
// between the updates of one launch.  Where it pays (see the
// configurations), rows whose results can no longer reach the interior are
// skipped: the band that matters shrinks by one row per update.
//
// Four implementations: one-frame tiles on column strips (fused_tile_rows)
// or on 4 x 4 pixel blocks (fused_tile_micro; ATV, ITV2D and the Clip box)
// use scalar FP32 arithmetic; VTV tiles run pairs of frames through the
// packed FP32 instructions, with horizontal neighbours by warp shuffles
// (fused_tile_impl) or, for the 24-frame tile, through 128-bit shared blocks
// of every slot (fused_tile_blk).
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


// Packed FP32 arithmetic (sm_100 and later): one instruction applies the
// operation to both lanes of a float2 with the rounding of the scalar
// operation, so a packed update gives the same bits as the scalar one while
// issuing half the arithmetic instructions.  a - b is formed as
// fma(b, -1, a), which rounds once like a subtraction.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }
// A frame pair of the left / right lane.  The first / last lane gets its own
// value back: the tile's edge columns lie in its halo, and with a halo of
// K + 1 (left) and K (right) no value read there reaches the interior within
// K updates, so any finite stand-in for the missing neighbour serves.
__device__ __forceinline__ float2 shfl_up2(float2 v) {
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ float2 shfl_down2(float2 v) {
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}
// 128-bit shared-memory words of the block-layout VTV tiles (BlkCfg).
__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void sts4(float* p, float2 a, float2 b) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// Words of a per-thread shared-memory block holding n floats: n rounded up to
// a multiple of 4 whose quotient by 4 is odd.  Consecutive columns' blocks then
// start 16-byte aligned, and the 8 lanes of each phase of a 128-bit access
// fall on 8 different 16-byte bank groups.
__host__ __device__ constexpr int block_words(int n) {
    return ((n + 3) / 4) % 2 == 1 ? ((n + 3) / 4) * 4 : ((n + 3) / 4) * 4 + 4;
}


// Compile-time tile configuration.
template <int NT_, int Q_, int F_, int EW_LOG2_, bool REG_, bool SKIP_>
struct FusedCfg {
    static constexpr bool MICRO = false;
    static constexpr bool SHFL = true;        // fused_tile_impl (shuffles); BlkCfg: fused_tile_blk
    static constexpr int NT = NT_;            // threads per CTA
    static constexpr int Q = Q_;              // rows per strip (pixels per thread)
    static constexpr int F = F_;              // frames held per CTA
    static constexpr int EW_LOG2 = EW_LOG2_;
    static constexpr int EW = 1 << EW_LOG2;   // tile width (columns)
    static constexpr int NS = NT / EW;        // strips
    static constexpr int EH = NS * Q;         // tile height (rows)
    static constexpr bool REG = REG_;         // x-tilde of owned slots in registers (else shared memory)
    static constexpr bool SKIP = SKIP_;       // skip rows that can no longer reach the interior
    static constexpr int E = F * Q;           // slots per thread
    static constexpr int NP = E / 2;          // packed register pairs per thread: element (q, f) is q F + f
    // Shared memory, in float2 words (frame pairs).  A warp is one row of a
    // strip, so a slot's left and right neighbours are adjacent lanes and
    // cross by warp shuffles; shared memory carries what crosses between
    // strips, and x-tilde and theta where they do not fit in registers
    // (REG: both in registers, only each strip's first row of theta shared).
    // Word (row q, pair k, column c) of a strip sits at (q NPR + k) EW + c, so
    // a warp's 64-bit accesses are conflict-free (a 128-bit shared access
    // moves half as many bytes per cycle as two 64-bit ones).
    static constexpr int NPR = F / 2;                     // frame pairs per row
    static constexpr int RW = NPR * EW;                   // float2 words of one tile row
    static constexpr int TS = REG ? RW : Q * RW;          // theta words per strip
    static constexpr int A_TH = 0;                        // theta [NS][TS]
    static constexpr int A_WV = A_TH + NS * TS;           // w_v (then p_v) of each strip's last row [NS][NPR][EW]
    static constexpr int A_U = A_WV + NS * RW;            // ADMM u^(t) for x in the last launch [NS][Q][NPR][EW]
    static constexpr int A_XT = A_U + NS * Q * RW;        // x-tilde [NS][Q][NPR][EW] (only when !REG)
    static constexpr size_t SMEM = (size_t)(A_XT + (REG ? 0 : NS * Q * RW)) * sizeof(float2);
    static_assert(NT % EW == 0, "a CTA must cover whole rows");
    static_assert(EW == 32, "a warp is one strip row");
    static_assert(F % 2 == 0, "frames pair up for packed arithmetic");
    static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
};

// The same tile with every slot's theta and w_h in padded 128-bit shared
// blocks (the horizontal neighbours read the adjacent blocks): kept for the
// 24-frame tile, where 256 threads of 48 slots each left the shuffle form
// 5% (single) to 14% (batched, FP32) slower.
template <int NT_, int Q_, int F_, int EW_LOG2_, bool REG_, bool SKIP_>
struct BlkCfg {
    static constexpr bool MICRO = false;
    static constexpr bool SHFL = false;
    static constexpr int NT = NT_;            // threads per CTA
    static constexpr int Q = Q_;              // rows per strip (pixels per thread)
    static constexpr int F = F_;              // frames held per CTA
    static constexpr int EW_LOG2 = EW_LOG2_;
    static constexpr int EW = 1 << EW_LOG2;   // tile width (columns)
    static constexpr int NS = NT / EW;        // strips
    static constexpr int EH = NS * Q;         // tile height (rows)
    static constexpr bool REG = REG_;         // x-tilde of owned slots in registers (else shared memory)
    static constexpr bool SKIP = SKIP_;       // skip rows that can no longer reach the interior
    static constexpr int E = F * Q;           // slots per thread
    static constexpr int NP = E / 2;          // packed register pairs per thread: element (q, f) is q F + f
    // Shared memory, in floats.  Every thread's slots form one block of BLK
    // words, element (q, f) at q FP + f with each row's frames padded to a
    // multiple of 4 (FP), so rows and groups of 4 frames move as 128-bit
    // words.  The blocks of a strip sit column by column, with one zero pad
    // block on each side (columns -1 and EW): a thread reads its left and
    // right neighbours' blocks with 128-bit loads and edge columns need no
    // tests.  w_v of a strip's last row has blocks of BLKV words (one word for
    // one-frame tiles).
    static constexpr int FP = (F + 3) / 4 * 4;
    static constexpr int ES = Q * FP;                           // shared words of a thread's slots
    static constexpr int BLK = block_words(ES);
    static constexpr int BLKV = block_words(FP);
    static constexpr int SROW = (EW + 2) * BLK;                 // one strip of a padded slot array
    static constexpr int A_TH = 0;                              // theta          [NS][EW + 2][BLK]
    static constexpr int A_WH = A_TH + NS * SROW;               // w_h (then p_h) [NS][EW + 2][BLK]
    static constexpr int A_WV = A_WH + NS * SROW;               // w_v (then p_v) of each strip's last row [NS][EW][BLKV]
    static constexpr int A_XT = A_WV + ((NS * EW * BLKV + 3) & ~3);  // x-tilde [NS][EW][BLK] (only when !REG)
    static constexpr size_t SMEM = (size_t)(A_XT + (REG ? 0 : NS * EW * BLK)) * sizeof(float);
    static_assert(NT % EW == 0, "a CTA must cover whole rows");
    static_assert(EW % 32 == 0, "a warp must stay inside one strip row");
    static_assert(F % 2 == 0, "frames pair up for packed arithmetic");
    static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
};

// Element (q, f) of a packed register array: pair (q F + f) / 2, lane (q F + f) % 2.
template <int F>
__device__ __forceinline__ float& el(float2* a, int q, int f) {
    float2& p = a[(q * F + f) >> 1];
    return ((q * F + f) & 1) ? p.y : p.x;
}

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
    __device__ const T* warm_in(int i) const { return b->warm_in[i]; }
    __device__ T* warm_out(int i) const { return b->warm_out[i]; }
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
    __device__ const T* warm_in(int) const { return nullptr; }  // batched solves start w at 0
    __device__ T* warm_out(int) const { return nullptr; }
};

// One VTV tile (bx, by) of one problem.  `a` carries the launch-wide settings (K, halo, first/last, lambda, momentum),
// `p` the problem's geometry and buffers.
//
// Per dual update (Algorithm 1, ATV-FGP box), in the order of scalar FP32
// operations that the one-update-per-launch kernel also follows, so the two
// paths agree bit for bit:
//   theta = fma(-lambda, (w_h,left - w_h) + (w_v,up - w_v), xt)
//   a_h   = fma(theta_right - theta, step_h, w_h),  a_v likewise downwards
//   p     = a / max(1, |a|): clamp (ATV); a * min(1, rsqrt(fma(a_h, a_h, a_v a_v)))
//           (ITV2D); a * min(1, rsqrt(n2_even + n2_odd)) with n2_par = fma(a_h, a_h,
//           fma(a_v, a_v, n2_par)) over the frames of that parity (VTV)
//   w     = fma(c, p - p_prev, p)
// (In the first launch w = 0, and fma(-lambda, 0, xt) = xt exactly.)  The
// tile packs pairs of frames of one pixel into float2 lanes and always
// updates all F frames: frames B..F-1 hold zeros, their a is zero and they
// add exact zeros to the norm.
//
// BORDER: the tile has rows outside the image or its last row, so the
// gradient steps carry per-row factors (zero where a difference is not
// defined).  Interior tiles fold the column conditions into one factor per
// thread: where a factor is zero, w starts at zero and stays zero (a = w +
// 0 * difference projects to zero), as the per-row form gives.
template <typename T, int TV, class Cfg, bool BORDER, class Prob>
__device__ __forceinline__ void fused_tile_impl(const FusedArgs& a, const Prob& p, int bx, int by, int bz,
                                                float* smem) {
    constexpr int Q = Cfg::Q, F = Cfg::F, EW = Cfg::EW, EH = Cfg::EH, NS = Cfg::NS;
    constexpr int NP = Cfg::NP, NPR = Cfg::NPR, RW = Cfg::RW, TS = Cfg::TS;
    constexpr bool REG = Cfg::REG, SKIP = Cfg::SKIP;
    static_assert(F > 1 && TV == SCI_TV_VTV, "frame tiles are for VTV (one-frame tiles: fused_tile_rows)");

    const Geo g = p.g();
    const int H = a.halo;
    const int TI = fused_interior(EH, H), TJ = fused_interior(EW, H);  // interior size
    const int gi0 = by * TI - H, gj0 = bx * TJ - H;
    const int nfr = g.B;                         // frames of the problem in this CTA
    constexpr int f0 = 0;                        // global frame of slot f = 0 (bz unused)
    (void)bz;
    const int tid = threadIdx.x;
    const int col = tid & (EW - 1);              // = the lane
    const int strip = tid >> Cfg::EW_LOG2;       // = the warp
    const int r0 = strip * Q;                    // first row of the strip
    const int gj = gj0 + col;
    const bool col_in = gj >= 0 && gj < g.ny;
    const bool col_int = col >= H && col < EW - H + 1;
    const int gi_top = gi0 + r0;

    // Shared float2 words: theta (REG: of the strip's first row only), w_v of
    // the strip's last row, and the strips above / below (strip-uniform tests
    // guard the reads past the first and last strip).
    float2* const sm2 = reinterpret_cast<float2*>(smem);
    float2* const th_own = sm2 + Cfg::A_TH + strip * TS + col;   // (q, k) at (q NPR + k) EW
    float2* const wv_own = sm2 + Cfg::A_WV + strip * RW + col;
    const float2* const th_down = th_own + TS;   // read only when has_down
    const float2* const wv_up = wv_own - RW;     // read only when has_up
    float2* const u_own = sm2 + Cfg::A_U + strip * Q * RW + col;   // [q][k] at (q NPR + k) EW
    float2* const xt_own = sm2 + Cfg::A_XT + strip * Q * RW + col;  // only when !REG
    const bool has_up = strip > 0, has_down = strip < NS - 1;

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
    const float step = a.step;
    const float step_h = (col_in && gj < g.ny - 1) ? step : 0.f;
    const float step_v = col_in ? step : 0.f;
    auto fac = [&](unsigned m, int q) -> float { return ((m >> q) & 1u) ? step : 0.f; };

    float2 PH[NP], PV[NP], WH[NP], WV[NP];
    float2 X[REG ? NP : 1], TH[REG ? NP : 1];

    // ---- load x-tilde (and the carried duals) for the whole extended tile ----
    // Every load is issued unconditionally -- a pixel outside the image reads
    // pixel 0 of its frame and is zeroed afterwards -- and none is consumed
    // before all are issued, so a thread's loads are in flight together
    // rather than one row at a time.
    const long long pix_top = (long long)gi_top * g.ny + gj;
    auto pix_of = [&](int q) -> long long { return ((in_m >> q) & 1u) ? pix_top + (long long)q * g.ny : 0; };
    float2 XS[REG ? 1 : NP];  // x-tilde staging for tiles that keep it in shared memory
    auto xe = [&](int q, int f) -> float& { return REG ? el<F>(X, q, f) : el<F>(XS, q, f); };
    const bool warm_first = a.first && a.warm;  // w from the previous TVdenoise, p = 0
    if (!a.first) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long pix = pix_of(q);
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                const long long gidx = (long long)(f0 + f) * g.n + pix;
                el<F>(PH, q, f) = ldraw<T>(p.st_in(0), gidx);
                el<F>(PV, q, f) = ldraw<T>(p.st_in(1), gidx);
                el<F>(WH, q, f) = ldraw<T>(p.st_in(2), gidx);
                el<F>(WV, q, f) = ldraw<T>(p.st_in(3), gidx);
            }
        }
    } else if (warm_first) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long pix = pix_of(q);
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                const long long gidx = (long long)(f0 + f) * g.n + pix;
                el<F>(WH, q, f) = ldraw<T>(p.warm_in(0), gidx);
                el<F>(WV, q, f) = ldraw<T>(p.warm_in(1), gidx);
            }
        }
    }
    if (a.mode == OuterMode::Prox) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long pix = pix_of(q);
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                xe(q, f) = __ldg(p.xin() + (long long)(f0 + f) * g.n + pix);
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
                xe(q, f) = ldraw<T>(p.theta_in(), (long long)(f0 + f) * g.n + pix);
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                xe(q, f) = rt<T>(cvraw<T>(xe(q, f)) + mask_bit(word[q], f0 + f) * rv[q]);
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long pix = pix_of(q);
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                xe(q, f) = ldraw<T>(p.xt(), (long long)(f0 + f) * g.n + pix);
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                xe(q, f) = cvraw<T>(xe(q, f));
            }
        }
    }
    if (!a.first || warm_first) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                el<F>(PH, q, f) = cvraw<T>(el<F>(PH, q, f));
                el<F>(PV, q, f) = cvraw<T>(el<F>(PV, q, f));
                el<F>(WH, q, f) = cvraw<T>(el<F>(WH, q, f));
                el<F>(WV, q, f) = cvraw<T>(el<F>(WV, q, f));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const bool in = (in_m >> q) & 1u;
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const bool live = in && f < nfr;
            if (!live) xe(q, f) = 0.f;
            if (a.first || !live) {
                el<F>(PH, q, f) = 0.f;
                el<F>(PV, q, f) = 0.f;
            }
            if ((a.first && !a.warm) || !live) {
                el<F>(WH, q, f) = 0.f;
                el<F>(WV, q, f) = 0.f;
            }
        }
    }
    // a register pair (row q, frames 2k, 2k + 1) is element q NPR + k
    if (!REG) {
#pragma unroll
        for (int e2 = 0; e2 < NP; ++e2) xt_own[e2 * EW] = XS[e2];
    }
#pragma unroll
    for (int k = 0; k < NPR; ++k) wv_own[k * EW] = WV[(Q - 1) * NPR + k];
    __syncthreads();

    const float2 nlam2 = dup2(-a.lambda);
    const float2 steph2 = dup2(step_h), stepv2 = dup2(step_v);
    // Two updates per loop trip let the compiler alternate registers instead
    // of copying the loop-carried duals; the 16- and 24-frame VTV tiles, near
    // the register limit, run one.
    constexpr int kUnroll = F > 10 ? 1 : 2;
#pragma unroll kUnroll
    for (int s = 0; s < a.K; ++s) {
        const float2 c2 = dup2(a.coef[s]);
        // rows whose p stays exact after this update: [1 + s, EH - 1 - s);
        // theta is needed on those rows and the one below (strip-uniform, so
        // every lane of a warp runs the same shuffles)
        const int rlo = 1 + s, rhi = EH - 1 - s;
        const int qlo = SKIP ? max(rlo - r0, 0) : 0;
        const int qhi_p = SKIP ? min(rhi - r0, Q) : Q, qhi_t = SKIP ? min(rhi + 1 - r0, Q) : Q;
        // ---- theta = xt - lambda (D^T w), frames paired; w_h of the left
        //      neighbour by shuffle, w_v of the row above from the strip above ----
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (q < qlo || q >= qhi_t) continue;
#pragma unroll
            for (int k = 0; k < NPR; ++k) {
                const int e2 = q * NPR + k;
                const float2 wl = shfl_up2(WH[e2]);
                float2 wu = make_float2(0.f, 0.f);
                if (q > 0) wu = WV[q > 0 ? e2 - NPR : 0];
                else if (has_up) wu = wv_up[k * EW];
                const float2 x2 = REG ? X[REG ? e2 : 0] : xt_own[e2 * EW];
                const float2 t = fma2(nlam2, add2(sub2(wl, WH[e2]), sub2(wu, WV[e2])), x2);
                if (REG) TH[REG ? e2 : 0] = t;
                if (!REG || q == 0) th_own[e2 * EW] = t;
            }
        }
        __syncthreads();
        // ---- a = w + step * D theta (kept in the w registers), norm over frames,
        //      projection onto the per-pixel ball, momentum ----
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (q < qlo || q >= qhi_p) continue;
            float2 sh = steph2, sv = stepv2;
            if (BORDER) {
                sh = dup2(fac(ah_m, q));
                sv = dup2(fac(av_m, q));
            }
            float2 n2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < NPR; ++k) {
                const int e2 = q * NPR + k;
                const float2 tt = REG ? TH[REG ? e2 : 0] : th_own[e2 * EW];
                const float2 tr = shfl_down2(tt);
                float2 td = tt;
                if (q < Q - 1) td = REG ? TH[REG && q < Q - 1 ? e2 + NPR : 0] : th_own[(e2 + NPR) * EW];
                else if (has_down) td = th_down[k * EW];
                const float2 ah = fma2(sub2(tr, tt), sh, WH[e2]);
                const float2 av = fma2(sub2(td, tt), sv, WV[e2]);
                WH[e2] = ah;
                WV[e2] = av;
                n2 = fma2(ah, ah, fma2(av, av, n2));
            }
            const float2 vs = dup2(fminf(1.f, rsqrt_ftz(n2.x + n2.y)));
#pragma unroll
            for (int k = 0; k < NPR; ++k) {
                const int e2 = q * NPR + k;
                const float2 nh = mul2(WH[e2], vs), nv = mul2(WV[e2], vs);
                WH[e2] = fma2(c2, sub2(nh, PH[e2]), nh);
                WV[e2] = fma2(c2, sub2(nv, PV[e2]), nv);
                PH[e2] = nh;
                PV[e2] = nv;
            }
        }
#pragma unroll
        for (int k = 0; k < NPR; ++k) wv_own[k * EW] = WV[(Q - 1) * NPR + k];
        __syncthreads();
    }

    // ---- epilogue ----
    auto x_of = [&](int q, int f) -> float {  // x-tilde of slot (q, f)
        if constexpr (REG) return el<F>(X, q, f);
        const float2 v = xt_own[((q * F + f) >> 1) * EW];
        return (f & 1) ? v.y : v.x;
    };
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
                if (a.first && a.mode != OuterMode::Prox) st<T>(p.xt(), gidx, x_of(q, f));
                st<T>(p.st_out(0), gidx, el<F>(PH, q, f));
                st<T>(p.st_out(1), gidx, el<F>(PV, q, f));
                st<T>(p.st_out(2), gidx, el<F>(WH, q, f));
                st<T>(p.st_out(3), gidx, el<F>(WV, q, f));
            }
        }
        return;
    }
    // theta = xt - lambda D^T p needs p_h of the left neighbour (a shuffle,
    // into the theta registers or words, free now) and p_v of the row above
    // (staged where w_v was: the loop ended with a barrier).
#pragma unroll
    for (int e2 = 0; e2 < NP; ++e2) {
        const float2 pl = shfl_up2(PH[e2]);
        if (REG) TH[REG ? e2 : 0] = pl;
        else th_own[e2 * EW] = pl;
    }
#pragma unroll
    for (int k = 0; k < NPR; ++k) wv_own[k * EW] = PV[(Q - 1) * NPR + k];
    // x^(t+1) = xt - u^(t) for ADMM (only when x is requested): u^(t) is read
    // before u^(t+1) overwrites it.  Issue every load first (into the
    // thread's own words of a shared array) so none waits behind a store it
    // might alias.
    const bool want_xu = a.mode == OuterMode::Admm && p.x_out() != nullptr;
    if (want_xu) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int r = r0 + q;
            const bool mine = ((in_m >> q) & 1u) && col_int && r >= H && r < EH - H + 1;
            const long long pix = mine ? (long long)(gi_top + q) * g.ny + gj : 0;
#pragma unroll
            for (int k = 0; k < NPR; ++k) {
                const int f = 2 * k;
                float2 uv = make_float2(0.f, 0.f);
                if (mine && f < nfr) uv.x = ldg<T>(p.u_in(), (long long)(f0 + f) * g.n + pix);
                if (mine && f + 1 < nfr) uv.y = ldg<T>(p.u_in(), (long long)(f0 + f + 1) * g.n + pix);
                u_own[(q * NPR + k) * EW] = uv;
            }
        }
    }
    __syncthreads();
    // VTV tiles hold every frame of a pixel: form the next residual here (the
    // per-pixel order of the separate residual pass)
    const bool fold_r = a.r_next != nullptr && a.mode != OuterMode::Prox;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int r = r0 + q;
        if (!((in_m >> q) & 1u) || !col_int || r < H || r >= EH - H + 1) continue;
        const long long pix = (long long)(gi_top + q) * g.ny + gj;
        const uint32_t word = fold_r ? __ldg(p.bits() + pix) : 0u;
        float acc = 0.f;
#pragma unroll
        for (int f = 0; f < F; ++f) {
            if (f >= nfr) break;
            float pl;
            if constexpr (REG) {
                pl = el<F>(TH, q, f);
            } else {
                const float2 v = th_own[((q * F + f) >> 1) * EW];
                pl = (f & 1) ? v.y : v.x;
            }
            float pu = 0.f;
            if (q > 0) {
                pu = el<F>(PV, q > 0 ? q - 1 : 0, f);
            } else if (has_up) {
                const float2 v = wv_up[(f >> 1) * EW];
                pu = (f & 1) ? v.y : v.x;
            }
            const float x0 = x_of(q, f);
            const float th = __fmaf_rn(-a.lambda, (pl - el<F>(PH, q, f)) + (pu - el<F>(PV, q, f)), x0);
            const long long gidx = (long long)(f0 + f) * g.n + pix;
            if (a.mode == OuterMode::Prox) {
                p.theta_f32()[gidx] = th;
                continue;
            }
            st<T>(p.theta_out(), gidx, th);
            const float thr = rt<T>(th);
            float v = thr;
            if (a.mode == OuterMode::Gap) {
                if (p.x_out() != nullptr) p.x_out()[gidx] = x0;
            } else {
                const float un = rt<T>(x0 - thr);
                st<T>(p.u_out(), gidx, un);
                if (want_xu) {
                    const float2 uv = u_own[((q * F + f) >> 1) * EW];
                    p.x_out()[gidx] = x0 - ((f & 1) ? uv.y : uv.x);
                }
                v = thr - un;
            }
            if (fold_r) acc = __fmaf_rn(mask_bit(word, f0 + f), v, acc);
            if (a.warm) {
                st<T>(p.warm_out(0), gidx, el<F>(WH, q, f));
                st<T>(p.warm_out(1), gidx, el<F>(WV, q, f));
            }
        }
        if (fold_r) a.r_next[pix] = __ldg(a.rinv + pix) * (__ldg(a.y + pix) - acc);
    }
}

// One VTV tile (bx, by) of one problem on the block layout (BlkCfg); the
// same arithmetic, in the same order, as fused_tile_impl.  `a` carries the launch-wide settings (K, halo, first/last, lambda, momentum),
// `p` the problem's geometry and buffers.
//
// Per dual update (Algorithm 1, ATV-FGP box), in the order of scalar FP32
// operations that the one-update-per-launch kernel also follows, so the two
// paths agree bit for bit:
//   theta = fma(-lambda, (w_h,left - w_h) + (w_v,up - w_v), xt)
//   a_h   = fma(theta_right - theta, step_h, w_h),  a_v likewise downwards
//   p     = a / max(1, |a|): clamp (ATV); a * min(1, rsqrt(fma(a_h, a_h, a_v a_v)))
//           (ITV2D); a * min(1, rsqrt(n2_even + n2_odd)) with n2_par = fma(a_h, a_h,
//           fma(a_v, a_v, n2_par)) over the frames of that parity (VTV)
//   w     = fma(c, p - p_prev, p)
// (In the first launch w = 0, and fma(-lambda, 0, xt) = xt exactly.)  The
// tile packs pairs of frames of one pixel into float2 lanes and always
// updates all F frames: frames B..F-1 hold zeros, their a is zero and they
// add exact zeros to the norm.
//
// BORDER: the tile has rows outside the image or its last row, so the
// gradient steps carry per-row factors (zero where a difference is not
// defined).  Interior tiles fold the column conditions into one factor per
// thread: where a factor is zero, w starts at zero and stays zero (a = w +
// 0 * difference projects to zero), as the per-row form gives.
template <typename T, int TV, class Cfg, bool BORDER, class Prob>
__device__ __forceinline__ void fused_tile_blk(const FusedArgs& a, const Prob& p, int bx, int by, int bz,
                                                float* smem) {
    constexpr int Q = Cfg::Q, F = Cfg::F, EW = Cfg::EW, EH = Cfg::EH, NS = Cfg::NS, FP = Cfg::FP;
    constexpr int NP = Cfg::NP, BLK = Cfg::BLK, BLKV = Cfg::BLKV, SROW = Cfg::SROW;
    constexpr bool REG = Cfg::REG, SKIP = Cfg::SKIP;
    static_assert(F > 1 && TV == SCI_TV_VTV, "frame tiles are for VTV (one-frame tiles: fused_tile_rows)");

    const Geo g = p.g();
    const int H = a.halo;
    const int TI = fused_interior(EH, H), TJ = fused_interior(EW, H);  // interior size
    const int gi0 = by * TI - H, gj0 = bx * TJ - H;
    const int nfr = g.B;                         // frames of the problem in this CTA
    constexpr int f0 = 0;                        // global frame of slot f = 0 (bz unused)
    (void)bz;
    const int tid = threadIdx.x;
    const int col = tid & (EW - 1);
    const int strip = tid >> Cfg::EW_LOG2;
    const int r0 = strip * Q;                    // first row of the strip
    const int gj = gj0 + col;
    const bool col_in = gj >= 0 && gj < g.ny;
    const bool col_int = col >= H && col < EW - H + 1;
    const int gi_top = gi0 + r0;

    // This thread's blocks and its neighbours'.  th_down (strip NS - 1) and
    // wv_up (strip 0) then point at other, valid shared words, whose values
    // are replaced before use.
    float* const th_own = smem + Cfg::A_TH + strip * SROW + (col + 1) * BLK;
    float* const wh_own = smem + Cfg::A_WH + strip * SROW + (col + 1) * BLK;
    const float* const th_right = th_own + BLK;
    const float* const wh_left = wh_own - BLK;
    const float* const th_down = th_own + SROW;
    float* const wv_own = smem + Cfg::A_WV + (strip * EW + col) * BLKV;
    const float* const wv_up = wv_own - EW * BLKV;
    float* const xt_own = smem + Cfg::A_XT + (strip * EW + col) * BLK;  // only when !REG
    const bool has_up = strip > 0, has_down = strip < NS - 1;

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
    const float step = a.step;
    const float step_h = (col_in && gj < g.ny - 1) ? step : 0.f;
    const float step_v = col_in ? step : 0.f;
    auto fac = [&](unsigned m, int q) -> float { return ((m >> q) & 1u) ? step : 0.f; };

    float2 PH[NP], PV[NP], WH[NP], WV[NP];
    float2 X[REG ? NP : 1];

    // ---- load x-tilde (and the carried duals) for the whole extended tile ----
    // Every load is issued unconditionally -- a pixel outside the image reads
    // pixel 0 of its frame and is zeroed afterwards -- and none is consumed
    // before all are issued, so a thread's loads are in flight together
    // rather than one row at a time.
    const long long pix_top = (long long)gi_top * g.ny + gj;
    auto pix_of = [&](int q) -> long long { return ((in_m >> q) & 1u) ? pix_top + (long long)q * g.ny : 0; };
    float2 XS[REG ? 1 : NP];  // x-tilde staging for tiles that keep it in shared memory
    auto xe = [&](int q, int f) -> float& { return REG ? el<F>(X, q, f) : el<F>(XS, q, f); };
    const bool warm_first = a.first && a.warm;  // w from the previous TVdenoise, p = 0
    if (!a.first) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long pix = pix_of(q);
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                const long long gidx = (long long)(f0 + f) * g.n + pix;
                el<F>(PH, q, f) = ldraw<T>(p.st_in(0), gidx);
                el<F>(PV, q, f) = ldraw<T>(p.st_in(1), gidx);
                el<F>(WH, q, f) = ldraw<T>(p.st_in(2), gidx);
                el<F>(WV, q, f) = ldraw<T>(p.st_in(3), gidx);
            }
        }
    } else if (warm_first) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long pix = pix_of(q);
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                const long long gidx = (long long)(f0 + f) * g.n + pix;
                el<F>(WH, q, f) = ldraw<T>(p.warm_in(0), gidx);
                el<F>(WV, q, f) = ldraw<T>(p.warm_in(1), gidx);
            }
        }
    }
    if (a.mode == OuterMode::Prox) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long pix = pix_of(q);
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                xe(q, f) = __ldg(p.xin() + (long long)(f0 + f) * g.n + pix);
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
                xe(q, f) = ldraw<T>(p.theta_in(), (long long)(f0 + f) * g.n + pix);
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                xe(q, f) = rt<T>(cvraw<T>(xe(q, f)) + mask_bit(word[q], f0 + f) * rv[q]);
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long pix = pix_of(q);
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                xe(q, f) = ldraw<T>(p.xt(), (long long)(f0 + f) * g.n + pix);
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                xe(q, f) = cvraw<T>(xe(q, f));
            }
        }
    }
    if (!a.first || warm_first) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                el<F>(PH, q, f) = cvraw<T>(el<F>(PH, q, f));
                el<F>(PV, q, f) = cvraw<T>(el<F>(PV, q, f));
                el<F>(WH, q, f) = cvraw<T>(el<F>(WH, q, f));
                el<F>(WV, q, f) = cvraw<T>(el<F>(WV, q, f));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const bool in = (in_m >> q) & 1u;
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const bool live = in && f < nfr;
            if (!live) xe(q, f) = 0.f;
            if (a.first || !live) {
                el<F>(PH, q, f) = 0.f;
                el<F>(PV, q, f) = 0.f;
            }
            if ((a.first && !a.warm) || !live) {
                el<F>(WH, q, f) = 0.f;
                el<F>(WV, q, f) = 0.f;
            }
        }
    }
    // A register pair (frames f, f+1 of row q) is the 128-bit half at words
    // q FP + f of a shared block; the padding frames of a row store zeros.
    auto put_block = [&](float* blk, const float2* R) {
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int c = 0; c < FP / 4; ++c) {
                const int e2 = (q * F + 4 * c) / 2;
                sts4(blk + q * FP + 4 * c, R[e2], 4 * c + 2 < F ? R[4 * c + 2 < F ? e2 + 1 : 0] : make_float2(0.f, 0.f));
            }
    };
    auto put_last_row = [&](float* blk, const float2* R) {
#pragma unroll
        for (int c = 0; c < FP / 4; ++c) {
            const int e2 = ((Q - 1) * F + 4 * c) / 2;
            sts4(blk + 4 * c, R[e2], 4 * c + 2 < F ? R[4 * c + 2 < F ? e2 + 1 : 0] : make_float2(0.f, 0.f));
        }
    };
    put_block(wh_own, WH);
    if (!REG) put_block(xt_own, XS);
    put_last_row(wv_own, WV);
    // zero pad blocks (columns -1 and EW of every strip) of theta and w_h
    for (int e = tid; e < NS * 2 * (BLK / 4); e += Cfg::NT) {
        const int s = e / (2 * (BLK / 4)), rem = e - s * 2 * (BLK / 4);
        const int side = rem / (BLK / 4), w4 = rem - side * (BLK / 4);
        const int off = s * SROW + (side ? (EW + 1) * BLK : 0) + 4 * w4;
        *reinterpret_cast<float4*>(smem + Cfg::A_TH + off) = make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float4*>(smem + Cfg::A_WH + off) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();

    const float2 nlam2 = dup2(-a.lambda);
    const float2 steph2 = dup2(step_h), stepv2 = dup2(step_v);
    // Two updates per loop trip let the compiler alternate registers instead
    // of copying the loop-carried duals; the 16- and 24-frame VTV tiles, near
    // the register limit, run one.
    constexpr int kUnroll = F > 10 ? 1 : 2;
#pragma unroll kUnroll
    for (int s = 0; s < a.K; ++s) {
        const float2 c2 = dup2(a.coef[s]);
        // rows whose p stays exact after this update: [1 + s, EH - 1 - s);
        // theta is needed on those rows and the one below
        const int rlo = 1 + s, rhi = EH - 1 - s;
        const int qlo = SKIP ? max(rlo - r0, 0) : 0;
        const int qhi_p = SKIP ? min(rhi - r0, Q) : Q, qhi_t = SKIP ? min(rhi + 1 - r0, Q) : Q;
        // ---- theta = xt - lambda (D^T w), frames paired ----
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (q < qlo || q >= qhi_t) continue;
#pragma unroll
            for (int c = 0; c < FP / 4; ++c) {
                const float4 wl = lds4(wh_left + q * FP + 4 * c);
                float4 xv = make_float4(0.f, 0.f, 0.f, 0.f);
                if (!REG) xv = lds4(xt_own + q * FP + 4 * c);
                float4 wu = make_float4(0.f, 0.f, 0.f, 0.f);
                if (q == 0) {
                    const float4 w = lds4(wv_up + 4 * c);
                    if (has_up) wu = w;
                }
                float2 th[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (4 * c + 2 * h >= F) continue;
                    const int e2 = (q * F + 4 * c) / 2 + h;
                    const float2 x2 = REG ? X[REG ? e2 : 0] : (h ? hi2(xv) : lo2(xv));
                    const float2 wu2 = q > 0 ? WV[q > 0 ? e2 - F / 2 : 0] : (h ? hi2(wu) : lo2(wu));
                    th[h] = fma2(nlam2, add2(sub2(h ? hi2(wl) : lo2(wl), WH[e2]), sub2(wu2, WV[e2])), x2);
                }
                sts4(th_own + q * FP + 4 * c, th[0], th[1]);
            }
        }
        __syncthreads();
        // ---- a = w + step * D theta (kept in the w registers), norm over frames,
        //      projection onto the per-pixel ball, momentum ----
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (q < qlo || q >= qhi_p) continue;
            float2 sh = steph2, sv = stepv2;
            if (BORDER) {
                sh = dup2(fac(ah_m, q));
                sv = dup2(fac(av_m, q));
            }
            float2 n2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < FP / 4; ++c) {
                const float4 tr = lds4(th_right + q * FP + 4 * c);
                const float4 t0 = lds4(th_own + q * FP + 4 * c);
                float4 td;
                if (q < Q - 1) {
                    td = lds4(th_own + (q + 1) * FP + 4 * c);
                } else {
                    const float4 d = lds4(th_down + 4 * c);
                    td = has_down ? d : t0;
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (4 * c + 2 * h >= F) continue;
                    const int e2 = (q * F + 4 * c) / 2 + h;
                    const float2 tt = h ? hi2(t0) : lo2(t0);
                    const float2 ah = fma2(sub2(h ? hi2(tr) : lo2(tr), tt), sh, WH[e2]);
                    const float2 av = fma2(sub2(h ? hi2(td) : lo2(td), tt), sv, WV[e2]);
                    WH[e2] = ah;
                    WV[e2] = av;
                    n2 = fma2(ah, ah, fma2(av, av, n2));
                }
            }
            const float2 vs = dup2(fminf(1.f, rsqrt_ftz(n2.x + n2.y)));
#pragma unroll
            for (int f = 0; f < F; f += 2) {
                const int e2 = (q * F + f) / 2;
                const float2 nh = mul2(WH[e2], vs), nv = mul2(WV[e2], vs);
                WH[e2] = fma2(c2, sub2(nh, PH[e2]), nh);
                WV[e2] = fma2(c2, sub2(nv, PV[e2]), nv);
                PH[e2] = nh;
                PV[e2] = nv;
            }
#pragma unroll
            for (int c = 0; c < FP / 4; ++c) {
                const int e2 = (q * F + 4 * c) / 2;
                sts4(wh_own + q * FP + 4 * c, WH[e2],
                     4 * c + 2 < F ? WH[4 * c + 2 < F ? e2 + 1 : 0] : make_float2(0.f, 0.f));
            }
        }
        put_last_row(wv_own, WV);
        __syncthreads();
    }

    // ---- epilogue ----
    auto sidx = [&](int q, int f) { return q * FP + f; };  // element (q, f) of a shared block
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
                    st<T>(p.xt(), gidx, REG ? el<F>(X, q, f) : xt_own[sidx(q, f)]);
                st<T>(p.st_out(0), gidx, el<F>(PH, q, f));
                st<T>(p.st_out(1), gidx, el<F>(PV, q, f));
                st<T>(p.st_out(2), gidx, el<F>(WH, q, f));
                st<T>(p.st_out(3), gidx, el<F>(WV, q, f));
            }
        }
        return;
    }
    // theta = xt - lambda D^T p needs p_h of the left neighbour and p_v of the
    // row above: stage them where w_h / w_v were (the loop ended with a barrier).
    put_block(wh_own, PH);
    put_last_row(wv_own, PV);
    // x^(t+1) = xt - u^(t) for ADMM (only when x is requested): u^(t) is read
    // before u^(t+1) overwrites it.  Issue every load first (into the thread's
    // own theta block, free now) so none waits behind a store it might alias.
    if (a.mode == OuterMode::Admm && p.x_out() != nullptr) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int r = r0 + q;
            const bool mine = ((in_m >> q) & 1u) && col_int && r >= H && r < EH - H + 1;
            const long long pix = mine ? (long long)(gi_top + q) * g.ny + gj : 0;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nfr) break;
                th_own[sidx(q, f)] = mine ? ldg<T>(p.u_in(), (long long)(f0 + f) * g.n + pix) : 0.f;
            }
        }
    }
    __syncthreads();
    // VTV tiles hold every frame of a pixel: form the next residual here (the
    // per-pixel order of the separate residual pass)
    const bool fold_r = F > 1 && a.r_next != nullptr && a.mode != OuterMode::Prox;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int r = r0 + q;
        if (!((in_m >> q) & 1u) || !col_int || r < H || r >= EH - H + 1) continue;
        const long long pix = (long long)(gi_top + q) * g.ny + gj;
        const uint32_t word = fold_r ? __ldg(p.bits() + pix) : 0u;
        float acc = 0.f;
#pragma unroll
        for (int f = 0; f < F; ++f) {
            if (f >= nfr) break;
            const float pl = wh_left[sidx(q, f)];
            float pu;
            if (q > 0) pu = el<F>(PV, q > 0 ? q - 1 : 0, f);
            else pu = has_up ? wv_up[f] : 0.f;
            const float x0 = REG ? el<F>(X, q, f) : xt_own[sidx(q, f)];
            const float th = __fmaf_rn(-a.lambda, (pl - el<F>(PH, q, f)) + (pu - el<F>(PV, q, f)), x0);
            const long long gidx = (long long)(f0 + f) * g.n + pix;
            if (a.mode == OuterMode::Prox) {
                p.theta_f32()[gidx] = th;
                continue;
            }
            st<T>(p.theta_out(), gidx, th);
            const float thr = rt<T>(th);
            float v = thr;
            if (a.mode == OuterMode::Gap) {
                if (p.x_out() != nullptr) p.x_out()[gidx] = x0;
            } else {
                const float un = rt<T>(x0 - thr);
                st<T>(p.u_out(), gidx, un);
                if (p.x_out() != nullptr) p.x_out()[gidx] = x0 - th_own[sidx(q, f)];
                v = thr - un;
            }
            if (fold_r) acc = __fmaf_rn(mask_bit(word, f0 + f), v, acc);
            if (a.warm) {
                st<T>(p.warm_out(0), gidx, el<F>(WH, q, f));
                st<T>(p.warm_out(1), gidx, el<F>(WV, q, f));
            }
        }
        if (fold_r) a.r_next[pix] = __ldg(a.rinv + pix) * (__ldg(a.y + pix) - acc);
    }
}

// ---------------------------------------------------------------- one-frame tiles
//
// ATV, ITV2D and the Clip box update every frame independently, so a CTA
// holds one frame of its tile, each thread a vertical strip of Q rows of one
// column with p, w, x-tilde and theta in registers.  Vertical neighbours are
// register reads; shared memory carries theta and w_h of every slot (the
// left / right neighbours) and w_v of each strip's last row, in row-major
// arrays with one zero pad word at each row end, so edge columns need no
// tests.  The arithmetic is scalar: packed pairs of rows, tried here, needed
// aligned register pairs that pushed this 128-register tile into spilling
// inside the update loop, which cost more than the halved arithmetic issue.
template <int NT_, int Q_, int EW_LOG2_>
struct RowCfg {
    static constexpr bool MICRO = false;
    static constexpr int NT = NT_;            // threads per CTA
    static constexpr int Q = Q_;              // rows per strip (pixels per thread)
    static constexpr int F = 1;               // one frame per CTA (blockIdx.z picks it)
    static constexpr int EW_LOG2 = EW_LOG2_;
    static constexpr int EW = 1 << EW_LOG2;   // tile width (columns)
    static constexpr int NS = NT / EW;        // strips
    static constexpr int EH = NS * Q;         // tile height (rows)
    // slot (r, c) of a slot array sits at 1 + r * LD + c; words 0, LD, 2 LD, ...
    // are the pad words (zero) left of column 0 and right of column EW - 1
    static constexpr int LD = EW + 1;
    static constexpr int FPP = EH * LD + 1;
    // shared memory: theta, w_h, and (Clip box) theta_v slot arrays [FPP]; w_v [NS][EW]
    static constexpr size_t SMEM = ((size_t)FPP * 3 + (size_t)NS * EW) * sizeof(float);
    static_assert(NT % EW == 0, "a CTA must cover whole rows");
    static_assert(EW % 32 == 0, "a warp must stay inside one strip row");
};

// One tile (bx, by) of frame bz.  Per dual update, in the scalar order the
// one-update-per-launch kernel follows (the two agree bit for bit):
//   theta = fma(-lambda, (w_h,left - w_h) + (w_v,up - w_v), xt)
//   a_h = fma(theta_right - theta, step_h, w_h), a_v likewise downwards
//   p = clamp(a, -1, 1) (ATV, Clip) or a * min(1, rsqrt(fma(a_h, a_h, a_v a_v))) (ITV2D)
//   w = fma(c, p - p_prev, p)  (Clip: w = p)
// The Clip box (kTvClip) forms theta_h = fma(-lambda, w_h,left - w_h, xt) and
// theta_v = fma(-lambda, w_v,up - w_v, xt) and takes each direction's
// gradient of its own theta.
template <typename T, int TV, class Cfg, class Prob>
__device__ __forceinline__ void fused_tile_rows(const FusedArgs& a, const Prob& p, int bx, int by, int bz,
                                                float* smem) {
    constexpr int Q = Cfg::Q, EW = Cfg::EW, EH = Cfg::EH, LD = Cfg::LD, FP = Cfg::FPP;
    constexpr bool CLIP = TV == kTvClip;
    float* s_th = smem;                      // [FPP] theta (Clip: theta_h)
    float* s_wh = s_th + FP;                 // [FPP]
    float* s_tv = s_wh + FP;                 // [FPP] Clip box: theta_v
    float* s_wv = s_tv + FP;                 // [NS][EW]: w_v of each strip's last row

    const Geo g = p.g();
    const int H = a.halo;
    const int TI = fused_interior(EH, H), TJ = fused_interior(EW, H);
    const int gi0 = by * TI - H, gj0 = bx * TJ - H;
    const int f0 = bz;
    const int tid = threadIdx.x;
    const int col = tid & (EW - 1);
    const int strip = tid >> Cfg::EW_LOG2;
    const int r0 = strip * Q;
    const int gj = gj0 + col;
    const bool col_in = gj >= 0 && gj < g.ny;
    const bool col_int = col >= H && col < EW - H + 1;
    const int gi_top = gi0 + r0;

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
    // steps, zero where the gradient component is defined as zero; w stays
    // zero there, so the masked and unmasked forms agree.
    const bool rows_inner = gi_top >= 0 && gi_top + Q - 1 < g.nx - 1;
    const float step_h = (col_in && gj < g.ny - 1) ? a.step : 0.f;
    const float step_v = col_in ? a.step : 0.f;

    float ph[Q], pv[Q], wh[Q], wv[Q], xr[Q], thr[Q];

    // ---- loads for the whole extended tile, all issued before any is used ----
    const long long fbase = (long long)f0 * g.n;
    const long long pix_top = (long long)gi_top * g.ny + gj;
    auto pix_of = [&](int q) -> long long { return ((in_m >> q) & 1u) ? pix_top + (long long)q * g.ny : 0; };
    const bool warm_first = a.first && a.warm;  // w from the previous TVdenoise, p = 0
    if (!a.first) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long gidx = fbase + pix_of(q);
            ph[q] = ldraw<T>(p.st_in(0), gidx);
            pv[q] = ldraw<T>(p.st_in(1), gidx);
            wh[q] = ldraw<T>(p.st_in(2), gidx);
            wv[q] = ldraw<T>(p.st_in(3), gidx);
        }
    } else if (warm_first) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long gidx = fbase + pix_of(q);
            wh[q] = ldraw<T>(p.warm_in(0), gidx);
            wv[q] = ldraw<T>(p.warm_in(1), gidx);
        }
    }
    if (a.mode == OuterMode::Prox) {
#pragma unroll
        for (int q = 0; q < Q; ++q) xr[q] = __ldg(p.xin() + fbase + pix_of(q));
    } else if (a.first) {
        uint32_t word[Q];
        float rv[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const long long pix = pix_of(q);
            word[q] = __ldg(p.bits() + pix);
            rv[q] = __ldg(p.r() + pix);
            xr[q] = ldraw<T>(p.theta_in(), fbase + pix);
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) xr[q] = rt<T>(cvraw<T>(xr[q]) + mask_bit(word[q], f0) * rv[q]);
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) xr[q] = ldraw<T>(p.xt(), fbase + pix_of(q));
#pragma unroll
        for (int q = 0; q < Q; ++q) xr[q] = cvraw<T>(xr[q]);
    }
    if (!a.first || warm_first) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            ph[q] = cvraw<T>(ph[q]);
            pv[q] = cvraw<T>(pv[q]);
            wh[q] = cvraw<T>(wh[q]);
            wv[q] = cvraw<T>(wv[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const bool in = (in_m >> q) & 1u;
        if (!in) xr[q] = 0.f;
        if (a.first || !in) {
            ph[q] = 0.f;
            pv[q] = 0.f;
        }
        if ((a.first && !a.warm) || !in) {
            wh[q] = 0.f;
            wv[q] = 0.f;
        }
        s_wh[1 + (r0 + q) * LD + col] = wh[q];
        if (q == Q - 1) s_wv[strip * EW + col] = wv[q];
    }
    for (int e = tid; e < EH + 1; e += Cfg::NT) {  // pad words
        s_th[e * LD] = 0.f;
        s_wh[e * LD] = 0.f;
        s_tv[e * LD] = 0.f;
    }
    __syncthreads();

    const float lam = a.lambda, step = a.step;
    // two updates per loop trip let the compiler alternate registers instead
    // of copying the loop-carried duals (measured: ATV launch 63 -> 59 us);
    // the Clip box, whose extra theta_v array already spills, runs one
    constexpr int kUnroll = CLIP ? 1 : 2;
#pragma unroll kUnroll
    for (int s = 0; s < a.K; ++s) {
        const bool skip_theta = a.first && !a.warm && s == 0;  // w = 0 there: theta = xt
        // ---- theta = xt - lambda (D^T w) ----
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int o = 1 + (r0 + q) * LD + col;
            float th = xr[q], tv = xr[q];
            if (!skip_theta) {
                const float wl = s_wh[o - 1];
                float wu;
                if (q > 0) wu = wv[q > 0 ? q - 1 : 0];
                else wu = strip > 0 ? s_wv[(strip - 1) * EW + col] : 0.f;
                if (CLIP) {
                    th = __fmaf_rn(-lam, wl - wh[q], xr[q]);
                    tv = __fmaf_rn(-lam, wu - wv[q], xr[q]);
                } else {
                    th = __fmaf_rn(-lam, (wl - wh[q]) + (wu - wv[q]), xr[q]);
                }
            }
            thr[q] = th;
            s_th[o] = th;
            if (CLIP) s_tv[o] = tv;
        }
        __syncthreads();
        // ---- a = w + step * D theta, projection, momentum ----
        const float c = a.coef[s];
        auto dual_step = [&](auto masked_c) {
            constexpr bool MASKED = decltype(masked_c)::value;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const bool mh = (ah_m >> q) & 1u, mv = (av_m >> q) & 1u;
                const int o = 1 + (r0 + q) * LD + col;
                const float t0 = thr[q];
                const float tr = s_th[o + 1];
                float dv;
                if (CLIP) {
                    const float v0 = s_tv[o];
                    const float vd = (r0 + q < EH - 1) ? s_tv[o + LD] : v0;
                    dv = vd - v0;
                } else {
                    float td;
                    if (q < Q - 1) td = thr[q < Q - 1 ? q + 1 : 0];
                    else td = (r0 + q < EH - 1) ? s_th[o + LD] : t0;
                    dv = td - t0;
                }
                float ah, av;
                if (MASKED) {
                    ah = mh ? fmaf(tr - t0, step, wh[q]) : 0.f;
                    av = mv ? fmaf(dv, step, wv[q]) : 0.f;
                } else {
                    ah = fmaf(tr - t0, step_h, wh[q]);
                    av = fmaf(dv, step_v, wv[q]);
                }
                if (TV == SCI_TV_ATV || CLIP) {
                    ah = fminf(fmaxf(ah, -1.f), 1.f);
                    av = fminf(fmaxf(av, -1.f), 1.f);
                } else {
                    // a / max(1, |a|) = a * min(1, 1/|a|); 1/sqrt(0) = inf gives 1
                    const float sc = fminf(1.f, rsqrt_ftz(fmaf(ah, ah, av * av)));
                    ah *= sc;
                    av *= sc;
                }
                if (CLIP) {
                    wh[q] = ah;
                    wv[q] = av;
                } else {
                    wh[q] = fmaf(c, ah - ph[q], ah);
                    wv[q] = fmaf(c, av - pv[q], av);
                }
                ph[q] = ah;
                pv[q] = av;
                s_wh[o] = wh[q];
                if (q == Q - 1) s_wv[strip * EW + col] = wv[q];
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
            const long long gidx = fbase + (long long)(gi_top + q) * g.ny + gj;
            if (a.first && a.mode != OuterMode::Prox) st<T>(p.xt(), gidx, xr[q]);
            st<T>(p.st_out(0), gidx, ph[q]);
            st<T>(p.st_out(1), gidx, pv[q]);
            st<T>(p.st_out(2), gidx, wh[q]);
            st<T>(p.st_out(3), gidx, wv[q]);
        }
        return;
    }
    // theta = xt - lambda D^T p needs p_h of the left neighbour and p_v of the
    // row above: stage them where w_h / w_v were (the loop ended with a barrier).
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        s_wh[1 + (r0 + q) * LD + col] = ph[q];
        if (q == Q - 1) s_wv[strip * EW + col] = pv[q];
    }
    // x^(t+1) = xt - u^(t) for ADMM (only when x is requested): u^(t) is read
    // before u^(t+1) overwrites it, into the thread's own theta slots (free now)
    if (a.mode == OuterMode::Admm && p.x_out() != nullptr) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int r = r0 + q;
            const bool mine = ((in_m >> q) & 1u) && col_int && r >= H && r < EH - H + 1;
            const long long pix = mine ? (long long)(gi_top + q) * g.ny + gj : 0;
            s_th[1 + r * LD + col] = mine ? ldg<T>(p.u_in(), fbase + pix) : 0.f;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int r = r0 + q;
        if (!((in_m >> q) & 1u) || !col_int || r < H || r >= EH - H + 1) continue;
        const int o = 1 + r * LD + col;
        const float pl = s_wh[o - 1];
        float pu;
        if (q > 0) pu = pv[q > 0 ? q - 1 : 0];
        else pu = strip > 0 ? s_wv[(strip - 1) * EW + col] : 0.f;
        const float x0 = xr[q];
        const float th = __fmaf_rn(-lam, (pl - ph[q]) + (pu - pv[q]), x0);
        const long long gidx = fbase + (long long)(gi_top + q) * g.ny + gj;
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
        if (a.warm) {
            st<T>(p.warm_out(0), gidx, wh[q]);
            st<T>(p.warm_out(1), gidx, wv[q]);
        }
    }
}

// One-frame micro-tiles: thread (ty, tx) owns the MR x MC block of slots at
// rows ty MR .. ty MR + MR - 1 and columns tx MC .. tx MC + MC - 1 of an
// extended tile of (NT / TX) MR rows by TX MC columns.  A slot's left, right,
// up and down neighbours are the thread's own registers except on the block's
// edges, so one dual update exchanges four short vectors per thread -- theta
// of its first column and first row, w_h of its last column and w_v of its
// last row -- where a one-column strip exchanges every slot's theta and w_h.
// A warp holds whole rows of threads, so the left and right neighbours are
// the adjacent lanes: theta and w_h cross by warp shuffles (one 32-bit word
// per lane per cycle), and only the vertical vectors go through shared
// memory, as 64-bit halves (a 128-bit shared access moves half as many bytes
// per cycle as two 64-bit ones).
template <int NT_, int TX_LOG2_, int MR_, int MC_>
struct MicroCfg {
    static constexpr bool MICRO = true;
    static constexpr int NT = NT_;            // threads per CTA
    static constexpr int F = 1;               // one frame per CTA (blockIdx.z picks it)
    static constexpr int TX_LOG2 = TX_LOG2_;
    static constexpr int TX = 1 << TX_LOG2;   // threads along a tile row
    static constexpr int TY = NT / TX;        // threads along a tile column
    static constexpr int MR = MR_, MC = MC_;  // block rows and columns per thread
    static constexpr int EW = TX * MC;        // tile width (columns)
    static constexpr int EH = TY * MR;        // tile height (rows)
    // Exchange arrays, in floats: one MC-vector per thread as MC / 2 float2
    // planes (columns 0-1, 2-3, ...: HALF floats apart), entry (row, tx) at
    // float2 index row TX + tx of each plane, so a warp's 64-bit accesses are
    // conflict-free; zero pad rows where a tile-edge thread reads past the tile.
    //   XT: theta (Clip: theta_v) of the block's first row, rows 0 .. TY - 1 = ty, pad row TY
    //   WB: w_v (at the end p_v) of the block's last row,    rows 1 .. TY = ty + 1, pad row 0
    static constexpr int HALF = (TY + 1) * TX * 2;
    static constexpr int A_XT = 0;
    static constexpr int A_WB = A_XT + (MC / 2) * HALF;
    // Two staging tiles [EH][SW] for the epilogue's stores (see fused_tile_micro).
    static constexpr int SW = EW + 4;
    static constexpr int A_ST = A_WB + (MC / 2) * HALF;
    static constexpr size_t SMEM = (size_t)(A_ST + 2 * EH * SW) * sizeof(float);
    static_assert(NT % TX == 0 && TX >= 8 && TX <= 32 && 32 % TX == 0, "whole rows of threads in each warp");
    static_assert((MR == 2 || MR == 4) && (MC == 4 || MC == 8), "blocks of 2 or 4 rows by 4 or 8 columns");
};

// An N-vector of an exchange array: N / 2 float2 planes HALF floats apart.
template <int HALF, int N>
__device__ __forceinline__ void ld4h(const float* base, int idx, float (&v)[N]) {
#pragma unroll
    for (int p = 0; p < N / 2; ++p) {
        const float2 t = reinterpret_cast<const float2*>(base + p * HALF)[idx];
        v[2 * p] = t.x, v[2 * p + 1] = t.y;
    }
}
template <int HALF, int N>
__device__ __forceinline__ void st4h(float* base, int idx, const float (&v)[N]) {
#pragma unroll
    for (int p = 0; p < N / 2; ++p) reinterpret_cast<float2*>(base + p * HALF)[idx] = make_float2(v[2 * p], v[2 * p + 1]);
}

// One tile (bx, by) of frame bz on micro-tiles.  The arithmetic of every slot
// is fused_tile_rows's, operation for operation, so the two give the same
// bits at every interior voxel; only the tile edges, which the halo keeps away
// from the interior, read other pad values.
template <typename T, int TV, class Cfg, class Prob>
__device__ __forceinline__ void fused_tile_micro(const FusedArgs& a, const Prob& p, int bx, int by, int bz,
                                                 float* smem) {
    constexpr int MR = Cfg::MR, MC = Cfg::MC, TX = Cfg::TX, TY = Cfg::TY, EW = Cfg::EW, EH = Cfg::EH;
    constexpr bool CLIP = TV == kTvClip;

    const Geo g = p.g();
    const int H = a.halo;
    const int TI = fused_interior(EH, H), TJ = fused_interior(EW, H);
    const int gi0 = by * TI - H, gj0 = bx * TJ - H;
    const int tid = threadIdx.x;
    const int tx = tid & (TX - 1), ty = tid >> Cfg::TX_LOG2;
    const int r0 = ty * MR, c0 = tx * MC;  // the block's first row and column in the tile
    const int gi_top = gi0 + r0, gj_left = gj0 + c0;
    const long long fbase = (long long)bz * g.n;

    constexpr int HALF = Cfg::HALF;
    float* const XT = smem + Cfg::A_XT;
    float* const WB = smem + Cfg::A_WB;
    const int xt_own = ty * TX + tx, xt_down = xt_own + TX;  // exchange-array entries
    const int wb_own = (ty + 1) * TX + tx, wb_up = wb_own - TX;
    // w_h / p_h of the left neighbour's last column, theta of the right
    // neighbour's first column: adjacent lanes.  On the tile's left and right
    // edge the lane reads another value of this warp, which serves as well
    // as zero: those columns lie in the halo, whose values never reach the
    // interior within K updates.  Every lane of the CTA runs every shuffle:
    // the loop trip counts are uniform.
    auto from_left = [&](float v) { return __shfl_up_sync(0xffffffffu, v, 1); };
    auto from_right = [&](float v) { return __shfl_down_sync(0xffffffffu, v, 1); };

    // row / column flags (bit i: row r0 + i; bit j: column c0 + j)
    unsigned rin = 0, rv = 0, cin = 0, chm = 0;
#pragma unroll
    for (int i = 0; i < MR; ++i) {
        const int gi = gi_top + i;
        rin |= (unsigned)(gi >= 0 && gi < g.nx) << i;
        rv |= (unsigned)(gi >= 0 && gi < g.nx - 1) << i;
    }
#pragma unroll
    for (int j = 0; j < MC; ++j) {
        const int gj = gj_left + j;
        cin |= (unsigned)(gj >= 0 && gj < g.ny) << j;
        chm |= (unsigned)(gj >= 0 && gj < g.ny - 1) << j;
    }
    // Blocks whose rows all lie inside the image and above its last row -- the
    // same for every thread of a warp when a warp is one row of threads -- need
    // no masks: the column conditions fold into one horizontal step per
    // column, zero outside the image and on its last column, where w_h starts
    // at zero and so stays zero.  The vertical step needs no column factor:
    // outside the image theta and w_v stay exactly zero once w_h does.
    const bool rows_inner = rv == (1u << MR) - 1;
    float step_h[MC];
#pragma unroll
    for (int j = 0; j < MC; ++j) step_h[j] = ((chm >> j) & 1u) ? a.step : 0.f;
    auto in_ij = [&](int i, int j) { return ((rin >> i) & (cin >> j) & 1u) != 0; };
    auto own_ij = [&](int i, int j) {  // an interior slot of this tile, inside the image
        const int r = r0 + i, c = c0 + j;
        return in_ij(i, j) && r >= H && r < EH - H + 1 && c >= H && c < EW - H + 1;
    };
    auto gidx_of = [&](int i, int j) -> long long {
        return in_ij(i, j) ? fbase + (long long)(gi_top + i) * g.ny + gj_left + j : fbase;
    };

    float xr[MR][MC], ph[MR][MC], pv[MR][MC], wh[MR][MC], wv[MR][MC], th[MR][MC];
    float tv[CLIP ? MR : 1][CLIP ? MC : 1];  // Clip box: theta_v
    (void)tv;
    // The Clip box's p is its w: ph / pv stay unused there.
    float(&PH)[MR][MC] = *[&] { if constexpr (CLIP) return &wh; else return &ph; }();
    float(&PV)[MR][MC] = *[&] { if constexpr (CLIP) return &wv; else return &pv; }();

    // ---- loads for the whole extended tile, all issued before any is used ----
    const bool warm_first = a.first && a.warm;  // w from the previous TVdenoise, p = 0
    if (!a.first) {
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < MC; ++j) {
                const long long gi = gidx_of(i, j);
                if constexpr (!CLIP) {
                    ph[i][j] = ldraw<T>(p.st_in(0), gi);
                    pv[i][j] = ldraw<T>(p.st_in(1), gi);
                }
                wh[i][j] = ldraw<T>(p.st_in(2), gi);
                wv[i][j] = ldraw<T>(p.st_in(3), gi);
            }
    } else if (warm_first) {
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < MC; ++j) {
                const long long gi = gidx_of(i, j);
                wh[i][j] = ldraw<T>(p.warm_in(0), gi);
                wv[i][j] = ldraw<T>(p.warm_in(1), gi);
            }
    }
    if (a.mode == OuterMode::Prox) {
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < MC; ++j) xr[i][j] = __ldg(p.xin() + gidx_of(i, j));
    } else if (a.first) {
        uint32_t word[MR][MC];
        float rr[MR][MC];
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < MC; ++j) {
                const long long pix = gidx_of(i, j) - fbase;
                word[i][j] = __ldg(p.bits() + pix);
                rr[i][j] = __ldg(p.r() + pix);
                xr[i][j] = ldraw<T>(p.theta_in(), fbase + pix);
            }
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < MC; ++j)
                xr[i][j] = rt<T>(cvraw<T>(xr[i][j]) + mask_bit(word[i][j], bz) * rr[i][j]);
    } else {
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < MC; ++j) xr[i][j] = cvraw<T>(ldraw<T>(p.xt(), gidx_of(i, j)));
    }
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
        for (int j = 0; j < MC; ++j) {
            const bool in = in_ij(i, j);
            if (!a.first || warm_first) {
                if constexpr (!CLIP) {
                    ph[i][j] = cvraw<T>(ph[i][j]);
                    pv[i][j] = cvraw<T>(pv[i][j]);
                }
                wh[i][j] = cvraw<T>(wh[i][j]);
                wv[i][j] = cvraw<T>(wv[i][j]);
            }
            if (!in) xr[i][j] = 0.f;
            if constexpr (!CLIP) {
                if (a.first || !in) {
                    ph[i][j] = 0.f;
                    pv[i][j] = 0.f;
                }
            }
            if ((a.first && !a.warm) || !in) {
                wh[i][j] = 0.f;
                wv[i][j] = 0.f;
            }
        }

    // zero the pad rows (XT row TY, WB row 0), then publish w_v of the last row
    if (tid < TX) {
        const float zero[MC] = {};
        st4h<HALF>(XT, TY * TX + tid, zero);
        st4h<HALF>(WB, tid, zero);
    }
    {
        float vb[MC];
#pragma unroll
        for (int j = 0; j < MC; ++j) vb[j] = wv[MR - 1][j];
        st4h<HALF>(WB, wb_own, vb);
    }
    __syncthreads();

    const float lam = a.lambda, step = a.step;
    constexpr int kUnroll = CLIP ? 1 : 2;
#pragma unroll kUnroll
    for (int s = 0; s < a.K; ++s) {
        const bool skip_theta = a.first && !a.warm && s == 0;  // w = 0 there: theta = xt
        // ---- theta = xt - lambda (D^T w) ----
        {
            float wl[MR], wu[MC];
#pragma unroll
            for (int i = 0; i < MR; ++i) wl[i] = from_left(wh[i][MC - 1]);
            ld4h<HALF>(WB, wb_up, wu);
#pragma unroll
            for (int i = 0; i < MR; ++i)
#pragma unroll
                for (int j = 0; j < MC; ++j) {
                    float t = xr[i][j], v = xr[i][j];
                    if (!skip_theta) {
                        const float l = j > 0 ? wh[i][j > 0 ? j - 1 : 0] : wl[i];
                        const float u = i > 0 ? wv[i > 0 ? i - 1 : 0][j] : wu[j];
                        if constexpr (CLIP) {
                            t = __fmaf_rn(-lam, l - wh[i][j], xr[i][j]);
                            v = __fmaf_rn(-lam, u - wv[i][j], xr[i][j]);
                        } else {
                            t = __fmaf_rn(-lam, (l - wh[i][j]) + (u - wv[i][j]), xr[i][j]);
                        }
                    }
                    th[i][j] = t;
                    if constexpr (CLIP) tv[i][j] = v;
                }
            float vt[MC];
#pragma unroll
            for (int j = 0; j < MC; ++j) {
                if constexpr (CLIP) vt[j] = tv[0][j];
                else vt[j] = th[0][j];
            }
            st4h<HALF>(XT, xt_own, vt);
        }
        __syncthreads();
        // ---- a = w + step * D theta, projection, momentum ----
        const float c = a.coef[s];
        float tr[MR], td[MC];
#pragma unroll
        for (int i = 0; i < MR; ++i) tr[i] = from_right(th[i][0]);  // Clip: theta_h
        ld4h<HALF>(XT, xt_down, td);
        auto dual_step = [&](auto masked_c) {
            constexpr bool MASKED = decltype(masked_c)::value;
            // the flags pass through an empty asm each update, so the per-slot
            // tests are formed here rather than held in registers across the loop
            unsigned m_rin = rin, m_chm = chm, m_rv = rv, m_cin = cin;
            asm volatile("" : "+r"(m_rin), "+r"(m_chm), "+r"(m_rv), "+r"(m_cin));
#pragma unroll
            for (int i = 0; i < MR; ++i)
#pragma unroll
                for (int j = 0; j < MC; ++j) {
                    const float t0 = th[i][j];
                    const float trt = j < MC - 1 ? th[i][j < MC - 1 ? j + 1 : 0] : tr[i];
                    float dv;
                    if constexpr (CLIP) {
                        const float v0 = tv[i][j];
                        dv = (i < MR - 1 ? tv[i < MR - 1 ? i + 1 : 0][j] : td[j]) - v0;
                    } else {
                        dv = (i < MR - 1 ? th[i < MR - 1 ? i + 1 : 0][j] : td[j]) - t0;
                    }
                    float ah, av;
                    if constexpr (MASKED) {
                        const bool mh = ((m_rin >> i) & (m_chm >> j) & 1u) != 0;
                        const bool mv = ((m_rv >> i) & (m_cin >> j) & 1u) != 0;
                        ah = mh ? fmaf(trt - t0, step, wh[i][j]) : 0.f;
                        av = mv ? fmaf(dv, step, wv[i][j]) : 0.f;
                    } else {
                        ah = fmaf(trt - t0, step_h[j], wh[i][j]);
                        av = fmaf(dv, step, wv[i][j]);
                    }
                    if constexpr (TV == SCI_TV_ATV || CLIP) {
                        ah = fminf(fmaxf(ah, -1.f), 1.f);
                        av = fminf(fmaxf(av, -1.f), 1.f);
                    } else {
                        const float sc = fminf(1.f, rsqrt_ftz(fmaf(ah, ah, av * av)));
                        ah *= sc;
                        av *= sc;
                    }
                    if constexpr (CLIP) {
                        wh[i][j] = ah;
                        wv[i][j] = av;
                    } else {
                        wh[i][j] = fmaf(c, ah - ph[i][j], ah);
                        wv[i][j] = fmaf(c, av - pv[i][j], av);
                        ph[i][j] = ah;
                        pv[i][j] = av;
                    }
                }
        };
        if (rows_inner) dual_step(std::false_type{});
        else dual_step(std::true_type{});
        {
            float vb[MC];
#pragma unroll
            for (int j = 0; j < MC; ++j) vb[j] = wv[MR - 1][j];
            st4h<HALF>(WB, wb_own, vb);
        }
        __syncthreads();
    }

    // ---- epilogue ----
    // The interior's fields are written through shared memory: each block row
    // goes to a staging tile as one 16-byte word, and each warp then stores
    // whole runs of a tile row, where a thread's four adjacent columns would
    // fill a quarter of each 32-byte sector per store instruction.  Two
    // staging tiles alternate, so one barrier per field separates its writes
    // from the reads that drain it.
    constexpr int SW = Cfg::SW;
    const int lane = tid & 31, warp = tid >> 5;
    const int r_end = min(EH - H + 1, g.nx - gi0), c_end = min(EW - H + 1, g.ny - gj0);
    int stage = 0;
    auto put = [&](auto&& val, auto&& store) {
        float* const sb = smem + Cfg::A_ST + (stage & 1) * EH * SW;
        ++stage;
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < MC; j += 4)
                *reinterpret_cast<float4*>(sb + (r0 + i) * SW + c0 + j) =
                    make_float4(val(i, j), val(i, j + 1), val(i, j + 2), val(i, j + 3));
        __syncthreads();
        for (int r = H + warp; r < r_end; r += Cfg::NT / 32) {
            const long long row = fbase + (long long)(gi0 + r) * g.ny + gj0;
            for (int c = H + lane; c < c_end; c += 32) store(row + c, sb[r * SW + c]);
        }
    };
    auto st_T = [](T* dst) { return [dst](long long i, float v) { st<T>(dst, i, v); }; };
    auto st_f = [](float* dst) { return [dst](long long i, float v) { dst[i] = v; }; };
    if (!a.last) {
        // carry x-tilde (first launch of a solve), p and w of the interior
        if (a.first && a.mode != OuterMode::Prox) put([&](int i, int j) { return xr[i][j]; }, st_T(p.xt()));
        put([&](int i, int j) { return PH[i][j]; }, st_T(p.st_out(0)));
        put([&](int i, int j) { return PV[i][j]; }, st_T(p.st_out(1)));
        put([&](int i, int j) { return wh[i][j]; }, st_T(p.st_out(2)));
        put([&](int i, int j) { return wv[i][j]; }, st_T(p.st_out(3)));
        return;
    }
    // theta = xt - lambda D^T p reads p_h of the left neighbour (a shuffle)
    // and p_v of the row above: publish the block's last row of p where w_v
    // was (the loop ended with a barrier, and no one reads w_v any more).
    float pl[MR], pu[MC];
#pragma unroll
    for (int i = 0; i < MR; ++i) pl[i] = from_left(PH[i][MC - 1]);
    {
        float vb[MC];
#pragma unroll
        for (int j = 0; j < MC; ++j) vb[j] = PV[MR - 1][j];
        st4h<HALF>(WB, wb_own, vb);
    }
    // ADMM with x requested: x^(t+1) = xt - u^(t), u^(t) read (into the free
    // theta registers) before u^(t+1) overwrites it
    const bool want_xu = a.mode == OuterMode::Admm && p.x_out() != nullptr;
    if (want_xu) {
        // fresh copies of the block origin: these addresses are formed here
        // rather than kept live across the update loop
        int e_top = gi_top, e_left = gj_left;
        unsigned e_rin = rin, e_cin = cin;
        asm volatile("" : "+r"(e_top), "+r"(e_left), "+r"(e_rin), "+r"(e_cin));
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < MC; ++j) {
                const bool in = ((e_rin >> i) & (e_cin >> j) & 1u) != 0;
                th[i][j] = in ? ldg<T>(p.u_in(), fbase + (long long)(e_top + i) * g.ny + e_left + j) : 0.f;
            }
    }
    __syncthreads();
    ld4h<HALF>(WB, wb_up, pu);
    float tt[MR][MC];  // theta^(t+1)
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
        for (int j = 0; j < MC; ++j) {
            const float l = j > 0 ? PH[i][j > 0 ? j - 1 : 0] : pl[i];
            const float u = i > 0 ? PV[i > 0 ? i - 1 : 0][j] : pu[j];
            tt[i][j] = __fmaf_rn(-lam, (l - PH[i][j]) + (u - PV[i][j]), xr[i][j]);
        }
    if (a.mode == OuterMode::Prox) {
        put([&](int i, int j) { return tt[i][j]; }, st_f(p.theta_f32()));
        return;
    }
    put([&](int i, int j) { return tt[i][j]; }, st_T(p.theta_out()));
    if (a.mode == OuterMode::Gap) {
        if (p.x_out() != nullptr) put([&](int i, int j) { return xr[i][j]; }, st_f(p.x_out()));
    } else {
        put([&](int i, int j) { return xr[i][j] - rt<T>(tt[i][j]); }, st_T(p.u_out()));
        if (want_xu) put([&](int i, int j) { return xr[i][j] - th[i][j]; }, st_f(p.x_out()));
    }
    if (a.warm) {
        put([&](int i, int j) { return wh[i][j]; }, st_T(p.warm_out(0)));
        put([&](int i, int j) { return wv[i][j]; }, st_T(p.warm_out(1)));
    }
}

// A tile all of whose rows lie inside the image and above its last row runs
// the interior form; the others the border form.
template <typename T, int TV, class Cfg, class Prob>
__device__ __forceinline__ void fused_tile(const FusedArgs& a, const Prob& p, int bx, int by, int bz,
                                           float* smem) {
    if constexpr (Cfg::MICRO) {
        fused_tile_micro<T, TV, Cfg>(a, p, bx, by, bz, smem);
    } else if constexpr (Cfg::F == 1) {
        fused_tile_rows<T, TV, Cfg>(a, p, bx, by, bz, smem);
    } else {
        const Geo g = p.g();
        const int gi0 = by * fused_interior(Cfg::EH, a.halo) - a.halo;
        const bool border = !(gi0 >= 0 && gi0 + Cfg::EH - 1 < g.nx - 1);
        if constexpr (Cfg::SHFL) {
            if (!border) fused_tile_impl<T, TV, Cfg, false>(a, p, bx, by, bz, smem);
            else fused_tile_impl<T, TV, Cfg, true>(a, p, bx, by, bz, smem);
        } else {
            if (!border) fused_tile_blk<T, TV, Cfg, false>(a, p, bx, by, bz, smem);
            else fused_tile_blk<T, TV, Cfg, true>(a, p, bx, by, bz, smem);
        }
    }
}

// ---------------------------------------------------------------- configurations

// One-frame tiles update every row: idling a 16-row strip, or a warp of 4 x 4
// blocks whose rows can no longer reach an exact row, costs more than it
// saves (the test splits the two-update loop body the compiler interleaves).
// So do the 8- and 10-frame VTV tiles (measured 7-12% faster than skipping
// rows: every warp then reaches each barrier with the same work).  The 16-
// and 24-frame tiles skip such rows: updating every row measured slower for
// the first and spills for the second.
using CfgF1 = RowCfg<512, 16, 7>;    // 128 x 64 tile, one frame
using CfgF1s = RowCfg<256, 8, 6>;    // 64 x 32 tile, one frame (small images)
using CfgM1 = MicroCfg<512, 5, 4, 4>;   // 128 x 64 tile of 4 x 4 blocks, one frame
using CfgM1s = MicroCfg<256, 4, 2, 4>;  // 64 x 32 tile of 2 x 4 blocks, one frame
using CfgV8 = FusedCfg<512, 2, 8, 5, true, false>;     // 32 x 32 tile, up to 8 frames
using CfgV10 = FusedCfg<512, 2, 10, 5, false, false>;  // 32 x 32 tile, up to 10 frames
using CfgV16 = FusedCfg<512, 1, 16, 5, false, true>;   // 32 x 16 tile, up to 16 frames
using CfgV24 = BlkCfg<256, 2, 24, 5, false, true>;     // 32 x 16 tile, up to 24 frames

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

std::atomic<unsigned long long> g_attr_done[128];

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

// One "attribute set" flag word per (storage type, TV kernel code, configuration).
template <typename T>
constexpr int type_slot(int tv, int cfg) {
    return (std::is_same<T, float>::value ? 0 : (std::is_same<T, __half>::value ? 1 : 2)) * 32 + tv * 8 + cfg;
}

template <typename T, int TV>
bool launch_tv(const FusedArgs& a, const FusedBufs<T>& b, cudaStream_t s) {
    // if constexpr: each TV form instantiates only the tiles it can launch.
    // a.cls = 0: the library's class; otherwise the class asked for (checked
    // against the TV form and frame count by the caller).
    if constexpr (TV != SCI_TV_VTV) {
        // classes 1 and 3: 64 x 128 tiles (4 x 4 blocks / 16-row strips);
        // 2 and 4: 32 x 64 tiles (8-row strips / 2 x 4 blocks)
        if (a.cls == 3) return launch_cfg<T, TV, CfgF1>(type_slot<T>(TV, 0), a, b, s);
        if (a.cls == 4) return launch_cfg<T, TV, CfgM1s>(type_slot<T>(TV, 7), a, b, s);
        const bool small = a.cls == 2 ||
                           (a.cls == 0 && a.halo <= 8 && (long long)a.g.nx * a.g.ny < 192LL * 192);
        if (small) return launch_cfg<T, TV, CfgF1s>(type_slot<T>(TV, 1), a, b, s);
        return launch_cfg<T, TV, CfgM1>(type_slot<T>(TV, 6), a, b, s);
    } else {
        const int c = a.cls != 0 ? a.cls : fused_class(SCI_TV_VTV, a.g.B);
        switch (c) {
            case 8: return launch_cfg<T, TV, CfgV8>(type_slot<T>(TV, 2), a, b, s);
            case 10: return launch_cfg<T, TV, CfgV10>(type_slot<T>(TV, 3), a, b, s);
            case 16: return launch_cfg<T, TV, CfgV16>(type_slot<T>(TV, 4), a, b, s);
            case 24: return launch_cfg<T, TV, CfgV24>(type_slot<T>(TV, 5), a, b, s);
            default: return false;
        }
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

bool fused_class_fits(int tv, int B, int cls) {
    if (tv != SCI_TV_VTV) return cls >= 1 && cls <= 4;
    return (cls == 8 || cls == 10 || cls == 16 || cls == 24) && B <= cls;
}

int fused_class_max_halo(int cls) {
    switch (cls) {
        case 1: case 3: return 20;    // 64 x 128 one-frame tiles
        case 2: case 4: return 12;    // 32 x 64 one-frame tiles
        case 8: case 10: return 8;    // 32 x 32 VTV tiles
        case 16: case 24: return 4;   // 32 x 16 VTV tiles
        default: return 0;
    }
}

void fused_class_dims(int cls, int* EH, int* EW) {
    int h = 0, w = 0;
    switch (cls) {
        case 1: dims_of<CfgM1>(h, w); break;
        case 2: dims_of<CfgF1s>(h, w); break;
        case 3: dims_of<CfgF1>(h, w); break;
        case 4: dims_of<CfgM1s>(h, w); break;
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
std::atomic<unsigned long long> g_battr_done[128];

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
        return launch_batched_cfg<T, TV, CfgM1>(type_slot<T>(TV, 6), a, items, nitems, total, tpar, spar, want_x,
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
        case kTvClip: return launch_tv<T, kTvClip>(a, b, s);
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
