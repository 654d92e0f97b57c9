// 3x3x3 convolution with 32 input and 32 output channels on the 5th-generation
// tensor cores (tcgen05), BF16 operands, FP32 accumulation in tensor memory.
// Used by the learned TV prox (its two hidden 32->32 layers, forward and
// input-gradient passes).
//
// Implicit GEMM with the three column taps side by side.  A tile covers 4
// rows x 30 output columns of one frame of one volume.  Its A operand is a
// 128-voxel window (4 rows x 32 columns, starting one column left of the
// tile) of the channels-last activations [volume][frame][row][column]
// [channel], taken from TMA boxes of a 5-D tensor map -- one 6-row box per dz
// serves the three dy windows (rows 2 KB apart); out-of-range voxels arrive
// as zeros, which is the convolution's zero padding.  Its B operand for a
// (dz, dy) pair is the 96 x 32 block of the three dx taps' weights (output
// channel blocks for dx = -1, 0, +1), resident in shared memory for the whole
// kernel.  Two tcgen05.mma (M = 128, N = 96, K = 16) per (dz, dy) accumulate
// G_dx[v][c] = sum over dz, dy of act[v + (dz, dy)] . W[dz, dy, dx][c] in a
// 128-lane x 96-column FP32 tile of tensor memory, and the epilogue forms
// out[x] = G_-1[x - 1] + G_0[x] + G_+1[x + 1] with two warp shuffles per
// channel (a warp holds one row of the window).  Eighteen N = 96 MMAs replace
// 54 N = 32 ones per tile: with 32 output channels the MMA issue rate, not
// the tensor datapath, bounds the narrow form.
//
// Warp-specialised and persistent: each CTA walks whole columns of tiles
// (one row block and column block of a volume) frame by frame, so each
// frame's box, loaded once, serves the three tiles that read it; one lane
// issues TMA loads into a ring of A stages, one lane issues the MMAs (a
// commit frees a frame's stage once its last tile is issued), and four
// warps read the double-buffered accumulator with tcgen05.ld (warp w owns
// lanes 32w..32w+31, i.e. voxels 32w..32w+31 of the tile) and apply the
// epilogue while the next tile accumulates.  Every mbarrier wait is
// bounded: on timeout the kernel records an error code, stops issuing work,
// drains what it issued, frees its tensor memory and returns.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "sci_internal.cuh"

namespace sci {

namespace {

constexpr int kStages = 4;
constexpr int kTileM = 128;
constexpr int kC = 32;
// A stage: one TMA box of 32 columns x 6 rows (the tile's 4 rows plus one
// above and one below) of one frame; the three row taps (dy = -1, 0, +1) of a
// (dz, dx) pair are 128-row windows of it starting 32 rows (2 KB) apart, which
// keeps every window aligned to the 512-byte period of the 64-byte swizzle.
constexpr int kBW = 32, kBH = 4;                             // A window: 4 rows x 32 columns
constexpr int kOutW = kBW - 2;                               // output columns per tile
constexpr int kN = 3 * kC;                                   // MMA N: three dx taps x 32 channels
constexpr uint32_t kAccCols = 128;                           // tensor-memory columns per accumulator
constexpr uint32_t kRowBytes = kC * 2;                       // 64 B per voxel
constexpr uint32_t kABytes = kBW * (kBH + 2) * kRowBytes;    // 12 KB per A stage
constexpr uint32_t kWTapBytes = kC * kC * 2;       // 2 KB per tap
constexpr uint32_t kWBytes = 27 * kWTapBytes;      // 54 KB
// The 32 -> 1 output layer runs the same kernel with N = 16: one 16-row
// weight block per (dz, dy) pair holds output channel 0 of its three dx taps
// (rows 0-2) and zeros (rows 3-15), so an MMA computes G_-1, G_0, G_+1 of that
// channel in accumulator columns 0-2 (an N = 96 form would carry 31 zero
// channels per tap).
constexpr int kN1 = 16;
constexpr uint32_t kW1PairBytes = kN1 * kC * 2;    // 1 KB per (dz, dy) pair
constexpr uint32_t kW1Bytes = 9 * kW1PairBytes;    // 9 KB
template <int NN> constexpr uint32_t w_bytes() { return NN == kN ? kWBytes : kW1Bytes; }
constexpr long long kSpinLimit = 1LL << 26;        // bounded mbarrier waits

// ---- PTX helpers --------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Wait for the phase with the given parity; false if the spin limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < kSpinLimit; ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6, "
        "%7}], [%2];" ::"r"(dst),
        "l"(map), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(dst),
        "l"(map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// K-major operand in the 64-byte swizzled layout (rows of 32 BF16 = 64 B,
// 8-row groups 512 B apart), as written by TMA with 64-byte swizzling.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)(16u >> 4) << 16;           // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(512u >> 4) << 32;          // stride byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)4 << 61;                    // layout: 64-byte swizzle
    return d;
}

// kind::f16 instruction descriptor: D = FP32, A = B = BF16, both K-major, M = 128, N = NN.
template <int NN>
constexpr uint32_t idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NN >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

template <int NN>
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc<NN>()), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld_32cols(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct ConvTcArgs {
    int nvol, D, H, W;      // volumes and their frames x rows x columns
    int BW, BH;             // tile: BH rows x BW output columns
    int tiles_w, tiles_h;   // tiles per row block / per frame
    long long ntiles;
    int mode;               // ConvEpilogue
    const float* bias;      // [32] (forward)
    const __nv_bfloat16* mask_act;  // input-gradient mode: zero where this activation is <= 0
    __nv_bfloat16* out;     // [nvol][D][H][W][32]
    const float* xres;      // mode 3: residual input x [nvol][D][H][W]
    float* out1;            // mode 3: x + bias + output channel 0, FP32 [nvol][D][H][W]
    int* err;               // set to 1 on a wait timeout
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Warp roles: warps 0-3 run the epilogue (warp w reads tensor-memory lanes
// 32w..32w+31, i.e. window row w); lane 0 of warp 4 issues the TMA loads;
// lane 0 of warp 5 issues the MMAs.  The accumulator is double buffered in
// tensor memory (2 x 128 columns, 96 used), so the epilogue of tile j
// overlaps the MMAs of tile j + 1 and the loads run ahead across tiles.
constexpr int kThreads = 192;

template <int NN>
__global__ void __launch_bounds__(kThreads, 1)
k_conv3d_c32_tc(const __grid_constant__ CUtensorMap act_map, const __grid_constant__ CUtensorMap w_map,
                ConvTcArgs a) {
    static_assert(NN == kN || NN == kN1, "the 32-channel form or the one-channel output form");
    extern __shared__ __align__(1024) unsigned char dsmem[];
    unsigned char* base = (unsigned char*)(((uintptr_t)dsmem + 1023) & ~(uintptr_t)1023);
    unsigned char* s_w = base;                        // 27 x 2 KB weights
    unsigned char* s_a = base + w_bytes<NN>();        // kStages x 12 KB A ring
    uint64_t* bars = reinterpret_cast<uint64_t*>(s_a + kStages * kABytes);
    // bars: full[kStages], empty[kStages], acc_full[2], acc_empty[2], weights, drain
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 6);
    volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar_full = smem_u32(bars), bar_empty = smem_u32(bars + kStages);
    const uint32_t bar_accf = smem_u32(bars + 2 * kStages), bar_acce = smem_u32(bars + 2 * kStages + 2);
    const uint32_t bar_w = smem_u32(bars + 2 * kStages + 4), bar_drain = smem_u32(bars + 2 * kStages + 5);

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_accf + 8 * b, 1);
            mbar_init(bar_acce + 8 * b, 4);  // one arrival per epilogue warp
        }
        mbar_init(bar_w, 1);
        mbar_init(bar_drain, 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;
    // Each CTA walks whole columns of tiles -- (volume, row block, column
    // block) -- frame by frame, so a frame's activation box serves the three
    // tiles (frames z - 1, z, z + 1) that read it: a column of D tiles loads
    // D + 2 boxes (frames -1 and D arrive as zeros) where tile by tile it
    // would load 3 D.  Ring slot q holds the column's frame q - q0 - 1.
    const long long ncols = (long long)a.nvol * a.tiles_h * a.tiles_w;
    const long long my_cols = ncols > blockIdx.x ? (ncols - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long my_tiles = my_cols * a.D;
    auto column = [&](long long cj, int& tw, int& th, int& vol) {
        long long c = blockIdx.x + cj * gridDim.x;
        tw = (int)(c % a.tiles_w);
        c /= a.tiles_w;
        th = (int)(c % a.tiles_h);
        vol = (int)(c / a.tiles_h);
    };

    if (warp == 4 && lane == 0) {
        // ---------------- TMA producer ----------------
        mbar_expect_tx(bar_w, w_bytes<NN>());
        if constexpr (NN == kN) {
            for (int t = 0; t < 27; ++t) tma_load_3d(smem_u32(s_w + t * kWTapBytes), &w_map, bar_w, 0, 0, t);
        } else {
            for (int t = 0; t < 9; ++t) tma_load_3d(smem_u32(s_w + t * kW1PairBytes), &w_map, bar_w, 0, 0, t);
        }
        uint32_t q = 0;
        for (long long cj = 0; cj < my_cols && !*s_abort; ++cj) {
            int tw, th, vol;
            column(cj, tw, th, vol);
            const int w0 = tw * a.BW, h0 = th * a.BH;
            bool ok = true;
            for (int f = -1; f <= a.D; ++f, ++q) {  // the column's frames, with a zero frame at each end
                const uint32_t s = q % kStages, use = q / kStages;
                if (use > 0 && !mbar_wait(bar_empty + 8 * s, (use - 1) & 1)) { ok = false; break; }
                mbar_expect_tx(bar_full + 8 * s, kABytes);
                tma_load_5d(smem_u32(s_a + s * kABytes), &act_map, bar_full + 8 * s, 0, w0 - 1, h0 - 1, f, vol);
            }
            if (!ok) { *s_abort = 1; atomicExch(a.err, 1); break; }
        }
        // drain: every load issued must have landed before the CTA exits
        for (uint32_t k = (q >= kStages ? q - kStages : 0); k < q; ++k)
            mbar_wait(bar_full + 8 * (k % kStages), (k / kStages) & 1);
    }
    if (warp == 5 && lane == 0) {
        // ---------------- MMA issuer ----------------
        bool ok = mbar_wait(bar_w, 0);
        uint32_t q0 = 0;  // ring index of the current column's frame -1
        long long j = 0;  // tiles issued (the accumulator buffers alternate)
        for (long long cj = 0; cj < my_cols && ok && !*s_abort; ++cj) {
        for (int z = 0; z < a.D; ++z, ++j) {
            const uint32_t b = (uint32_t)(j & 1), use_b = (uint32_t)(j >> 1);
            if (use_b > 0 && !mbar_wait(bar_acce + 8 * b, (use_b - 1) & 1)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t d = tmem + b * kAccCols;
            for (int k = 0; k < 3; ++k) {  // dz = k - 1: frame z + k - 1, ring index q0 + z + k
                const uint32_t q = q0 + (uint32_t)(z + k);
                const uint32_t s = q % kStages, use = q / kStages;
                // each frame is waited for once, by the first tile that reads it
                if ((z == 0 || k == 2) && !mbar_wait(bar_full + 8 * s, use & 1)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int dyi = 0; dyi < 3; ++dyi) {
                    // taps (dz, dy, dx = -1..+1) are consecutive 2 KB blocks: one N = 96
                    // operand (N = 16: the pair's 1 KB block)
                    const int t = k * 9 + dyi * 3;
                    const uint32_t abase = smem_u32(s_a + s * kABytes) + (uint32_t)dyi * kBW * kRowBytes;
                    const uint32_t bbase = NN == kN ? smem_u32(s_w + t * kWTapBytes)
                                                    : smem_u32(s_w + (k * 3 + dyi) * kW1PairBytes);
                    umma_bf16<NN>(d, smem_desc_sw64(abase), smem_desc_sw64(bbase), (k > 0 || dyi > 0) ? 1u : 0u);
                    umma_bf16<NN>(d, smem_desc_sw64(abase + 32), smem_desc_sw64(bbase + 32), 1u);
                }
            }
            if (!ok) break;
            umma_commit(bar_accf + 8 * b);
            umma_commit(bar_empty + 8 * ((q0 + (uint32_t)z) % kStages));  // frame z - 1 is read no more
        }
        if (!ok) break;
        // the column's last two frames
        umma_commit(bar_empty + 8 * ((q0 + (uint32_t)a.D) % kStages));
        umma_commit(bar_empty + 8 * ((q0 + (uint32_t)a.D + 1) % kStages));
        q0 += (uint32_t)a.D + 2;
        }
        if (!ok) {
            // every MMA issued so far must finish before tensor memory is freed
            umma_commit(bar_drain);
            mbar_wait(bar_drain, 0);
            *s_abort = 1;
            atomicExch(a.err, 1);
        }
    }
    if (warp < 4) {
        // ---------------- epilogue ----------------
        for (long long j = 0; j < my_tiles; ++j) {
            const uint32_t b = (uint32_t)(j & 1), use_b = (uint32_t)(j >> 1);
            const bool got = __all_sync(0xffffffffu, mbar_wait(bar_accf + 8 * b, use_b & 1));
            if (!got) {
                if (lane == 0) { *s_abort = 1; atomicExch(a.err, 1); }
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // lane x of warp w holds window voxel (row w, column x); the output
            // at tile column i = x is G_-1[x] + G_0[x + 1] + G_+1[x + 2]
            float v[32], g[32];
            const uint32_t lanes = (uint32_t)(warp * 32) << 16;
            const bool one = a.mode == 3;  // only output channel 0 is used
            tmem_ld_32cols(tmem + b * kAccCols + lanes, v);
            if constexpr (NN == kN1) {
                // columns 0-2: G_-1, G_0, G_+1 of output channel 0
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_acce + 8 * b);
                v[0] += __shfl_down_sync(0xffffffffu, v[1], 1);
                v[0] += __shfl_down_sync(0xffffffffu, v[2], 2);
            } else {
            tmem_ld_32cols(tmem + b * kAccCols + 32 + lanes, g);
            if (one) {
                v[0] += __shfl_down_sync(0xffffffffu, g[0], 1);
            } else {
#pragma unroll
                for (int c = 0; c < 32; ++c) v[c] += __shfl_down_sync(0xffffffffu, g[c], 1);
            }
            tmem_ld_32cols(tmem + b * kAccCols + 64 + lanes, g);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_acce + 8 * b);  // this warp's lanes of buffer b are free
            if (one) {
                v[0] += __shfl_down_sync(0xffffffffu, g[0], 2);
            } else {
#pragma unroll
                for (int c = 0; c < 32; ++c) v[c] += __shfl_down_sync(0xffffffffu, g[c], 2);
            }
            }
            int tw, th, vol;
            column(j / a.D, tw, th, vol);
            const int z = (int)(j % a.D);
            const int hh = th * a.BH + warp, ww = tw * a.BW + lane;
            if (lane < kOutW && hh < a.H && ww < a.W) {
                const long long vox = (((long long)vol * a.D + z) * a.H + hh) * a.W + ww;
                if (one) {  // 32 -> 1 output layer: theta = x + (bias + f)
                    a.out1[vox] = a.xres[vox] + (v[0] + a.bias[0]);
                    continue;
                }
                __nv_bfloat16* dst = a.out + vox * kC;
                if (a.mode == 0) {  // forward: bias + ReLU
#pragma unroll
                    for (int c = 0; c < 32; ++c) v[c] = fmaxf(v[c] + a.bias[c], 0.f);
                } else if (a.mode == 1) {  // input gradient masked by the activation's ReLU
                    const __nv_bfloat16* m = a.mask_act + vox * kC;
#pragma unroll
                    for (int c = 0; c < 32; ++c) v[c] = __bfloat162float(m[c]) > 0.f ? v[c] : 0.f;
                }
                uint4 pk[4];
                uint32_t* pw = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * c], v[2 * c + 1]);
                    pw[c] = *reinterpret_cast<uint32_t*>(&h2);
                }
                uint4* d4 = reinterpret_cast<uint4*>(dst);
#pragma unroll
                for (int c = 0; c < 4; ++c) d4[c] = pk[c];
            }
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 5) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
    }
}

// ---- weight gradients of a 32 -> 32 layer --------------------------------
// dW[(dz, dy, dx)][o][i] = sum_v g[v][o] act[v + (dz, dy, dx)][i] is, with
// u = v + dx along the row, sum_u g[u - dx][o] act[u + (dz, dy)][i]: a GEMM
// over voxels, K-major in both operands once the fields are transposed so a
// row's voxels are contiguous per channel (actT[row][c][x], and three copies
// of gT shifted by dx = -1, 0, +1).  A tile is 32 voxels of one row (K = 32,
// two MMAs of K = 16).  Operand A stacks four (dz, dy) pairs' 32-channel x
// 32-voxel TMA boxes (M = 128), B the three shifted gradient boxes (N = 96,
// rows (dx, o)), in the same 64-byte-swizzled K-major layout as the forward
// pass.  Pairs 0-3, 4-7 and 8 make three accumulators; the fourth block of
// the last group holds ones, so its rows give sum_u gT[o][u] (the bias
// gradient, from the dx = 0 copy).  Each CTA walks its tiles and writes its
// totals to its own slot (27 x 32 x 32 weights, then 32 biases), which a
// fixed-order reduction adds up.
constexpr int kWgStages = 7;
constexpr uint32_t kWgBox = 32 * 32 * 2;                  // 2 KB: 32 rows x 64 B
constexpr uint32_t kWgABytes = 12 * kWgBox;               // three groups of four blocks
constexpr uint32_t kWgStage = kWgABytes + 3 * kWgBox;     // + the three B boxes: 30 KB
constexpr uint32_t kWgTx = 12 * kWgBox;                   // loaded per tile: 9 A + 3 B boxes
constexpr int kWgSlotLen = 27 * kC * kC + kC;

struct WgradTcArgs {
    int nvol, D, H, tiles_x;  // rows nvol x D x H of 32 tiles_x (padded) voxels
    long long ntiles;
    float* part;              // [gridDim.x][kWgSlotLen]
    int* err;
};

__global__ void __launch_bounds__(kThreads, 1)
k_wgrad_c32_tc(const __grid_constant__ CUtensorMap a_map, const __grid_constant__ CUtensorMap g_map,
               WgradTcArgs a) {
    extern __shared__ __align__(1024) unsigned char dsmem[];
    unsigned char* base = (unsigned char*)(((uintptr_t)dsmem + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + kWgStages * kWgStage);
    // bars: full[kWgStages], empty[kWgStages], acc_full, drain
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 2 * kWgStages + 2);
    volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar_full = smem_u32(bars), bar_empty = smem_u32(bars + kWgStages);
    const uint32_t bar_acc = smem_u32(bars + 2 * kWgStages), bar_drain = smem_u32(bars + 2 * kWgStages + 1);

    if (tid == 0) {
        for (int s = 0; s < kWgStages; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        mbar_init(bar_acc, 1);
        mbar_init(bar_drain, 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // blocks 9-11 of every stage are never loaded: 9 holds BF16 ones (rows of
    // equal values, which the swizzle leaves unchanged), 10 and 11 zeros
    for (int e = tid; e < kWgStages * 3 * (int)(kWgBox / 4); e += kThreads) {
        const int st = e / (3 * (kWgBox / 4)), w = e % (3 * (kWgBox / 4));
        uint32_t* blk = reinterpret_cast<uint32_t*>(base + st * kWgStage + 9 * kWgBox);
        blk[w] = w < (int)(kWgBox / 4) ? 0x3F803F80u : 0u;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes, read by the MMAs
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;
    const long long my_tiles = a.ntiles > blockIdx.x ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == 4 && lane == 0) {
        // ---------------- TMA producer ----------------
        long long j = 0;
        for (; j < my_tiles && !*s_abort; ++j) {
            long long tr = blockIdx.x + j * gridDim.x;
            const int tx = (int)(tr % a.tiles_x); tr /= a.tiles_x;
            const int y = (int)(tr % a.H); tr /= a.H;
            const int z = (int)(tr % a.D), vol = (int)(tr / a.D);
            const uint32_t s = (uint32_t)(j % kWgStages), use = (uint32_t)(j / kWgStages);
            if (use > 0 && !mbar_wait(bar_empty + 8 * s, (use - 1) & 1)) {
                *s_abort = 1;
                atomicExch(a.err, 1);
                break;
            }
            const uint32_t st = smem_u32(base + s * kWgStage);
            mbar_expect_tx(bar_full + 8 * s, kWgTx);
            for (int p = 0; p < 9; ++p)  // pair (dz, dy) = (p / 3 - 1, p % 3 - 1)
                tma_load_5d(st + p * kWgBox, &a_map, bar_full + 8 * s, tx * 32, 0, y + p % 3 - 1, z + p / 3 - 1, vol);
            for (int c = 0; c < 3; ++c)  // dx = c - 1
                tma_load_5d(st + kWgABytes + c * kWgBox, &g_map, bar_full + 8 * s, tx * 32, 0, y, z,
                            c * a.nvol + vol);
        }
        // drain: every load issued must have landed before the CTA exits
        for (long long k = (j >= kWgStages ? j - kWgStages : 0); k < j; ++k)
            mbar_wait(bar_full + 8 * (uint32_t)(k % kWgStages), (uint32_t)(k / kWgStages) & 1);
    }
    if (warp == 5 && lane == 0) {
        // ---------------- MMA issuer ----------------
        bool ok = true;
        for (long long j = 0; j < my_tiles && !*s_abort; ++j) {
            const uint32_t s = (uint32_t)(j % kWgStages), use = (uint32_t)(j / kWgStages);
            if (!mbar_wait(bar_full + 8 * s, use & 1)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = smem_u32(base + s * kWgStage);
#pragma unroll
            for (int grp = 0; grp < 3; ++grp)
#pragma unroll
                for (int kk = 0; kk < 2; ++kk)
                    umma_bf16<kN>(tmem + grp * 128, smem_desc_sw64(st + grp * 4 * kWgBox + kk * 32),
                                  smem_desc_sw64(st + kWgABytes + kk * 32), (j > 0 || kk > 0) ? 1u : 0u);
            umma_commit(bar_empty + 8 * s);
        }
        if (!ok) {
            // every MMA issued so far must finish before tensor memory is freed
            umma_commit(bar_drain);
            mbar_wait(bar_drain, 0);
            *s_abort = 1;
            atomicExch(a.err, 1);
        }
        umma_commit(bar_acc);
    }
    if (warp < 4) {
        // ---------------- epilogue: this CTA's totals ----------------
        const bool got = __all_sync(0xffffffffu, mbar_wait(bar_acc, 0));
        if (got && !*s_abort) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float* dst = a.part + (size_t)blockIdx.x * kWgSlotLen;
            const uint32_t lanes = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
            for (int grp = 0; grp < 3; ++grp) {
                const int blk = grp * 4 + warp;  // this warp's lanes: rows (blk, i = lane)
#pragma unroll 1
                for (int c = 0; c < 3; ++c) {
                    float v[32];
                    tmem_ld_32cols(tmem + grp * 128 + c * 32 + lanes, v);  // v[o]: dx = c - 1
                    if (blk < 9) {
                        const int tap = blk * 3 + c;
#pragma unroll
                        for (int o = 0; o < 32; ++o) dst[(tap * kC + o) * kC + lane] = v[o];
                    } else if (blk == 9 && c == 1 && lane == 0) {
#pragma unroll
                        for (int o = 0; o < 32; ++o) dst[27 * kC * kC + o] = v[o];
                    }
                }
            }
        } else if (lane == 0) {
            *s_abort = 1;
            atomicExch(a.err, 1);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 5) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

// ---- host: tensor maps ---------------------------------------------------
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        // the entry point as introduced with CUDA 12.0
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    return fn;
}

}  // namespace

// 2 CTAs per SM (the N = 96 form)
template <int NN>
size_t conv_smem() { return w_bytes<NN>() + kStages * kABytes + 1024 + 256; }

namespace {

template <int NN>
bool launch_conv(const __nv_bfloat16* act, const __nv_bfloat16* w, ConvTcArgs a, cudaStream_t s) {
    EncodeFn enc = encode_fn();
    if (enc == nullptr) return false;
    const int nvol = a.nvol, D = a.D, H = a.H, W = a.W;
    a.BW = kOutW;
    a.BH = kBH;
    a.tiles_w = (W + a.BW - 1) / a.BW;
    a.tiles_h = (H + a.BH - 1) / a.BH;
    a.ntiles = (long long)nvol * D * a.tiles_h * a.tiles_w;
    if (((uintptr_t)act & 15) != 0 || ((uintptr_t)w & 15) != 0) return false;

    CUtensorMap amap, wmap;
    std::memset(&amap, 0, sizeof(amap));
    std::memset(&wmap, 0, sizeof(wmap));
    const cuuint64_t adims[5] = {(cuuint64_t)kC, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)nvol};
    const cuuint64_t astr[4] = {(cuuint64_t)kC * 2, (cuuint64_t)W * kC * 2, (cuuint64_t)H * W * kC * 2,
                                (cuuint64_t)D * H * W * kC * 2};
    const cuuint32_t abox[5] = {(cuuint32_t)kC, (cuuint32_t)kBW, (cuuint32_t)(kBH + 2), 1, 1};
    const cuuint32_t ones[5] = {1, 1, 1, 1, 1};
    if (enc(&amap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16*>(act), adims, astr, abox, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    // weights: [27][32 out][32 in] (N = 96), or [9][16][32] (N = 16: the one-channel layer)
    const cuuint32_t wrows = NN == kN ? (cuuint32_t)kC : (cuuint32_t)kN1;
    const cuuint64_t wdims[3] = {(cuuint64_t)kC, (cuuint64_t)wrows, NN == kN ? 27u : 9u};
    const cuuint64_t wstr[2] = {(cuuint64_t)kC * 2, (cuuint64_t)wrows * kC * 2};
    const cuuint32_t wbox[3] = {(cuuint32_t)kC, wrows, 1};
    if (enc(&wmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(w), wdims, wstr, wbox, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;

    static bool attr = false;
    const size_t smem = conv_smem<NN>();
    if (!attr) {
        if (cudaFuncSetAttribute(k_conv3d_c32_tc<NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return false;
        attr = true;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long ncols = a.ntiles / a.D;  // columns of tiles, each walked by one CTA
    const long long grid = std::max(1LL, std::min<long long>(ncols, (long long)sms * 2));
    k_conv3d_c32_tc<NN><<<(unsigned)grid, kThreads, smem, s>>>(amap, wmap, a);
    return true;
}

bool launch_wgrad(const __nv_bfloat16* actT, const __nv_bfloat16* gT, int nvol, int D, int H, int Wp, float* part,
                  int max_slots, int* err, int* nslots, cudaStream_t s) {
    EncodeFn enc = encode_fn();
    if (enc == nullptr || Wp % 32 != 0 || max_slots < 1) return false;
    if (((uintptr_t)actT & 15) != 0 || ((uintptr_t)gT & 15) != 0) return false;
    CUtensorMap amap, gmap;
    std::memset(&amap, 0, sizeof(amap));
    std::memset(&gmap, 0, sizeof(gmap));
    // [vol][z][y][c][x] with x contiguous; the gradient's three shifted copies stack along vol
    const cuuint64_t row = (cuuint64_t)Wp * 2;
    const cuuint64_t str[4] = {row, row * kC, row * kC * H, row * kC * H * D};
    const cuuint32_t box[5] = {32, (cuuint32_t)kC, 1, 1, 1};
    const cuuint32_t ones[5] = {1, 1, 1, 1, 1};
    const cuuint64_t adims[5] = {(cuuint64_t)Wp, (cuuint64_t)kC, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)nvol};
    const cuuint64_t gdims[5] = {(cuuint64_t)Wp, (cuuint64_t)kC, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)3 * nvol};
    if (enc(&amap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16*>(actT), adims, str, box, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    if (enc(&gmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16*>(gT), gdims, str, box, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    WgradTcArgs a{};
    a.nvol = nvol;
    a.D = D;
    a.H = H;
    a.tiles_x = Wp / 32;
    a.ntiles = (long long)nvol * D * H * a.tiles_x;
    a.part = part;
    a.err = err;
    static bool attr = false;
    const size_t smem = (size_t)kWgStages * kWgStage + 1024 + 256;  // one CTA per SM (512 tensor-memory columns)
    if (!attr) {
        if (cudaFuncSetAttribute(k_wgrad_c32_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return false;
        attr = true;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // every CTA gets at least one tile (its accumulators start with its first MMA)
    const long long grid = std::min<long long>({a.ntiles, (long long)sms, (long long)max_slots});
    if (grid < 1) return false;
    k_wgrad_c32_tc<<<(unsigned)grid, kThreads, smem, s>>>(amap, gmap, a);
    *nslots = (int)grid;
    return true;
}

}  // namespace

// out[vol][z][h][w][:] = epilogue(sum_tap W[tap] * act[vol][z+dz][h+dy][w+dx][:]).
// act, out: BF16 [nvol][D][H][W][32]; w: BF16 [27][32 out][32 in].
// mode 0: + bias, ReLU; mode 1: x (mask_act > 0); mode 2: plain.
bool launch_conv3d_c32_tc(const __nv_bfloat16* act, const __nv_bfloat16* w, const float* bias,
                          const __nv_bfloat16* mask_act, int mode, int nvol, int D, int H, int W,
                          __nv_bfloat16* out, int* err, cudaStream_t s) {
    ConvTcArgs a{};
    a.nvol = nvol;
    a.D = D;
    a.H = H;
    a.W = W;
    a.mode = mode;
    a.bias = bias;
    a.mask_act = mask_act;
    a.out = out;
    a.err = err;
    return launch_conv<kN>(act, w, a, s);
}

// The 32 -> 1 output layer with the residual: theta = x + bias[0] + sum_tap
// W[tap][0] . act[voxel + tap], on the same tensor-core kernel at N = 16
// (w: BF16 [9][16][32], block (dz, dy) = rows dx + 1 for dx = -1..+1 holding
// W[(dz, dy, dx)][0][:], rows 3-15 zero); x, theta: FP32 [nvol][D][H][W].
bool launch_conv3d_c32_to1_tc(const __nv_bfloat16* act, const __nv_bfloat16* w, const float* bias, const float* x,
                              float* theta, int nvol, int D, int H, int W, int* err, cudaStream_t s) {
    ConvTcArgs a{};
    a.nvol = nvol;
    a.D = D;
    a.H = H;
    a.W = W;
    a.mode = 3;
    a.bias = bias;
    a.xres = x;
    a.out1 = theta;
    a.err = err;
    return launch_conv<kN1>(act, w, a, s);
}

// Weight and bias gradients of a 32 -> 32 layer on the tensor cores, per-CTA
// totals: actT [nvol][D][H][32][Wp] (the layer's input, transposed per row),
// gT [3][nvol][D][H][32][Wp] (its output gradient, transposed per row and
// shifted by dx = -1, 0, +1: gT[c][..][o][x] = g[..][x - (c - 1)][o], zero
// outside the row); Wp a multiple of 32.  Slot b of part (at most max_slots)
// receives dW[27][32 o][32 i] then db[32]; *nslots the number written.
bool launch_wgrad_c32_tc(const __nv_bfloat16* actT, const __nv_bfloat16* gT, int nvol, int D, int H, int Wp,
                         float* part, int max_slots, int* err, int* nslots, cudaStream_t s) {
    return launch_wgrad(actT, gT, nvol, D, H, Wp, part, max_slots, err, nslots, s);
}

}  // namespace sci

extern "C" sci_status sci_conv3d_c32_bf16(const void* act, const void* w, const float* bias, int relu, int nvol,
                                          int D, int H, int W, void* out, int* err, sci_stream_t stream) {
    if (act == nullptr || w == nullptr || out == nullptr || err == nullptr || act == out) return SCI_ERR_ARG;
    if (nvol <= 0 || D <= 0 || H <= 0 || W <= 0 || (relu && bias == nullptr)) return SCI_ERR_ARG;
    if ((double)nvol * D * H * W > 2.0e9) return SCI_ERR_SHAPE;
    if (!sci::launch_conv3d_c32_tc(static_cast<const __nv_bfloat16*>(act), static_cast<const __nv_bfloat16*>(w),
                                   bias, nullptr, relu ? 0 : 2, nvol, D, H, W, static_cast<__nv_bfloat16*>(out), err,
                                   (cudaStream_t)stream))
        return SCI_ERR_CUDA;
    return sci::check_launch();
}
