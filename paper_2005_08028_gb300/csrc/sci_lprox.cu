// Learned TV prox: theta = x + f(x), f a 4-layer 3x3x3 convolutional network
// (1 -> 32 -> 32 -> 32 -> 1 channels, ReLU between layers, zero "same"
// padding over frame, row and column), BF16 weights and activations with
// FP32 accumulation, FP32 master weights trained with Adam.
//
// The two 32 -> 32 layers (97% of the arithmetic) run on the tensor cores
// (sci_conv_tc.cu), forward and input-gradient.  The 1-channel layers, the
// weight gradients and the optimizer run on the CUDA cores here.
//
// The paper has no learned component (its future-work paragraph points at
// plug-and-play reconstruction); this network stands in for S FGP dual
// updates inside GAP-TV and is trained on (x, FGP_S(x)) pairs that the plain
// method produces.
//
// Parameters (FP32, contiguous): w1 [27][32][1], b1 [32], w2 [27][32][32],
// b2 [32], w3 [27][32][32], b3 [32], w4 [27][1][32], b4 [1]; tap index
// (dz+1)*9 + (dy+1)*3 + (dx+1); layer l computes
// out[v][o] = b[o] + sum_tap sum_i w[tap][o][i] * in[v + offset(tap)][i].
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sci_internal.cuh"

namespace sci {

bool launch_conv3d_c32_tc(const __nv_bfloat16* act, const __nv_bfloat16* w, const float* bias,
                          const __nv_bfloat16* mask_act, int mode, int nvol, int D, int H, int W,
                          __nv_bfloat16* out, int* err, cudaStream_t s);
bool launch_conv3d_c32_to1_tc(const __nv_bfloat16* act, const __nv_bfloat16* w, const float* bias, const float* x,
                              float* theta, int nvol, int D, int H, int W, int* err, cudaStream_t s);
bool launch_wgrad_c32_tc(const __nv_bfloat16* actT, const __nv_bfloat16* gT, int nvol, int D, int H, int Wp,
                         float* part, int max_slots, int* err, int* nslots, cudaStream_t s);

namespace {

constexpr int C = 32;
constexpr size_t kW1 = 0, kB1 = 864, kW2 = 896, kB2 = kW2 + 27648, kW3 = kB2 + 32, kB3 = kW3 + 27648,
                 kW4 = kB3 + 32, kB4 = kW4 + 864, kParams = kB4 + 1;

struct Vol {
    int nvol, D, H, W;
    long long V;  // voxels
};

// neighbour (z+dz, y+dy, x+dx) of voxel (n, z, y, x), or -1 outside the volume
__device__ __forceinline__ long long nb(const Vol& g, int n, int z, int y, int x, int tap) {
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const int zz = z + dz, yy = y + dy, xx = x + dx;
    if (zz < 0 || zz >= g.D || yy < 0 || yy >= g.H || xx < 0 || xx >= g.W) return -1;
    return (((long long)n * g.D + zz) * g.H + yy) * g.W + xx;
}

__device__ __forceinline__ void decomp(const Vol& g, long long v, int& n, int& z, int& y, int& x) {
    x = (int)(v % g.W);
    long long t = v / g.W;
    y = (int)(t % g.H);
    t /= g.H;
    z = (int)(t % g.D);
    n = (int)(t / g.D);
}

__device__ __forceinline__ void load32(const __nv_bfloat16* p, float (&a)[32]) {
    const uint4* p4 = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint4 u = p4[c];
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 f = __bfloat1622float2(h[k]);
            a[8 * c + 2 * k] = f.x;
            a[8 * c + 2 * k + 1] = f.y;
        }
    }
}

__device__ __forceinline__ void store32(__nv_bfloat16* p, const float (&a)[32]) {
    uint4 pk[4];
    uint32_t* pw = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        __nv_bfloat162 h2 = __floats2bfloat162_rn(a[2 * c], a[2 * c + 1]);
        pw[c] = *reinterpret_cast<uint32_t*>(&h2);
    }
    uint4* d = reinterpret_cast<uint4*>(p);
#pragma unroll
    for (int c = 0; c < 4; ++c) d[c] = pk[c];
}

// BF16 copies of the 32 -> 32 weights: forward [tap][o][i] and, for the
// input gradient, the tap-reversed transpose wt[tap][i][o] = w[26 - tap][o][i];
// and of layer 4 (32 -> 1) for the tensor cores' N = 16 form: w4n[pair][row][i]
// with pair = (dz + 1) 3 + (dy + 1), rows 0-2 the taps dx = -1..+1, rows 3-15 zero.
__global__ void k_prep_weights(const float* __restrict__ prm, __nv_bfloat16* __restrict__ w2, __nv_bfloat16* w2t,
                               __nv_bfloat16* __restrict__ w3, __nv_bfloat16* w3t, __nv_bfloat16* __restrict__ w4n) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 27 * C * C) return;
    const int tap = idx / (C * C), o = (idx / C) % C, i = idx % C;
    const int tidx = (26 - tap) * C * C + i * C + o;
    w2[idx] = __float2bfloat16_rn(prm[kW2 + idx]);
    w3[idx] = __float2bfloat16_rn(prm[kW3 + idx]);
    if (idx < 9 * 16 * C) {
        const int pair = idx / (16 * C), row = (idx / C) % 16;
        w4n[idx] = row < 3 ? __float2bfloat16_rn(prm[kW4 + (pair * 3 + row) * C + i]) : __float2bfloat16_rn(0.f);
    }
    if (w2t) w2t[tidx] = __float2bfloat16_rn(prm[kW2 + idx]);
    if (w3t) w3t[tidx] = __float2bfloat16_rn(prm[kW3 + idx]);
}

// layer 1 (1 -> 32) + ReLU.  A CTA computes an 8-row x 64-column tile of one
// frame.  x, rounded to BF16 like the other layers' operands, is staged in
// shared memory with a one-voxel halo in all three directions; zeros outside
// the volume are the convolution's zero padding, so no tap needs a bounds
// test.  Thread t computes columns t % 32 and t % 32 + 32 of row t / 32: each
// weight, broadcast from shared memory, feeds both voxels.  Taps accumulate in
// the same order as a plain per-voxel loop (bias first, then tap 0..26).
constexpr int kCiH = 8, kCiW = 64;

__global__ void __launch_bounds__(256) k_conv_in(const float* __restrict__ x, const float* __restrict__ prm, Vol g,
                                                 int tiles_w, int tiles_h, __nv_bfloat16* __restrict__ act1) {
    __shared__ float4 sw4[(27 * C + C) / 4];          // weights [27][32], then bias [32]
    __shared__ float sx[3][kCiH + 2][kCiW + 2];       // frames z-1..z+1, rows y0-1.., columns x0-1..
    float* sw = reinterpret_cast<float*>(sw4);
    for (int i = threadIdx.x; i < 27 * C; i += blockDim.x)
        sw[i] = __bfloat162float(__float2bfloat16_rn(prm[kW1 + i]));
    for (int i = threadIdx.x; i < C; i += blockDim.x) sw[27 * C + i] = prm[kB1 + i];
    long long r = blockIdx.x;
    const int tw = (int)(r % tiles_w);
    r /= tiles_w;
    const int th = (int)(r % tiles_h);
    r /= tiles_h;
    const int z = (int)(r % g.D), n = (int)(r / g.D);
    const int x0 = tw * kCiW, y0 = th * kCiH;
    for (int e = threadIdx.x; e < 3 * (kCiH + 2) * (kCiW + 2); e += blockDim.x) {
        const int f = e / ((kCiH + 2) * (kCiW + 2)), rem = e % ((kCiH + 2) * (kCiW + 2));
        const int zz = z + f - 1, yy = y0 - 1 + rem / (kCiW + 2), xx = x0 - 1 + rem % (kCiW + 2);
        float v = 0.f;
        if (zz >= 0 && zz < g.D && yy >= 0 && yy < g.H && xx >= 0 && xx < g.W)
            v = __bfloat162float(__float2bfloat16_rn(x[(((long long)n * g.D + zz) * g.H + yy) * g.W + xx]));
        sx[f][rem / (kCiW + 2)][rem % (kCiW + 2)] = v;
    }
    __syncthreads();
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    float a0[32], a1[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) a0[c] = a1[c] = sw[27 * C + c];
#pragma unroll 3
    for (int t = 0; t < 27; ++t) {
        const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
        const float xv0 = sx[dz][ty + dy][tx + dx], xv1 = sx[dz][ty + dy][tx + 32 + dx];
#pragma unroll
        for (int c4 = 0; c4 < 8; ++c4) {
            const float4 w = sw4[t * 8 + c4];
            a0[4 * c4 + 0] = fmaf(w.x, xv0, a0[4 * c4 + 0]);
            a0[4 * c4 + 1] = fmaf(w.y, xv0, a0[4 * c4 + 1]);
            a0[4 * c4 + 2] = fmaf(w.z, xv0, a0[4 * c4 + 2]);
            a0[4 * c4 + 3] = fmaf(w.w, xv0, a0[4 * c4 + 3]);
            a1[4 * c4 + 0] = fmaf(w.x, xv1, a1[4 * c4 + 0]);
            a1[4 * c4 + 1] = fmaf(w.y, xv1, a1[4 * c4 + 1]);
            a1[4 * c4 + 2] = fmaf(w.z, xv1, a1[4 * c4 + 2]);
            a1[4 * c4 + 3] = fmaf(w.w, xv1, a1[4 * c4 + 3]);
        }
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        a0[c] = fmaxf(a0[c], 0.f);
        a1[c] = fmaxf(a1[c], 0.f);
    }
    const int yy = y0 + ty;
    if (yy >= g.H) return;
    const long long row = (((long long)n * g.D + z) * g.H + yy) * g.W;
    if (x0 + tx < g.W) store32(act1 + (row + x0 + tx) * C, a0);
    if (x0 + tx + 32 < g.W) store32(act1 + (row + x0 + tx + 32) * C, a1);
}

// layer 4 (32 -> 1) and the residual output theta = x + f.  With a target,
// also g = d loss / d f = 2 (theta - target) / n and per-block FP64 partial
// sums of (theta - target)^2.
__global__ void k_conv_out(const __nv_bfloat16* __restrict__ act3, const float* __restrict__ prm, Vol g,
                           const float* __restrict__ x, float* __restrict__ theta, const float* __restrict__ target,
                           float* __restrict__ g4, double* __restrict__ partials) {
    __shared__ float sw[27 * C + 1];
    for (int i = threadIdx.x; i < 27 * C; i += blockDim.x)
        sw[i] = __bfloat162float(__float2bfloat16_rn(prm[kW4 + i]));
    if (threadIdx.x == 0) sw[27 * C] = prm[kB4];
    __syncthreads();
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double d2 = 0.0;
    if (v < g.V) {
        int n, z, y, xx;
        decomp(g, v, n, z, y, xx);
        float acc = sw[27 * C];
        for (int t = 0; t < 27; ++t) {
            const long long u = nb(g, n, z, y, xx, t);
            if (u < 0) continue;
            float a[32];
            load32(act3 + u * C, a);
#pragma unroll
            for (int c = 0; c < 32; ++c) acc = fmaf(sw[t * C + c], a[c], acc);
        }
        const float th = x[v] + acc;
        if (theta) theta[v] = th;
        if (target) {
            const float d = th - target[v];
            g4[v] = 2.f * d / (float)g.V;
            d2 = (double)d * (double)d;
        }
    }
    if (partials) {
        d2 = block_sum(d2);
        if (threadIdx.x == 0) partials[blockIdx.x] = d2;
    }
}

// d loss / d act3 through layer 4, masked by act3's ReLU:
// g3[u][i] = (act3[u][i] > 0) sum_tap w4[tap][i] g4[u - offset(tap)]
__global__ void k_dgrad_out(const float* __restrict__ g4, const float* __restrict__ prm, Vol g,
                            const __nv_bfloat16* __restrict__ act3, __nv_bfloat16* __restrict__ g3) {
    __shared__ float sw[27 * C];
    for (int i = threadIdx.x; i < 27 * C; i += blockDim.x)
        sw[i] = __bfloat162float(__float2bfloat16_rn(prm[kW4 + i]));
    __syncthreads();
    const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= g.V) return;
    int n, z, y, xx;
    decomp(g, u, n, z, y, xx);
    float acc[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = 0.f;
    for (int t = 0; t < 27; ++t) {
        const long long v = nb(g, n, z, y, xx, 26 - t);  // u - offset(t)
        if (v < 0) continue;
        const float gv = g4[v];
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] = fmaf(sw[t * C + c], gv, acc[c]);
    }
    float a[32];
    load32(act3 + u * C, a);
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = a[c] > 0.f ? acc[c] : 0.f;
    store32(g3 + u * C, acc);
}

// Weight and bias gradients of a 32 -> 32 layer run on the tensor cores
// (k_wgrad_c32_tc), as a GEMM over voxels whose operands have each row's
// voxels contiguous per channel: the layer input transposed per row, and its
// output gradient transposed per row and shifted by dx = -1, 0, +1.
// (kWgTile / kWgCols: the one-channel layers' tiled gradient kernels below.)
constexpr int kWgTile = 64, kWgCols = kWgTile + 2, kWgMaxBlocks = 256, kWgSlot = 27 * C * C + C;

// Both operands in one pass over a 32-voxel x 32-channel tile of a row:
// actT[row][c][x] = act[row][x][c] and gT[k][row][c][x] = g[row][x - (k - 1)][c]
// for k = 0, 1, 2 and x < Wp (zero outside [0, W)).  The tile's activations
// and its gradient columns x0 - 1 .. x0 + 32 pass through shared memory, read
// as voxels' channel vectors and written as channels' voxel runs, both
// coalesced; the three shifted copies come from the one staged gradient tile.
__global__ void __launch_bounds__(256) k_wgrad_operands(const __nv_bfloat16* __restrict__ act,
                                                        const __nv_bfloat16* __restrict__ grad,
                                                        __nv_bfloat16* __restrict__ actT, __nv_bfloat16* __restrict__ gT,
                                                        long long rows, int W, int Wp) {
    // tiles of 64 voxels; a voxel's 32 channels move as four 16-byte words,
    // a channel's run of 8 voxels as one
    __shared__ unsigned short ta[32][64 + 2];
    __shared__ unsigned short tg[32][66 + 2];
    const int tiles = Wp / 32;
    const uint4* a4 = reinterpret_cast<const uint4*>(act);
    const uint4* g4 = reinterpret_cast<const uint4*>(grad);
    unsigned short* at16 = reinterpret_cast<unsigned short*>(actT);
    unsigned short* gt16 = reinterpret_cast<unsigned short*>(gT);
    const size_t copy = (size_t)rows * C * Wp;  // elements of one transposed field
    const int tiles2 = (tiles + 1) / 2;          // 64-voxel tiles per row
    for (long long tile = blockIdx.x; tile < rows * tiles2; tile += gridDim.x) {
        const long long row = tile / tiles2;
        const int x0 = (int)(tile % tiles2) * 64;
        const int nx = min(64, Wp - x0);  // 32 or 64 columns of this tile
        __syncthreads();  // the previous tile's reads are done
        for (int e = threadIdx.x; e < (nx + 2) * 4; e += blockDim.x) {
            const int j = e >> 2, q = e & 3, x = x0 - 1 + j;  // gradient columns x0 - 1 .. x0 + nx
            const bool in = x >= 0 && x < W;
            const uint4 gv = in ? __ldg(g4 + (row * W + x) * 4 + q) : make_uint4(0, 0, 0, 0);
            const unsigned short* gs = reinterpret_cast<const unsigned short*>(&gv);
#pragma unroll
            for (int k = 0; k < 8; ++k) tg[q * 8 + k][j] = gs[k];
            if (j >= 1 && j <= nx) {
                const uint4 av = in ? __ldg(a4 + (row * W + x) * 4 + q) : make_uint4(0, 0, 0, 0);
                const unsigned short* as = reinterpret_cast<const unsigned short*>(&av);
#pragma unroll
                for (int k = 0; k < 8; ++k) ta[q * 8 + k][j - 1] = as[k];
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * (nx / 8); e += blockDim.x) {
            const int c = e / (nx / 8), x8 = (e % (nx / 8)) * 8;
            const size_t at = ((size_t)row * C + c) * Wp + x0 + x8;
            auto pack = [](const unsigned short* r) {  // eight 16-bit values, first lowest
                return make_uint4((unsigned)r[0] | (unsigned)r[1] << 16, (unsigned)r[2] | (unsigned)r[3] << 16,
                                  (unsigned)r[4] | (unsigned)r[5] << 16, (unsigned)r[6] | (unsigned)r[7] << 16);
            };
            *reinterpret_cast<uint4*>(at16 + at) = pack(&ta[c][x8]);
#pragma unroll
            for (int d = 0; d < 3; ++d) *reinterpret_cast<uint4*>(gt16 + d * copy + at) = pack(&tg[c][x8 - d + 2]);
        }
    }
}

// Slots of `len` values (the first nw weight gradients, then bias gradients):
// dw[j] += sum over CTA slots b of part[b][j] (db likewise), in slot order.
__global__ void k_wgrad_reduce(const float* __restrict__ part, int nslots, int len, int nw,
                               float* __restrict__ dw, float* __restrict__ db) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= len) return;
    float s = 0.f;
    for (int b = 0; b < nslots; ++b) s += part[(size_t)b * len + j];
    if (j < nw) dw[j] += s;
    else db[j - nw] += s;
}

// Tile staging shared by the one-channel layers' gradients: tile (n, z, y, x0)
// of kWgTile voxels of one row.
__device__ __forceinline__ void wg_tile(const Vol& g, int tiles_x, long long tile, int& n, int& z, int& y, int& x0) {
    x0 = (int)(tile % tiles_x) * kWgTile;
    long long r = tile / tiles_x;
    y = (int)(r % g.H);
    r /= g.H;
    z = (int)(r % g.D);
    n = (int)(r / g.D);
}

// Layer 1 (input x, one channel): dw1[tap][o] = sum_v g1[v][o] x[v + offset(tap)],
// db1[o] = sum_v g1[v][o].  x enters as BF16-rounded (the forward's operand).
// Thread (row, o), 9 x 32 threads; sliding window of g1 over the x columns.
__global__ void __launch_bounds__(288) k_wgrad_in_tiled(const __nv_bfloat16* __restrict__ g1,
                                                        const float* __restrict__ x, Vol g, int tiles_x,
                                                        float* __restrict__ part) {
    __shared__ float sx[9][kWgCols];          // x rows (dz, dy), columns x0 - 1 ..
    __shared__ float sG[kWgCols + 2][C];      // g1 at columns x0 - 2 .., zero outside the tile
    const int row = threadIdx.x / C, o = threadIdx.x % C;
    float acc[3] = {0.f, 0.f, 0.f}, bacc = 0.f;
    const long long ntiles = (long long)g.nvol * g.D * g.H * tiles_x;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int n, z, y, x0;
        wg_tile(g, tiles_x, tile, n, z, y, x0);
        __syncthreads();
        for (int e = threadIdx.x; e < 9 * kWgCols; e += blockDim.x) {
            const int r = e / kWgCols, col = e % kWgCols;
            const int zz = z + r / 3 - 1, yy = y + r % 3 - 1, xx = x0 - 1 + col;
            float v = 0.f;
            if (zz >= 0 && zz < g.D && yy >= 0 && yy < g.H && xx >= 0 && xx < g.W)
                v = __bfloat162float(__float2bfloat16_rn(x[(((long long)n * g.D + zz) * g.H + yy) * g.W + xx]));
            sx[r][col] = v;
        }
        for (int e = threadIdx.x; e < (kWgCols + 2) * C; e += blockDim.x) {
            const int col = e / C, c = e % C, xx = x0 - 2 + col;
            float v = 0.f;
            if (xx >= x0 && xx < x0 + kWgTile && xx < g.W)
                v = __bfloat162float(g1[((((long long)n * g.D + z) * g.H + y) * g.W + xx) * C + c]);
            sG[col][c] = v;
        }
        __syncthreads();
        float gm = sG[0][o], g0 = sG[1][o];
        for (int c = 0; c < kWgCols; ++c) {
            const float gp = sG[c + 2][o], xv = sx[row][c];
            if (row == 0) bacc += g0;
            acc[0] = fmaf(gp, xv, acc[0]);  // dx = -1
            acc[1] = fmaf(g0, xv, acc[1]);  // dx = 0
            acc[2] = fmaf(gm, xv, acc[2]);  // dx = +1
            gm = g0;
            g0 = gp;
        }
    }
    float* dst = part + (size_t)blockIdx.x * (27 * C + C);
#pragma unroll
    for (int d = 0; d < 3; ++d) dst[(row * 3 + d) * C + o] = acc[d];
    if (row == 0) dst[27 * C + o] = bacc;
}

// Layer 4 (one output channel): dw4[tap][i] = sum_v g4[v] a3[v + offset(tap)][i],
// db4 = sum_v g4[v].  Thread (part, row, i-quad): three column ranges of the
// tile in parallel, combined in shared memory in a fixed order at the end.
__global__ void __launch_bounds__(256) k_wgrad_out_tiled(const float* __restrict__ g4,
                                                         const __nv_bfloat16* __restrict__ a3, Vol g, int tiles_x,
                                                         float* __restrict__ part) {
    extern __shared__ float4 wo_smem4[];
    float* sA = reinterpret_cast<float*>(wo_smem4);  // [9][kWgCols][32]
    float* sg = sA + 9 * kWgCols * C;               // [kWgCols + 2]: g4 at columns x0 - 2 ..
    float* red = sg + kWgCols + 2;                  // [3][27 * 32 + 1]
    const int tid = threadIdx.x, cp = tid / 72, row = (tid % 72) / 8, iq = (tid % 8) * 4;
    const bool active = tid < 216;
    constexpr int kSpan = (kWgCols + 2) / 3;  // 22 columns per part
    float acc[3][4] = {}, bacc = 0.f;
    const long long ntiles = (long long)g.nvol * g.D * g.H * tiles_x;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int n, z, y, x0;
        wg_tile(g, tiles_x, tile, n, z, y, x0);
        __syncthreads();
        for (int e = tid; e < 9 * kWgCols * 4; e += blockDim.x) {
            const int q = e & 3, col = (e >> 2) % kWgCols, r = (e >> 2) / kWgCols;
            const int zz = z + r / 3 - 1, yy = y + r % 3 - 1, xx = x0 - 1 + col;
            float f[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) f[k] = 0.f;
            if (zz >= 0 && zz < g.D && yy >= 0 && yy < g.H && xx >= 0 && xx < g.W) {
                const long long u = (((long long)n * g.D + zz) * g.H + yy) * g.W + xx;
                const uint4 raw = __ldg(reinterpret_cast<const uint4*>(a3 + u * C + q * 8));
                const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 v2 = __bfloat1622float2(h[k]);
                    f[2 * k] = v2.x;
                    f[2 * k + 1] = v2.y;
                }
            }
            float4* d = reinterpret_cast<float4*>(sA + (r * kWgCols + col) * C + q * 8);
            d[0] = make_float4(f[0], f[1], f[2], f[3]);
            d[1] = make_float4(f[4], f[5], f[6], f[7]);
        }
        for (int col = tid; col < kWgCols + 2; col += blockDim.x) {
            const int xx = x0 - 2 + col;
            sg[col] = (xx >= x0 && xx < x0 + kWgTile && xx < g.W)
                          ? g4[(((long long)n * g.D + z) * g.H + y) * g.W + xx] : 0.f;
        }
        __syncthreads();
        if (active) {
            const int c0 = cp * kSpan, c1 = min(c0 + kSpan, kWgCols);
            for (int c = c0; c < c1; ++c) {
                const float gp = sg[c + 2], g0 = sg[c + 1], gm = sg[c];
                if (row == 0 && iq == 0) bacc += g0;
                const float4 a = *reinterpret_cast<const float4*>(sA + (row * kWgCols + c) * C + iq);
                const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    acc[0][k] = fmaf(gp, av[k], acc[0][k]);  // dx = -1
                    acc[1][k] = fmaf(g0, av[k], acc[1][k]);  // dx = 0
                    acc[2][k] = fmaf(gm, av[k], acc[2][k]);  // dx = +1
                }
            }
        }
    }
    __syncthreads();
    constexpr int kLen = 27 * C + 1;
    if (active) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int k = 0; k < 4; ++k) red[cp * kLen + (row * 3 + d) * C + iq + k] = acc[d][k];
        if (row == 0 && iq == 0) red[cp * kLen + 27 * C] = bacc;
    }
    __syncthreads();
    float* dst = part + (size_t)blockIdx.x * kLen;
    for (int j = tid; j < kLen; j += blockDim.x) dst[j] = (red[j] + red[kLen + j]) + red[2 * kLen + j];
}

// Adam on the FP32 master parameters (bias-corrected step size).
__global__ void k_adam(float* __restrict__ prm, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr_t, float b1, float b2, float eps) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        prm[i] -= lr_t * mi / (sqrtf(vi) + eps);
    }
}

struct LWork {
    __nv_bfloat16 *a1, *a2, *a3, *ga, *gb, *w2, *w2t, *w3, *w3t, *w4n;
    __nv_bfloat16 *actT, *gT;  // weight gradients: the transposed operands (training)
    float *g4, *grad, *wpart;
    double* partials;
    int* err;
    size_t total;
};

int padded_width(int W) { return (W + 31) / 32 * 32; }

// V voxels in rows of W (the transposed weight-gradient operands pad rows to
// a multiple of 32 voxels).
LWork lwork_layout(long long V, int W, bool training, void* base) {
    LWork L{};
    size_t off = 0;
    char* b = static_cast<char*>(base);
    auto take = [&](size_t bytes) { char* p = b ? b + off : nullptr; off += align256(bytes); return p; };
    L.a1 = reinterpret_cast<__nv_bfloat16*>(take((size_t)V * C * 2));
    L.a2 = reinterpret_cast<__nv_bfloat16*>(take((size_t)V * C * 2));
    L.a3 = reinterpret_cast<__nv_bfloat16*>(take((size_t)V * C * 2));
    L.w2 = reinterpret_cast<__nv_bfloat16*>(take(27 * C * C * 2));
    L.w3 = reinterpret_cast<__nv_bfloat16*>(take(27 * C * C * 2));
    L.w4n = reinterpret_cast<__nv_bfloat16*>(take(9 * 16 * C * 2));
    L.err = reinterpret_cast<int*>(take(256));
    L.partials = reinterpret_cast<double*>(take((size_t)((V + 255) / 256 + 1) * 8));
    if (training) {
        L.ga = reinterpret_cast<__nv_bfloat16*>(take((size_t)V * C * 2));
        L.gb = reinterpret_cast<__nv_bfloat16*>(take((size_t)V * C * 2));
        L.w2t = reinterpret_cast<__nv_bfloat16*>(take(27 * C * C * 2));
        L.w3t = reinterpret_cast<__nv_bfloat16*>(take(27 * C * C * 2));
        L.g4 = reinterpret_cast<float*>(take((size_t)V * 4));
        L.grad = reinterpret_cast<float*>(take(kParams * 4));
        L.wpart = reinterpret_cast<float*>(take((size_t)kWgMaxBlocks * kWgSlot * 4));
        const size_t tbytes = (size_t)(V / W) * padded_width(W) * C * 2;
        L.actT = reinterpret_cast<__nv_bfloat16*>(take(tbytes));
        L.gT = reinterpret_cast<__nv_bfloat16*>(take(3 * tbytes));
    }
    L.total = off;
    return L;
}

int grid_for(long long V) { return (int)((V + 255) / 256); }

// Weight and bias gradients of a 32 -> 32 layer into dw / db (added): the
// operands transposed per row, the tensor-core totals per CTA, then the
// fixed-order sum over the CTAs' slots (the same gradient on every run).
bool enqueue_wgrad_c32(const __nv_bfloat16* gout, const __nv_bfloat16* ain, Vol g, const LWork& L, float* dw,
                       float* db, cudaStream_t s) {
    const int Wp = padded_width(g.W);
    const long long rows = (long long)g.nvol * g.D * g.H;
    const long long tiles = rows * ((Wp / 32 + 1) / 2);
    const unsigned tgrid = (unsigned)std::min<long long>(tiles, 152LL * 16);
    k_wgrad_operands<<<tgrid, 256, 0, s>>>(ain, gout, L.actT, L.gT, rows, g.W, Wp);
    int nslots = 0;
    if (!launch_wgrad_c32_tc(L.actT, L.gT, g.nvol, g.D, g.H, Wp, L.wpart, kWgMaxBlocks, L.err, &nslots, s))
        return false;
    k_wgrad_reduce<<<(kWgSlot + 255) / 256, 256, 0, s>>>(L.wpart, nslots, kWgSlot, 27 * C * C, dw, db);
    return true;
}

size_t wgrad_out_smem() { return (size_t)(9 * kWgCols * C + kWgCols + 2 + 3 * (27 * C + 1)) * sizeof(float); }

// Weight and bias gradients of layer 1 (from g1 and x) and layer 4 (from g4
// and a3) into dw / db (added).
bool enqueue_wgrad_1ch(bool layer1, const __nv_bfloat16* gact, const float* gx, const float* x,
                       const __nv_bfloat16* a3, Vol g, float* part, float* dw, float* db, cudaStream_t s) {
    static bool attr = false;
    if (!layer1 && !attr) {
        if (cudaFuncSetAttribute(k_wgrad_out_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)wgrad_out_smem()) != cudaSuccess)
            return false;
        attr = true;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles_x = (g.W + kWgTile - 1) / kWgTile;
    const long long ntiles = (long long)g.nvol * g.D * g.H * tiles_x;
    const int grid = (int)std::max(1LL, std::min<long long>({ntiles, 2LL * sms, (long long)kWgMaxBlocks}));
    if (layer1) {
        k_wgrad_in_tiled<<<grid, 9 * C, 0, s>>>(gact, x, g, tiles_x, part);
        k_wgrad_reduce<<<(27 * C + C + 255) / 256, 256, 0, s>>>(part, grid, 27 * C + C, 27 * C, dw, db);
    } else {
        k_wgrad_out_tiled<<<grid, 256, wgrad_out_smem(), s>>>(gx, a3, g, tiles_x, part);
        k_wgrad_reduce<<<(27 * C + 1 + 255) / 256, 256, 0, s>>>(part, grid, 27 * C + 1, 27 * C, dw, db);
    }
    return true;
}

// GAP projection for `count` volumes stored back to back:
// xt = theta + c_k R^+ (y - sum_k c_k theta_k); also x_out = xt when given.
__global__ void k_project_vols(const float* __restrict__ theta, const float* __restrict__ y,
                               const uint32_t* __restrict__ bits, int nx, int ny, int B, float* __restrict__ xt,
                               float* __restrict__ x_out) {
    const long long n = (long long)nx * ny;
    const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= n) return;
    const int vol = blockIdx.y;
    const long long vo = (long long)vol * B * n, po = (long long)vol * n;
    const uint32_t w = bits[po + pix];
    float acc = 0.f;
    for (int k = 0; k < B; ++k) acc += mask_bit(w, k) * theta[vo + k * n + pix];
    const uint32_t m = B >= 32 ? 0xffffffffu : ((1u << B) - 1u);
    const double R = (double)__popc(w & m);
    const float rinv = R == 0.0 ? 0.f : (float)(1.0 / R);
    const float r = rinv * (y[po + pix] - acc);
    for (int k = 0; k < B; ++k) {
        const long long i = vo + k * n + pix;
        const float v = theta[i] + mask_bit(w, k) * r;
        xt[i] = v;
        if (x_out) x_out[i] = v;
    }
}

// forward through the four layers; theta = x + f(x)
bool enqueue_forward(const float* prm, const float* x, Vol g, const LWork& L, float* theta, const float* target,
                     cudaStream_t s) {
    k_prep_weights<<<(27 * C * C + 255) / 256, 256, 0, s>>>(prm, L.w2, L.w2t, L.w3, L.w3t, L.w4n);
    {
        const int tiles_w = (g.W + kCiW - 1) / kCiW, tiles_h = (g.H + kCiH - 1) / kCiH;
        const long long blocks = (long long)g.nvol * g.D * tiles_h * tiles_w;
        k_conv_in<<<(unsigned)blocks, 256, 0, s>>>(x, prm, g, tiles_w, tiles_h, L.a1);
    }
    if (!launch_conv3d_c32_tc(L.a1, L.w2, prm + kB2, nullptr, 0, g.nvol, g.D, g.H, g.W, L.a2, L.err, s))
        return false;
    if (!launch_conv3d_c32_tc(L.a2, L.w3, prm + kB3, nullptr, 0, g.nvol, g.D, g.H, g.W, L.a3, L.err, s))
        return false;
    if (target == nullptr) {
        // inference: the 32 -> 1 layer on the tensor cores (N = 16: the three
        // dx taps of output channel 0 per MMA), which beats the per-voxel
        // CUDA-core form; training keeps k_conv_out for its loss terms
        return launch_conv3d_c32_to1_tc(L.a3, L.w4n, prm + kB4, x, theta, g.nvol, g.D, g.H, g.W, L.err, s);
    }
    k_conv_out<<<grid_for(g.V), 256, 0, s>>>(L.a3, prm, g, x, theta, target, L.g4, L.partials);
    return true;
}

bool vol_ok(int nx, int ny, int B, int count) {
    return nx > 0 && ny > 0 && B > 0 && count > 0 && (double)nx * ny * B * count < 2.0e9;
}

}  // namespace

}  // namespace sci

using namespace sci;

extern "C" {

size_t sci_lprox_param_count(void) { return kParams; }

size_t sci_lprox_workspace(int nx, int ny, int B, int count, int training) {
    if (!vol_ok(nx, ny, B, count)) return 0;
    return lwork_layout((long long)nx * ny * B * count, ny, training != 0, nullptr).total;
}

sci_status sci_lprox_apply(const float* params, const float* x, int nx, int ny, int B, int count, float* theta,
                           void* work, size_t work_bytes, sci_stream_t stream) {
    if (params == nullptr || x == nullptr || theta == nullptr || x == theta || !vol_ok(nx, ny, B, count))
        return SCI_ERR_ARG;
    const Vol g{count, B, nx, ny, (long long)nx * ny * B * count};
    const LWork need = lwork_layout(g.V, g.W, false, nullptr);
    if (work == nullptr || work_bytes < need.total || ((uintptr_t)work & 255u) != 0) return SCI_ERR_WORKSPACE;
    const LWork L = lwork_layout(g.V, g.W, false, work);
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(L.err, 0, sizeof(int), s);
    if (!enqueue_forward(params, x, g, L, theta, nullptr, s)) return SCI_ERR_CUDA;
    return check_launch();
}

sci_status sci_lprox_train_step(float* params, float* adam_m, float* adam_v, int step, float lr, const float* x,
                                const float* target, int nx, int ny, int B, int count, double* loss,
                                void* work, size_t work_bytes, sci_stream_t stream) {
    if (params == nullptr || adam_m == nullptr || adam_v == nullptr || x == nullptr || target == nullptr ||
        !vol_ok(nx, ny, B, count) || step < 1)
        return SCI_ERR_ARG;
    if (!std::isfinite(lr) || !(lr > 0.f)) return SCI_ERR_ARG;
    const Vol g{count, B, nx, ny, (long long)nx * ny * B * count};
    const LWork need = lwork_layout(g.V, g.W, true, nullptr);
    if (work == nullptr || work_bytes < need.total || ((uintptr_t)work & 255u) != 0) return SCI_ERR_WORKSPACE;
    const LWork L = lwork_layout(g.V, g.W, true, work);
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(L.err, 0, sizeof(int), s);
    if (!enqueue_forward(params, x, g, L, nullptr, target, s)) return SCI_ERR_CUDA;
    if (loss != nullptr) launch_sum_partials(L.partials, grid_for(g.V), loss, s);
    cudaMemsetAsync(L.grad, 0, kParams * 4, s);
    // layer 4
    if (!enqueue_wgrad_1ch(false, nullptr, L.g4, nullptr, L.a3, g, L.wpart, L.grad + kW4, L.grad + kB4, s))
        return SCI_ERR_CUDA;
    k_dgrad_out<<<grid_for(g.V), 256, 0, s>>>(L.g4, params, g, L.a3, L.ga);  // ga = g3
    // layer 3
    if (!enqueue_wgrad_c32(L.ga, L.a2, g, L, L.grad + kW3, L.grad + kB3, s)) return SCI_ERR_CUDA;
    if (!launch_conv3d_c32_tc(L.ga, L.w3t, nullptr, L.a2, 1, g.nvol, g.D, g.H, g.W, L.gb, L.err, s))
        return SCI_ERR_CUDA;  // gb = g2
    // layer 2
    if (!enqueue_wgrad_c32(L.gb, L.a1, g, L, L.grad + kW2, L.grad + kB2, s)) return SCI_ERR_CUDA;
    if (!launch_conv3d_c32_tc(L.gb, L.w2t, nullptr, L.a1, 1, g.nvol, g.D, g.H, g.W, L.ga, L.err, s))
        return SCI_ERR_CUDA;  // ga = g1
    // layer 1
    if (!enqueue_wgrad_1ch(true, L.ga, nullptr, x, nullptr, g, L.wpart, L.grad + kW1, L.grad + kB1, s))
        return SCI_ERR_CUDA;
    // Adam (beta1 0.9, beta2 0.999, eps 1e-8), bias-corrected step size
    const double b1 = 0.9, b2 = 0.999;
    const double lr_t = (double)lr * std::sqrt(1.0 - std::pow(b2, step)) / (1.0 - std::pow(b1, step));
    k_adam<<<64, 256, 0, s>>>(params, L.grad, adam_m, adam_v, (long long)kParams, (float)lr_t, 0.9f, 0.999f, 1e-8f);
    return check_launch();
}

// Gradients only (no update): grad[kParams] receives d loss / d params.
sci_status sci_lprox_grads(const float* params, const float* x, const float* target, int nx, int ny, int B,
                           int count, float* grad, double* loss, void* work, size_t work_bytes,
                           sci_stream_t stream) {
    if (params == nullptr || x == nullptr || target == nullptr || grad == nullptr || !vol_ok(nx, ny, B, count))
        return SCI_ERR_ARG;
    const Vol g{count, B, nx, ny, (long long)nx * ny * B * count};
    const LWork need = lwork_layout(g.V, g.W, true, nullptr);
    if (work == nullptr || work_bytes < need.total || ((uintptr_t)work & 255u) != 0) return SCI_ERR_WORKSPACE;
    LWork L = lwork_layout(g.V, g.W, true, work);
    L.grad = grad;
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(L.err, 0, sizeof(int), s);
    if (!enqueue_forward(params, x, g, L, nullptr, target, s)) return SCI_ERR_CUDA;
    if (loss != nullptr) launch_sum_partials(L.partials, grid_for(g.V), loss, s);
    cudaMemsetAsync(grad, 0, kParams * 4, s);
    if (!enqueue_wgrad_1ch(false, nullptr, L.g4, nullptr, L.a3, g, L.wpart, grad + kW4, grad + kB4, s))
        return SCI_ERR_CUDA;
    k_dgrad_out<<<grid_for(g.V), 256, 0, s>>>(L.g4, params, g, L.a3, L.ga);
    if (!enqueue_wgrad_c32(L.ga, L.a2, g, L, grad + kW3, grad + kB3, s)) return SCI_ERR_CUDA;
    if (!launch_conv3d_c32_tc(L.ga, L.w3t, nullptr, L.a2, 1, g.nvol, g.D, g.H, g.W, L.gb, L.err, s))
        return SCI_ERR_CUDA;
    if (!enqueue_wgrad_c32(L.gb, L.a1, g, L, grad + kW2, grad + kB2, s)) return SCI_ERR_CUDA;
    if (!launch_conv3d_c32_tc(L.gb, L.w2t, nullptr, L.a1, 1, g.nvol, g.D, g.H, g.W, L.ga, L.err, s))
        return SCI_ERR_CUDA;
    if (!enqueue_wgrad_1ch(true, L.ga, nullptr, x, nullptr, g, L.wpart, grad + kW1, grad + kB1, s))
        return SCI_ERR_CUDA;
    return check_launch();
}

size_t sci_gap_tv_lprox_workspace(int nx, int ny, int B, int count, const sci_params* plain) {
    if (!vol_ok(nx, ny, B, count) || plain == nullptr) return 0;
    const size_t N = (size_t)nx * ny * B * count;
    return align256(N * 4) * 2 + align256((size_t)count * 8) + align256(sci_reduce_workspace()) +
           std::max(lwork_layout((long long)N, ny, false, nullptr).total, sci_solver_workspace(nx, ny, B, plain));
}

sci_status sci_gap_tv_lprox(const float* params, const float* y, const uint32_t* bits, int nx, int ny, int B,
                            int count, int outer_iters, int init, float* theta, float* x_out, int check_every,
                            const double* resid_limit, float fallback_ratio, const sci_params* plain,
                            int* fell_back, double* resid_out, void* work, size_t work_bytes,
                            sci_stream_t stream) {
    if (params == nullptr || y == nullptr || bits == nullptr || theta == nullptr || plain == nullptr ||
        !vol_ok(nx, ny, B, count) || outer_iters < 0 || check_every < 0)
        return SCI_ERR_ARG;
    if (B > 32) return SCI_ERR_SHAPE;
    if (!std::isfinite(fallback_ratio) || fallback_ratio <= 0.f) return SCI_ERR_ARG;
    const size_t need = sci_gap_tv_lprox_workspace(nx, ny, B, count, plain);
    if (work == nullptr || work_bytes < need || ((uintptr_t)work & 255u) != 0) return SCI_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = (long long)nx * ny, Nv = n * B, N = Nv * count;
    char* w = static_cast<char*>(work);
    float* xt = reinterpret_cast<float*>(w);
    float* ckpt = reinterpret_cast<float*>(w + align256(N * 4));
    double* rdev = reinterpret_cast<double*>(w + 2 * align256(N * 4));
    void* rwork = w + 2 * align256(N * 4) + align256((size_t)count * 8);
    void* inner = static_cast<char*>(rwork) + align256(sci_reduce_workspace());
    const size_t inner_bytes = work_bytes - (size_t)(static_cast<char*>(inner) - w);
    const Vol g{count, B, nx, ny, N};
    const LWork L = lwork_layout(N, ny, false, inner);
    cudaMemsetAsync(L.err, 0, sizeof(int), s);
    if (init) {
        for (int v = 0; v < count; ++v)
            launch_adjoint<float>(y + v * n, bits + v * n, Geo{nx, ny, B, n}, theta + v * Nv, s);
    }
    std::vector<int> fell(count, 0), fall_t(count, 0);
    const int chunk = check_every > 0 ? check_every : std::max(outer_iters, 1);
    if (check_every > 0) cudaMemcpyAsync(ckpt, theta, (size_t)N * 4, cudaMemcpyDeviceToDevice, s);
    const dim3 pgrid((unsigned)((n + 255) / 256), (unsigned)count);
    int t = 0, c = 0;
    while (t < outer_iters) {
        const int it = std::min(chunk, outer_iters - t);
        for (int i = 0; i < it; ++i) {
            const bool last = t + i == outer_iters - 1;
            k_project_vols<<<pgrid, 256, 0, s>>>(theta, y, bits, nx, ny, B, xt, last ? x_out : nullptr);
            if (!enqueue_forward(params, xt, g, L, theta, nullptr, s)) return SCI_ERR_CUDA;
        }
        t += it;
        if (check_every > 0) {
            for (int v = 0; v < count; ++v)
                launch_residual_norm<float>(theta + v * Nv, y + v * n, bits + v * n, Geo{nx, ny, B, n},
                                            static_cast<double*>(rwork), rdev + v, s);
            std::vector<double> r(count);
            if (cudaMemcpyAsync(r.data(), rdev, (size_t)count * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return SCI_ERR_CUDA;
            for (int v = 0; v < count; ++v) {
                if (resid_out) resid_out[(size_t)v * ((outer_iters + check_every - 1) / check_every) + c] = r[v];
                if (!fell[v] && resid_limit && r[v] > (double)fallback_ratio * resid_limit[c]) {
                    fell[v] = 1;
                    fall_t[v] = t - it;  // restart from the checkpoint before this chunk
                }
                if (!fell[v])
                    cudaMemcpyAsync(ckpt + v * Nv, theta + v * Nv, (size_t)Nv * 4, cudaMemcpyDeviceToDevice, s);
            }
            ++c;
        }
    }
    // measurements whose residual left the plain run's band: plain GAP-TV from their checkpoint
    for (int v = 0; v < count; ++v) {
        if (fell_back) fell_back[v] = fell[v];
        if (!fell[v]) continue;
        cudaMemcpyAsync(theta + v * Nv, ckpt + v * Nv, (size_t)Nv * 4, cudaMemcpyDeviceToDevice, s);
        sci_params p = *plain;
        p.outer_iters = outer_iters - fall_t[v];
        p.init = 0;
        p.use_graph = 0;
        const sci_status st = sci_gap_tv(y + v * n, bits + v * n, nx, ny, B, &p, theta + v * Nv,
                                         x_out ? x_out + v * Nv : nullptr, nullptr, 0, inner, inner_bytes,
                                         stream);
        if (st != SCI_OK) return st;
    }
    return check_launch();
}

// Device word that the tensor-core kernel sets if one of its bounded waits
// gave up (0 = fine).  Read it after a synchronisation.
sci_status sci_lprox_error_word(void* work, size_t work_bytes, int nx, int ny, int B, int count, int training,
                                int** out) {
    if (out == nullptr || !vol_ok(nx, ny, B, count)) return SCI_ERR_ARG;
    const LWork need = lwork_layout((long long)nx * ny * B * count, ny, training != 0, nullptr);
    if (work == nullptr || work_bytes < need.total) return SCI_ERR_WORKSPACE;
    *out = lwork_layout((long long)nx * ny * B * count, ny, training != 0, work).err;
    return SCI_OK;
}

}  // extern "C"
