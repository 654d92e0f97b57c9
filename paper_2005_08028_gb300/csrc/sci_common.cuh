// Shared device helpers for libsci: storage types, mask bits, geometry.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sci.h"

namespace sci {

// Geometry of one measurement: B frames of nx x ny pixels, [B][nx][ny] layout.
struct Geo {
    int nx, ny, B;
    long long n;  // nx * ny pixels per frame
};

// ---- storage types: every field is loaded to FP32 and stored back rounded ----
template <typename T> __device__ __forceinline__ float ld(const T* p, long long i);
template <> __device__ __forceinline__ float ld<float>(const float* p, long long i) { return p[i]; }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p, long long i) {
    return __bfloat162float(p[i]);
}
template <> __device__ __forceinline__ float ld<__half>(const __half* p, long long i) {
    return __half2float(p[i]);
}

template <typename T> __device__ __forceinline__ void st(T* p, long long i, float v);
template <> __device__ __forceinline__ void st<float>(float* p, long long i, float v) { p[i] = v; }
template <> __device__ __forceinline__ void st<__nv_bfloat16>(__nv_bfloat16* p, long long i, float v) {
    p[i] = __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ void st<__half>(__half* p, long long i, float v) {
    p[i] = __float2half_rn(v);
}

// Two-step read-only load: ldraw issues the load and leaves a 16-bit field's
// bits in a float register; cvraw converts them.  Kernels that read many
// values issue every ldraw before the first cvraw: the 16-bit conversion,
// placed right after each load, kept the loads from overlapping.  FP32 fields
// pass through both steps unchanged.
template <typename T> __device__ __forceinline__ float ldraw(const T* p, long long i) {
    return __uint_as_float((unsigned)__ldg(reinterpret_cast<const unsigned short*>(p) + i));
}
template <> __device__ __forceinline__ float ldraw<float>(const float* p, long long i) { return __ldg(p + i); }
template <typename T> __device__ __forceinline__ float cvraw(float r);
template <> __device__ __forceinline__ float cvraw<float>(float r) { return r; }
template <> __device__ __forceinline__ float cvraw<__half>(float r) {
    return __half2float(__ushort_as_half((unsigned short)__float_as_uint(r)));
}
template <> __device__ __forceinline__ float cvraw<__nv_bfloat16>(float r) {
    return __bfloat162float(__ushort_as_bfloat16((unsigned short)__float_as_uint(r)));
}

template <typename T> struct dtype_of;
template <> struct dtype_of<float> { static constexpr int value = SCI_F32; };
template <> struct dtype_of<__nv_bfloat16> { static constexpr int value = SCI_BF16; };
template <> struct dtype_of<__half> { static constexpr int value = SCI_F16; };

inline size_t dtype_bytes(int dt) { return dt == SCI_F32 ? 4 : 2; }

// Mask value C_k(i, j) in {0, 1} from the packed word of pixel (i, j).
__device__ __forceinline__ float mask_bit(uint32_t word, int k) {
    return (float)((word >> k) & 1u);
}

// Pixel kernels use 1-D blocks of 256 threads covering a 32-column x 8-row
// tile: a warp reads 32 consecutive pixels of one row (one 128-byte line).
__device__ __forceinline__ void pixel_ij(int& i, int& j) {
    j = blockIdx.x * 32 + (threadIdx.x & 31);
    i = blockIdx.y * 8 + (threadIdx.x >> 5);
}

// Sum of one double per thread over a 1-D block (fixed order: warp shuffle
// tree, then warp 0 over the per-warp sums).  Valid in thread 0; every
// thread of the block must call it.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Host helpers -------------------------------------------------------------
inline dim3 pixel_block() { return dim3(256, 1, 1); }
inline dim3 pixel_grid(int nx, int ny) {
    return dim3((unsigned)((ny + 31) / 32), (unsigned)((nx + 7) / 8), 1);
}

inline sci_status check_launch() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SCI_OK : SCI_ERR_CUDA;
}

inline bool geo_ok(int nx, int ny, int B) {
    return nx > 0 && ny > 0 && B > 0;
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace sci
