// sci_tv_prox_noalloc: the FGP TV prox of sci_tv_prox with its dual scratch
// in a fixed device array compiled into the library, for callers that cannot
// allocate device memory (see include/sci.h).
#include <cmath>
#include <mutex>

#include "sci_internal.cuh"

using namespace sci;

namespace {

// Three rotating dual buffers of two FP32 fields each: 24 bytes per voxel.
constexpr size_t kNoAllocScratchBytes = (size_t)48 << 20;  // 48 MiB
constexpr long long kNoAllocMaxVoxels = (long long)(kNoAllocScratchBytes / 24);  // 2,097,152

// Every GPU that loads libsci holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};

// Device address of the scratch array on the current device, looked up once
// per device.  In host code the array's name is only a host-side handle, so
// the address must come from cudaGetSymbolAddress.
sci_status noalloc_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SCI_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
            return SCI_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return SCI_OK;
}

}  // namespace

extern "C" {

long long sci_tv_prox_noalloc_max_voxels(void) { return kNoAllocMaxVoxels; }

sci_status sci_tv_prox_noalloc(const float* x, int nx, int ny, int B, int tv, float lambda,
                               int inner_iters, float* theta, sci_stream_t stream) {
    if (x == nullptr || theta == nullptr || x == theta || nx <= 0 || ny <= 0 || B <= 0)
        return SCI_ERR_ARG;
    if (tv < SCI_TV_ATV || tv > SCI_TV_VTV || inner_iters < 1) return SCI_ERR_ARG;
    if (!std::isfinite(lambda)) return SCI_ERR_NONFINITE;
    if (!(lambda > 0.f)) return SCI_ERR_ARG;
    const long long N = (long long)nx * ny * B;
    if ((double)nx * ny * B > (double)kNoAllocMaxVoxels || N > kNoAllocMaxVoxels) return SCI_ERR_SHAPE;
    void* base = nullptr;
    const sci_status st = noalloc_scratch(&base);
    if (st != SCI_OK) return st;

    // The three dual buffers sit back to back (each 2N floats, 256-byte aligned).
    const size_t stride = align256((size_t)2 * N * sizeof(float));
    float* P[3] = {static_cast<float*>(base),
                   reinterpret_cast<float*>(static_cast<char*>(base) + stride),
                   reinterpret_cast<float*>(static_cast<char*>(base) + 2 * stride)};
    const Geo g{nx, ny, B, (long long)nx * ny};
    cudaStream_t s = (cudaStream_t)stream;

    // Momentum coefficients (nu_s - 1)/nu_{s+1}, nu_0 = 1, in FP64.
    double nu = 1.0;
    float coef_prev = 0.f;
    // The first update writes every entry of P[0] before anything reads it,
    // so no part of the shared array needs clearing between calls.
    launch_fgp_first<float>(tv, OuterMode::Prox, x, nullptr, nullptr, nullptr, g, lambda, nullptr, P[0], s);
    {
        const double nu1 = (1.0 + std::sqrt(1.0 + 4.0 * nu * nu)) / 2.0;
        coef_prev = (float)((nu - 1.0) / nu1);
        nu = nu1;
    }
    int cur = 0, prev = -1;
    for (int it = 1; it < inner_iters; ++it) {
        const int out = 3 - cur - (prev < 0 ? (cur == 0 ? 1 : 0) : prev);
        launch_fgp_iter<float>(tv, x, P[cur], prev >= 0 ? P[prev] : nullptr, coef_prev, g, lambda, P[out], s);
        const double nxt = (1.0 + std::sqrt(1.0 + 4.0 * nu * nu)) / 2.0;
        coef_prev = (float)((nu - 1.0) / nxt);
        nu = nxt;
        prev = cur;
        cur = out;
    }
    OutArgs oa{};
    oa.mode = OuterMode::Prox;
    oa.xin = x;
    oa.theta_f32 = theta;
    launch_fgp_out<float>(oa, x, P[cur], g, lambda, nullptr, nullptr, s);
    return check_launch();
}

}  // extern "C"
