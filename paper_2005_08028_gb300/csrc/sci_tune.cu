// Fuse-depth autotuner.  The number K of FGP dual updates that one temporally
// blocked launch runs sets the tile's halo (K + 1 / K pixels) and so the share
// of each tile that is useful output, against the launches per TVdenoise
// (ceil(S / K)).  The best K depends on the frame size, the frame count (the
// tile class), the storage type and the GPU, so it is measured: each
// candidate runs a short solve, timed with CUDA events on the caller's stream.
// With FP32 storage every depth gives bit-identical results; with 16-bit
// storage the duals carried between launches are rounded where launches end.
// sci_tune_launch times (depth, tile class) pairs: the tile classes that fit a
// TV form and frame count trade the tile's area (the useful share at a given
// halo) against threads and registers per CTA.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sci_internal.cuh"

namespace {

constexpr int kMaxCandidates = 64;
constexpr int kMaxReps = 100;
constexpr int kMaxProbeIters = 1000;

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

bool args_ok(const int* cand, int n, int probe_iters, int reps, const float* ms, const int* best) {
    if (cand == nullptr || ms == nullptr || best == nullptr) return false;
    if (n < 1 || n > kMaxCandidates || reps < 1 || reps > kMaxReps) return false;
    if (probe_iters < 1 || probe_iters > kMaxProbeIters) return false;
    for (int i = 0; i < n; ++i)
        if (cand[i] < -1) return false;
    return true;
}

// Runs run(k) once untimed and `reps` times timed for every candidate k;
// ms[i] = median time of candidate i, *best = the first candidate with the
// smallest median.  Synchronises the stream after each timed run.
template <class Run>
sci_status time_candidates(Run run, const int* cand, int n, int reps, float* ms, int* best, cudaStream_t s) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return SCI_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return SCI_ERR_ARG;  // timing needs real launches
    Events ev;
    if (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess) return SCI_ERR_CUDA;
    std::vector<float> t((size_t)reps);
    int best_i = 0;
    for (int i = 0; i < n; ++i) {
        sci_status st = run(cand[i]);  // warm-up: attributes, caches, clocks
        if (st != SCI_OK) return st;
        for (int r = 0; r < reps; ++r) {
            if (cudaEventRecord(ev.a, s) != cudaSuccess) return SCI_ERR_CUDA;
            st = run(cand[i]);
            if (st != SCI_OK) return st;
            if (cudaEventRecord(ev.b, s) != cudaSuccess || cudaEventSynchronize(ev.b) != cudaSuccess ||
                cudaEventElapsedTime(&t[(size_t)r], ev.a, ev.b) != cudaSuccess)
                return SCI_ERR_CUDA;
        }
        std::sort(t.begin(), t.end());
        ms[i] = t[(size_t)reps / 2];
        if (ms[i] < ms[best_i]) best_i = i;
    }
    *best = cand[best_i];
    return SCI_OK;
}

}  // namespace

extern "C" {

sci_status sci_tune_fuse(int algo, const float* y, const uint32_t* bits, int nx, int ny, int B,
                         const sci_params* params, float* theta, float* u, void* work, size_t work_bytes,
                         const int* candidates, int n_candidates, int probe_iters, int reps, float* ms,
                         int* best, sci_stream_t stream) {
    if (params == nullptr || !args_ok(candidates, n_candidates, probe_iters, reps, ms, best)) return SCI_ERR_ARG;
    if (algo < SCI_ALGO_GAP || algo > SCI_ALGO_FISTA || (algo == SCI_ALGO_ADMM && u == nullptr)) return SCI_ERR_ARG;
    sci_params p = *params;
    p.outer_iters = probe_iters;
    p.init = 1;
    p.use_graph = 0;
    auto run = [&](int k) -> sci_status {
        p.fuse_k = k;
        switch (algo) {
            case SCI_ALGO_ADMM:
                return sci_admm_tv(y, bits, nx, ny, B, &p, theta, u, nullptr, nullptr, 0, work, work_bytes, stream);
            case SCI_ALGO_FISTA:
                return sci_fista_tv(y, bits, nx, ny, B, &p, theta, nullptr, nullptr, 0, work, work_bytes, stream);
            default:
                return sci_gap_tv(y, bits, nx, ny, B, &p, theta, nullptr, nullptr, 0, work, work_bytes, stream);
        }
    };
    return time_candidates(run, candidates, n_candidates, reps, ms, best, (cudaStream_t)stream);
}

sci_status sci_tune_launch(int algo, const float* y, const uint32_t* bits, int nx, int ny, int B,
                           const sci_params* params, float* theta, float* u, void* work, size_t work_bytes,
                           const int* fuse_ks, const int* tiles, int n_candidates, int probe_iters, int reps,
                           float* ms, int* best, sci_stream_t stream) {
    if (params == nullptr || tiles == nullptr || !args_ok(fuse_ks, n_candidates, probe_iters, reps, ms, best))
        return SCI_ERR_ARG;
    if (algo < SCI_ALGO_GAP || algo > SCI_ALGO_FISTA || (algo == SCI_ALGO_ADMM && u == nullptr)) return SCI_ERR_ARG;
    for (int i = 0; i < n_candidates; ++i)
        if (tiles[i] < 0) return SCI_ERR_ARG;
    std::vector<int> idx((size_t)n_candidates);
    for (int i = 0; i < n_candidates; ++i) idx[(size_t)i] = i;
    sci_params p = *params;
    p.outer_iters = probe_iters;
    p.init = 1;
    p.use_graph = 0;
    auto run = [&](int i) -> sci_status {
        p.fuse_k = fuse_ks[i];
        p.tile = tiles[i];
        switch (algo) {
            case SCI_ALGO_ADMM:
                return sci_admm_tv(y, bits, nx, ny, B, &p, theta, u, nullptr, nullptr, 0, work, work_bytes, stream);
            case SCI_ALGO_FISTA:
                return sci_fista_tv(y, bits, nx, ny, B, &p, theta, nullptr, nullptr, 0, work, work_bytes, stream);
            default:
                return sci_gap_tv(y, bits, nx, ny, B, &p, theta, nullptr, nullptr, 0, work, work_bytes, stream);
        }
    };
    // candidates are indices into the pair arrays; the best one is returned as an index
    return time_candidates(run, idx.data(), n_candidates, reps, ms, best, (cudaStream_t)stream);
}

sci_status sci_tune_fuse_batched(const sci_problem* problems, int count, const sci_params* params, void* work,
                                 size_t work_bytes, const int* candidates, int n_candidates, int probe_iters,
                                 int reps, float* ms, int* best, sci_stream_t stream) {
    if (params == nullptr || !args_ok(candidates, n_candidates, probe_iters, reps, ms, best)) return SCI_ERR_ARG;
    sci_params p = *params;
    p.outer_iters = probe_iters;
    p.init = 1;
    p.use_graph = 0;
    auto run = [&](int k) -> sci_status {
        p.fuse_k = k;
        return sci_gap_tv_batched(problems, count, &p, work, work_bytes, stream);
    };
    return time_candidates(run, candidates, n_candidates, reps, ms, best, (cudaStream_t)stream);
}

}  // extern "C"
