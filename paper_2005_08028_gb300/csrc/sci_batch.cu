// Batched GAP-TV: many measurements of different sizes reconstructed
// together (Algorithm 1 applied to each).  Every launch covers all the
// measurements: the pixel kernels walk a table of 256-pixel blocks and the
// temporally blocked FGP kernel walks a table of tiles, both built once on the
// host and uploaded to the caller's workspace; the T outer iterations are
// captured as one CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <list>
#include <mutex>
#include <numeric>
#include <vector>

#include "sci_internal.cuh"

namespace sci {

// Default dual updates per fused launch (measured on 512x512x10: one-frame
// tiles run all 10 updates of an outer iteration in one launch; the 32 x 32
// VTV tiles are fastest at 6, i.e. launches of 6 + 4).
int default_fuse(int tv) { return tv == SCI_TV_VTV ? 6 : 10; }

namespace {

template <typename T>
__device__ __forceinline__ int find_item(const BatchItem<T>* items, int nitems, int w, bool by_pix) {
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((by_pix ? items[mid].pix_begin : items[mid].cta_begin) <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// rinv = 1/R (FP64, 0 where R = 0); theta^(0) = Phi^T y, or the caller's theta.
template <typename T>
__global__ void k_batch_setup(const BatchItem<T>* __restrict__ items, int nitems, int from_user) {
    const BatchItem<T>& it = items[find_item(items, nitems, blockIdx.x, true)];
    const long long pix = (long long)(blockIdx.x - it.pix_begin) * 256 + threadIdx.x;
    if (pix >= it.g.n) return;
    const uint32_t mask = it.g.B >= 32 ? 0xffffffffu : ((1u << it.g.B) - 1u);
    const uint32_t word = it.bits[pix];
    const double R = (double)__popc(word & mask);
    it.rinv[pix] = R == 0.0 ? 0.f : (float)(1.0 / R);
    const float yv = it.y[pix];
    for (int k = 0; k < it.g.B; ++k) {
        const long long idx = k * it.g.n + pix;
        st<T>(it.theta[0], idx, from_user ? it.theta_user[idx] : mask_bit(word, k) * yv);
    }
}

// r = rinv (y - sum_k c_k theta_k)
template <typename T>
__global__ void k_batch_residual(const BatchItem<T>* __restrict__ items, int nitems, int tpar) {
    const BatchItem<T>& it = items[find_item(items, nitems, blockIdx.x, true)];
    const long long pix = (long long)(blockIdx.x - it.pix_begin) * 256 + threadIdx.x;
    if (pix >= it.g.n) return;
    const uint32_t word = it.bits[pix];
    const T* th = it.theta[tpar];
    float acc = 0.f;
    for (int k = 0; k < it.g.B; ++k) acc += mask_bit(word, k) * ld<T>(th, k * it.g.n + pix);
    it.r[pix] = it.rinv[pix] * (it.y[pix] - acc);
}

// the caller's FP32 theta = theta^(T)
template <typename T>
__global__ void k_batch_finish(const BatchItem<T>* __restrict__ items, int nitems, int tpar) {
    const BatchItem<T>& it = items[find_item(items, nitems, blockIdx.x, true)];
    const long long pix = (long long)(blockIdx.x - it.pix_begin) * 256 + threadIdx.x;
    if (pix >= it.g.n) return;
    for (int k = 0; k < it.g.B; ++k) {
        const long long idx = k * it.g.n + pix;
        it.theta_user[idx] = ld<T>(it.theta[tpar], idx);
    }
}

struct ClassRun {
    int cls;          // tile class (fused_class)
    int ib, ie;       // its items in the table: [ib, ie)
    int K, halo;      // dual updates per launch and tile halo for this class
    int total_ctas;   // work items of this class
};

struct BatchPlan {
    int tv, total_pix_blocks;
    std::vector<int> order;  // problems in table order: by class, largest first
    std::vector<ClassRun> runs;
    size_t table_bytes, total_bytes;
    std::vector<size_t> off;  // per problem: base offset of its buffers
    std::vector<int> cls, tiles_x, tiles_y, ctas;
};

size_t per_problem_bytes(const sci_problem& p, size_t es) {
    const size_t n = (size_t)p.nx * p.ny, N = n * (size_t)p.B;
    return align256(n * 4) * 2 + align256(N * es) * 11;  // rinv, r; xt, theta x2, duals x8
}

sci_status make_plan(const sci_problem* probs, int count, const sci_params* prm, BatchPlan* plan) {
    if (probs == nullptr || count < 1 || prm == nullptr) return SCI_ERR_ARG;
    if (prm->tv < SCI_TV_ATV || prm->tv > SCI_TV_VTV) return SCI_ERR_ARG;
    if (!std::isfinite(prm->lambda)) return SCI_ERR_NONFINITE;
    if (!(prm->lambda > 0.f) || prm->outer_iters < 0 || prm->inner_iters < 1) return SCI_ERR_ARG;
    if (prm->storage < SCI_F32 || prm->storage > SCI_F16 || prm->fuse_k < -1) return SCI_ERR_ARG;
    // the batched driver runs the FGP and Chambolle boxes, without the dual warm start
    if (prm->dual != SCI_DUAL_FGP && prm->dual != SCI_DUAL_CHAM) return SCI_ERR_ARG;
    if (prm->warm_start != 0 || prm->check_input != 0 || prm->tile != 0) return SCI_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        const sci_problem& p = probs[i];
        if (p.nx <= 0 || p.ny <= 0 || p.B <= 0 || p.y == nullptr || p.bits == nullptr || p.theta == nullptr)
            return SCI_ERR_ARG;
        if (p.B > 32 || (double)p.nx * p.ny * p.B > 4.0e9) return SCI_ERR_SHAPE;
        if (fused_class(prm->tv, p.B) == 0) return SCI_ERR_SHAPE;  // VTV with B > 24
    }
    BatchPlan& P = *plan;
    P.tv = prm->tv;
    P.cls.resize(count);
    P.tiles_x.resize(count);
    P.tiles_y.resize(count);
    P.ctas.resize(count);
    for (int i = 0; i < count; ++i) P.cls[i] = fused_class(prm->tv, probs[i].B);
    // table order: grouped by class, largest problems first inside a class
    P.order.resize(count);
    std::iota(P.order.begin(), P.order.end(), 0);
    std::stable_sort(P.order.begin(), P.order.end(), [&](int a, int b) {
        if (P.cls[a] != P.cls[b]) return P.cls[a] < P.cls[b];
        return (long long)probs[a].nx * probs[a].ny * probs[a].B > (long long)probs[b].nx * probs[b].ny * probs[b].B;
    });
    P.runs.clear();
    for (int j = 0; j < count;) {
        const int c = P.cls[P.order[j]];
        int e = j;
        while (e < count && P.cls[P.order[e]] == c) ++e;
        ClassRun run{c, j, e, 0, 0, 0};
        const int maxh = fused_max_halo(prm->tv, probs[P.order[j]].B);
        int K = prm->fuse_k > 0 ? prm->fuse_k : default_fuse(prm->tv);
        K = std::max(1, std::min(std::min(K, maxh - 1), std::min(prm->inner_iters, kMaxFuse)));
        run.K = K;
        run.halo = K + 1;
        int EH = 0, EW = 0;
        fused_class_dims(c, &EH, &EW);
        const int TI = fused_interior(EH, run.halo), TJ = fused_interior(EW, run.halo);
        if (TI < 1 || TJ < 1) return SCI_ERR_SHAPE;
        long long tc = 0;
        for (int k = j; k < e; ++k) {
            const int i = P.order[k];
            const sci_problem& p = probs[i];
            P.tiles_x[i] = (p.ny + TJ - 1) / TJ;
            P.tiles_y[i] = (p.nx + TI - 1) / TI;
            const long long ct = (long long)P.tiles_x[i] * P.tiles_y[i] * (c == 1 ? p.B : 1);
            P.ctas[i] = (int)std::min(ct, 1LL << 30);
            tc += ct;
        }
        if (tc > (1LL << 31) - 1) return SCI_ERR_SHAPE;
        run.total_ctas = (int)tc;
        P.runs.push_back(run);
        j = e;
    }
    const size_t es = dtype_bytes(prm->storage);
    const size_t item_bytes = prm->storage == SCI_F32 ? sizeof(BatchItem<float>) : sizeof(BatchItem<__half>);
    P.table_bytes = align256(item_bytes * (size_t)count);
    size_t off = P.table_bytes;
    P.off.resize(count);
    long long tp = 0;
    for (int i = 0; i < count; ++i) {
        P.off[i] = off;
        off += per_problem_bytes(probs[i], es);
        tp += ((long long)probs[i].nx * probs[i].ny + 255) / 256;
    }
    if (tp > (1LL << 31) - 1) return SCI_ERR_SHAPE;
    P.total_pix_blocks = (int)tp;
    P.total_bytes = off;
    return SCI_OK;
}

template <typename T>
std::vector<BatchItem<T>> make_table(const sci_problem* probs, const BatchPlan& P, char* work) {
    std::vector<BatchItem<T>> items(P.order.size());
    int cta = 0, pixb = 0, run_cls = -1;
    for (size_t j = 0; j < P.order.size(); ++j) {
        const int i = P.order[j];
        if (P.cls[(size_t)i] != run_cls) {  // work items count from each class's start
            run_cls = P.cls[(size_t)i];
            cta = 0;
        }
        const sci_problem& p = probs[i];
        const size_t n = (size_t)p.nx * p.ny, N = n * (size_t)p.B;
        char* base = work + P.off[(size_t)i];
        BatchItem<T>& it = items[j];
        std::memset(&it, 0, sizeof(it));
        it.g = Geo{p.nx, p.ny, p.B, (long long)n};
        it.cls = P.cls[(size_t)i];
        it.tiles_x = P.tiles_x[(size_t)i];
        it.tiles_y = P.tiles_y[(size_t)i];
        it.cta_begin = cta;
        it.pix_begin = pixb;
        cta += P.ctas[(size_t)i];
        pixb += (int)((n + 255) / 256);
        it.y = p.y;
        it.bits = p.bits;
        it.x_out = p.x_out;
        it.theta_user = p.theta;
        size_t o = 0;
        it.rinv = reinterpret_cast<float*>(base + o); o += align256(n * 4);
        it.r = reinterpret_cast<float*>(base + o); o += align256(n * 4);
        it.xt = reinterpret_cast<T*>(base + o); o += align256(N * sizeof(T));
        for (int b = 0; b < 2; ++b) { it.theta[b] = reinterpret_cast<T*>(base + o); o += align256(N * sizeof(T)); }
        for (int b = 0; b < 2; ++b)
            for (int f = 0; f < 4; ++f) { it.st[b][f] = reinterpret_cast<T*>(base + o); o += align256(N * sizeof(T)); }
    }
    return items;
}

// Enqueue the whole batched solve; returns kernels launched or -1.
template <typename T>
int enqueue_batch(const BatchPlan& P, const sci_params* prm, const BatchItem<T>* d_items, int nitems,
                  bool want_x, cudaStream_t s) {
    int nk = 0;
    const int pb = P.total_pix_blocks;
    k_batch_setup<T><<<pb, 256, 0, s>>>(d_items, nitems, prm->init ? 0 : 1);
    ++nk;
    const int T_outer = prm->outer_iters, S = prm->inner_iters;
    int tpar = 0;
    if (T_outer > 0) { k_batch_residual<T><<<pb, 256, 0, s>>>(d_items, nitems, tpar); ++nk; }
    std::vector<double> nu_c((size_t)S, 0.0);  // momentum coefficients; zero for the Chambolle box
    if (prm->dual == SCI_DUAL_FGP) {
        double nu = 1.0;
        for (int i = 0; i < S; ++i) {
            const double nx = (1.0 + std::sqrt(1.0 + 4.0 * nu * nu)) / 2.0;
            nu_c[(size_t)i] = (nu - 1.0) / nx;
            nu = nx;
        }
    }
    std::vector<int> spar(P.runs.size(), 0);
    for (int t = 0; t < T_outer; ++t) {
        const bool last_outer = t == T_outer - 1;
        for (size_t c = 0; c < P.runs.size(); ++c) {
            const ClassRun& run = P.runs[c];
            for (int s0 = 0; s0 < S; s0 += run.K) {
                const int k = std::min(run.K, S - s0);
                FusedArgs a{};
                a.mode = OuterMode::Gap;
                a.K = k;
                a.halo = run.halo;  // fixed for the solve: the tile tables stay valid
                a.first = s0 == 0;
                a.last = s0 + k == S;
                a.lambda = prm->lambda;
                a.step = (float)(1.0 / (8.0 * (double)prm->lambda));
                for (int i = 0; i < k; ++i) a.coef[i] = (float)nu_c[(size_t)(s0 + i)];
                if (!launch_fgp_fused_batched<T>(P.tv, run.cls, a, d_items + run.ib, run.ie - run.ib,
                                                 run.total_ctas, tpar, spar[c],
                                                 (last_outer && a.last && want_x) ? 1 : 0, s))
                    return -1;
                ++nk;
                if (!a.last) spar[c] ^= 1;
            }
        }
        tpar ^= 1;
        if (!last_outer) { k_batch_residual<T><<<pb, 256, 0, s>>>(d_items, nitems, tpar); ++nk; }
    }
    k_batch_finish<T><<<pb, 256, 0, s>>>(d_items, nitems, tpar);
    ++nk;
    return nk;
}

struct BatchGraph {
    int device;
    std::vector<char> key;
    cudaGraphExec_t exec;
    int launches;
};
std::mutex g_bmu;
std::list<BatchGraph> g_bcache;
cudaStream_t g_bcapture[64] = {};
thread_local long long g_batch_launches = 0;

template <typename T>
sci_status run_batch(const sci_problem* probs, int count, const sci_params* prm, const BatchPlan& P, char* work,
                     cudaStream_t stream) {
    std::vector<BatchItem<T>> items = make_table<T>(probs, P, work);
    BatchItem<T>* d_items = reinterpret_cast<BatchItem<T>*>(work);
    bool want_x = false;
    for (int i = 0; i < count; ++i) want_x = want_x || probs[i].x_out != nullptr;
    // the table is copied (synchronously staged: pageable host memory) before the solve
    if (cudaMemcpyAsync(d_items, items.data(), sizeof(BatchItem<T>) * items.size(), cudaMemcpyHostToDevice,
                        stream) != cudaSuccess)
        return SCI_ERR_CUDA;
    if (!prm->use_graph) {
        const int nk = enqueue_batch<T>(P, prm, d_items, count, want_x, stream);
        if (nk < 0) return SCI_ERR_CUDA;
        g_batch_launches = nk;
        return check_launch();
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SCI_ERR_CUDA;
    std::vector<char> key(sizeof(sci_params) + sizeof(void*) + sizeof(sci_problem) * (size_t)count);
    std::memcpy(key.data(), prm, sizeof(sci_params));
    std::memcpy(key.data() + sizeof(sci_params), &work, sizeof(void*));
    std::memcpy(key.data() + sizeof(sci_params) + sizeof(void*), probs, sizeof(sci_problem) * (size_t)count);
    std::lock_guard<std::mutex> lock(g_bmu);
    for (auto it = g_bcache.begin(); it != g_bcache.end(); ++it) {
        if (it->device == dev && it->key == key) {
            g_bcache.splice(g_bcache.begin(), g_bcache, it);
            if (cudaGraphLaunch(g_bcache.front().exec, stream) != cudaSuccess) return SCI_ERR_CUDA;
            g_batch_launches = g_bcache.front().launches;
            return SCI_OK;
        }
    }
    if (g_bcapture[dev] == nullptr &&
        cudaStreamCreateWithFlags(&g_bcapture[dev], cudaStreamNonBlocking) != cudaSuccess)
        return SCI_ERR_CUDA;
    cudaStream_t cs = g_bcapture[dev];
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SCI_ERR_CUDA;
    const int nk = enqueue_batch<T>(P, prm, d_items, count, want_x, cs);
    const cudaError_t le = cudaGetLastError();
    cudaGraph_t graph = nullptr;
    if (cudaStreamEndCapture(cs, &graph) != cudaSuccess || le != cudaSuccess || nk < 0) {
        if (graph) cudaGraphDestroy(graph);
        return SCI_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return SCI_ERR_CUDA;
    g_bcache.push_front(BatchGraph{dev, std::move(key), exec, nk});
    while (g_bcache.size() > 8) {
        cudaGraphExecDestroy(g_bcache.back().exec);
        g_bcache.pop_back();
    }
    if (cudaGraphLaunch(exec, stream) != cudaSuccess) return SCI_ERR_CUDA;
    g_batch_launches = nk;
    return SCI_OK;
}

}  // namespace

}  // namespace sci

using namespace sci;

extern "C" {

size_t sci_gap_tv_batched_workspace(const sci_problem* probs, int count, const sci_params* params) {
    BatchPlan P;
    if (make_plan(probs, count, params, &P) != SCI_OK) return 0;
    return P.total_bytes;
}

sci_status sci_gap_tv_batched(const sci_problem* probs, int count, const sci_params* params, void* work,
                              size_t work_bytes, sci_stream_t stream) {
    BatchPlan P;
    sci_status st = make_plan(probs, count, params, &P);
    if (st != SCI_OK) return st;
    if (work == nullptr || work_bytes < P.total_bytes || ((uintptr_t)work & 255u) != 0) return SCI_ERR_WORKSPACE;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) return SCI_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return SCI_ERR_ARG;  // the table upload cannot be captured
    char* w = static_cast<char*>(work);
    switch (params->storage) {
        case SCI_BF16: return run_batch<__nv_bfloat16>(probs, count, params, P, w, (cudaStream_t)stream);
        case SCI_F16: return run_batch<__half>(probs, count, params, P, w, (cudaStream_t)stream);
        default: return run_batch<float>(probs, count, params, P, w, (cudaStream_t)stream);
    }
}

long long sci_last_batch_launches(void) { return g_batch_launches; }

void sci_batch_graph_cache_clear(void) {
    std::lock_guard<std::mutex> lock(g_bmu);
    for (auto& e : g_bcache) cudaGraphExecDestroy(e.exec);
    g_bcache.clear();
}

}  // extern "C"
