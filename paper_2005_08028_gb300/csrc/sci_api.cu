// C-ABI entry points of libsci (declared in include/sci.h): argument
// validation, workspace layout, the GAP-TV / ADMM-TV outer loop and its
// CUDA-graph cache.
//
// Outer loop (Algorithm 1 for GAP, Eqs. 24-26 for ADMM), with theta (and u)
// as the only state carried between iterations:
//   r  = rinv * (y - sum_k c_k (theta_k - u_k))     rinv = 1/R (GAP, pseudo-inverse)
//                                                    or 1/(R + rho) (ADMM); u = 0 for GAP
//   xt = theta + c_k r                               GAP: the projection x (Eq. 21)
//                                                    ADMM: u + x, x from Eq. 24
//   theta' = FGP prox of xt (S dual updates)
//   ADMM: u' = u + x - theta' = xt - theta'
// On the temporally blocked path one outer iteration is ceil(S/K) fused
// launches: the first forms xt = theta + c_k r on the fly (no separate
// projection pass), the last writes theta' (and u', x).  VTV tiles, which
// hold every frame of a pixel, also form the next residual r in that last
// launch; ATV / ITV2D tiles hold one frame, so one light residual pass
// (with 128-bit loads for fields above 64 MiB) follows their last launch.  The per-update path
// (fuse_k = -1) runs S launches of one dual update and an output kernel
// that forms the next residual.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <list>
#include <mutex>
#include <vector>

#include "sci_internal.cuh"

using namespace sci;

namespace {

constexpr int kVersion = 10000;  // 1.0.0

bool finite_pos(float v) { return std::isfinite(v) && v > 0.f; }

// Momentum coefficients (nu_s - 1)/nu_{s+1}, nu_0 = 1, computed in FP64
// (Algorithm 1, ATV-FGP box); all zero for the Chambolle box, whose dual
// update is the same projected step without momentum.
std::vector<float> momentum_coeffs(int S, int dual = SCI_DUAL_FGP) {
    std::vector<float> c((size_t)std::max(S, 1), 0.f);
    if (dual != SCI_DUAL_FGP) return c;  // the Chambolle and Clip boxes have no momentum
    double nu = 1.0;
    for (int s = 0; s < S; ++s) {
        const double nx = (1.0 + std::sqrt(1.0 + 4.0 * nu * nu)) / 2.0;
        c[(size_t)s] = (float)((nu - 1.0) / nx);
        nu = nx;
    }
    return c;
}

// ---- workspace layout ----
struct Layout {
    size_t rinv, r, r2, partials, xt, p[4], theta_s, theta_s2, u_s, xprev, lmax, warm, total;
};

// warm: room for the dual warm start's carried w (two ping-pong pairs of
// w_h, w_v fields in the storage type).
Layout solver_layout(int nx, int ny, int B, int storage, bool admm, bool warm = false) {
    Layout L{};
    const size_t n = (size_t)nx * ny, N = n * (size_t)B, es = dtype_bytes(storage);
    Geo g{nx, ny, B, (long long)n};
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off += align256(bytes); return at; };
    L.rinv = take(n * 4);
    L.r = take(n * 4);
    L.r2 = take(n * 4);  // the residual a VTV tile's last launch forms while its first launch read r
    L.partials = take((size_t)std::max(out_partial_count(g), kReduceParts) * 8);
    L.xt = take(N * es);
    for (int b = 0; b < 4; ++b) L.p[b] = take(2 * N * es);  // per-update path uses 3
    L.theta_s = storage != SCI_F32 ? take(N * es) : 0;
    L.theta_s2 = take(N * es);  // second theta buffer: the fused launch reads theta^(t) halos
                                // while other CTAs write theta^(t+1)
    L.u_s = (storage != SCI_F32 && admm) ? take(N * es) : 0;
    L.xprev = take(N * es);  // FISTA: x^(t-1)
    L.lmax = take(256);      // words 0-1: largest / smallest nonzero mask count (FISTA, TwIST);
                             // bytes 16-27: TwIST's weights; bytes 64-67: check_input's count
    L.warm = warm ? take(4 * N * es) : 0;
    L.total = off;
    return L;
}

Layout prox_layout(int nx, int ny, int B) {
    Layout L{};
    const size_t N = (size_t)nx * ny * B;
    size_t off = 0;
    for (int b = 0; b < 4; ++b) { L.p[b] = off; off += align256(2 * N * 4); }
    L.total = off;
    return L;
}

bool sizes_ok(int nx, int ny, int B) {
    if (nx <= 0 || ny <= 0 || B <= 0) return false;
    const double N = (double)nx * ny * B;
    return N < 9.0e15;
}

sci_status validate_params(const sci_params* p, bool admm) {
    if (p == nullptr) return SCI_ERR_ARG;
    if (p->tv < SCI_TV_ATV || p->tv > SCI_TV_VTV) return SCI_ERR_ARG;
    if (!std::isfinite(p->lambda) || !std::isfinite(p->rho)) return SCI_ERR_NONFINITE;
    if (!(p->lambda > 0.f)) return SCI_ERR_ARG;
    if (admm && !(p->rho >= 0.f)) return SCI_ERR_ARG;
    if (p->outer_iters < 0 || p->inner_iters < 1) return SCI_ERR_ARG;
    if (p->storage < SCI_F32 || p->storage > SCI_F16) return SCI_ERR_ARG;
    if (p->fuse_k < -1) return SCI_ERR_ARG;
    if (p->dual != SCI_DUAL_FGP && p->dual != SCI_DUAL_CHAM && p->dual != SCI_DUAL_CLIP) return SCI_ERR_ARG;
    if (p->dual == SCI_DUAL_CLIP && p->tv != SCI_TV_ATV) return SCI_ERR_ARG;  // Clip is an ATV box
    if (p->warm_start != 0 && p->warm_start != 1) return SCI_ERR_ARG;
    if (p->check_input != 0 && p->check_input != 1) return SCI_ERR_ARG;
    if (p->tile < 0) return SCI_ERR_ARG;
    return SCI_OK;
}

// check_input: count the non-finite entries of the solve's input arrays on
// the device (one word of the workspace), wait for the count, and report it.
sci_status check_inputs_finite(const float* const* arrays, const long long* sizes, int count, unsigned* word,
                               cudaStream_t s) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return SCI_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return SCI_ERR_ARG;  // the check must wait on the stream
    if (cudaMemsetAsync(word, 0, sizeof(unsigned), s) != cudaSuccess) return SCI_ERR_CUDA;
    for (int i = 0; i < count; ++i)
        if (arrays[i] != nullptr) launch_count_nonfinite(arrays[i], sizes[i], word, s);
    unsigned host = 0;
    if (cudaMemcpyAsync(&host, word, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SCI_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SCI_ERR_CUDA;
    return host ? SCI_ERR_NONFINITE : SCI_OK;
}

sci_status validate_work(void* work, size_t have, size_t need) {
    if (need == 0) return SCI_OK;
    if (work == nullptr || have < need) return SCI_ERR_WORKSPACE;
    if (((uintptr_t)work & 255u) != 0) return SCI_ERR_WORKSPACE;
    return SCI_OK;
}

// Dual updates per fused launch: fuse_k = -1 turns temporal blocking off;
// otherwise the largest count the tile halo allows (halo = K + 1), capped by
// fuse_k when it is positive.  Returns 0 when the per-update kernels serve.
int choose_fuse(int tv, int B, int S, int fuse_k, int tile = 0) {
    if (fuse_k < 0) return 0;
    const int maxh = tile != 0 ? fused_class_max_halo(tile) : fused_max_halo(tv, B);
    if (maxh < 2) return 0;
    int K = std::min(maxh - 1, default_fuse(tv));
    if (fuse_k > 0) K = std::min(fuse_k, maxh - 1);
    K = std::min(K, kMaxFuse);
    return std::max(1, std::min(K, S));
}

// Kernel code of the dual-update kernels for this TV form and TVdenoise box.
int kernel_tv(int tv, int dual) { return dual == SCI_DUAL_CLIP ? kTvClip : tv; }

// S dual updates of FGP in fused launches of K updates each and a last one
// of the rest (S = 10, K = 6: 6 + 4).  (Even splits such as 4 + 3 + 3 were
// measured slower in the full solve: each launch pays its tile loads and
// stores, and the tile count's rounding to whole waves of CTAs decides more
// than the longest launch.)
template <typename T>
int enqueue_fused_prox(int tv, OuterMode mode, int K, int S, float lam, const std::vector<float>& coef,
                       FusedArgs base, FusedBufs<T> bufs, float* x_out_last, cudaStream_t s) {
    int launches = 0;
    for (int s0 = 0; s0 < S;) {
        const int k = std::min(K, S - s0);
        FusedArgs a = base;
        a.mode = mode;
        a.K = k;
        a.halo = k + 1;
        a.first = s0 == 0;
        a.last = s0 + k == S;
        a.lambda = lam;
        a.step = (float)(1.0 / ((tv == kTvClip ? kClipAlpha : 8.0) * (double)lam));
        for (int j = 0; j < k; ++j) a.coef[j] = coef[(size_t)(s0 + j)];
        a.x_out = a.last ? x_out_last : nullptr;
        if (!launch_fgp_fused<T>(tv, a, bufs, s)) return -1;
        ++launches;
        // the next launch reads what this one wrote, and writes the other set
        for (int j = 0; j < 4; ++j) {
            T* written = bufs.st_out[j];
            bufs.st_out[j] = const_cast<T*>(bufs.st_in[j]);
            bufs.st_in[j] = written;
        }
        s0 += k;
    }
    return launches;
}

// ---- the outer loop ----
struct SolveArgs {
    bool admm;
    bool fista;  // FISTA or TwIST outer loop (admm is then false)
    bool twist;  // TwIST's two-step update in place of FISTA's momentum (fista is then true)
    const float* y;
    const uint32_t* bits;
    int nx, ny, B;
    sci_params prm;
    float* theta;
    float* u;
    float* x_out;
    double* resid;
    int resid_every;
    void* work;
};

// Enqueues one solve; returns the number of kernels launched, or -1 if a
// fused launch could not be configured.
template <typename T>
int enqueue_solve(const SolveArgs& A, cudaStream_t s) {
    int nk = 0;
    const Geo g{A.nx, A.ny, A.B, (long long)A.nx * A.ny};
    const long long N = (long long)A.B * g.n;
    const bool warm = A.prm.warm_start != 0;
    const Layout L = solver_layout(A.nx, A.ny, A.B, A.prm.storage, A.admm, warm);
    char* w = static_cast<char*>(A.work);
    float* rinv = reinterpret_cast<float*>(w + L.rinv);
    float* r = reinterpret_cast<float*>(w + L.r);
    float* r_alt = reinterpret_cast<float*>(w + L.r2);
    double* partials = reinterpret_cast<double*>(w + L.partials);
    T* xt = reinterpret_cast<T*>(w + L.xt);
    T* P[4] = {reinterpret_cast<T*>(w + L.p[0]), reinterpret_cast<T*>(w + L.p[1]),
               reinterpret_cast<T*>(w + L.p[2]), reinterpret_cast<T*>(w + L.p[3])};
    const bool f32 = std::is_same<T, float>::value;
    T* theta = f32 ? reinterpret_cast<T*>(A.theta) : reinterpret_cast<T*>(w + L.theta_s);
    T* theta_alt = reinterpret_cast<T*>(w + L.theta_s2);
    T* u = nullptr;
    if (A.admm) u = f32 ? reinterpret_cast<T*>(A.u) : reinterpret_cast<T*>(w + L.u_s);
    T* const theta_home = theta;

    T* xprev = reinterpret_cast<T*>(w + L.xprev);
    unsigned* counts = reinterpret_cast<unsigned*>(w + L.lmax);  // [0] max mask count, [1] smallest nonzero
    const float* twist_w = reinterpret_cast<const float*>(w + L.lmax + 16);  // TwIST's three weights
    if (A.fista) {
        // z = theta + (1/L) Phi^T (y - Phi theta): the GAP residual with 1/L for 1/R
        launch_fista_step(A.bits, g, counts, rinv, s);
        launch_zero(xprev, (size_t)N * sizeof(T), s);
        nk += 2;
        if (A.twist) {
            launch_twist_coef(A.bits, g, counts, const_cast<float*>(twist_w), s);
            nk += 2;
        }
    } else {
        launch_rinv(A.bits, g, A.admm ? A.prm.rho : 0.f, rinv, s);
        ++nk;
    }
    // FISTA momentum coefficients (tau_t - 1)/tau_{t+1}, tau_1 = 1, in FP64
    std::vector<float> beta((size_t)std::max(A.prm.outer_iters, 1), 0.f);
    if (A.fista) {
        double tau = 1.0;
        for (int t = 0; t < A.prm.outer_iters; ++t) {
            const double next = (1.0 + std::sqrt(1.0 + 4.0 * tau * tau)) / 2.0;
            beta[(size_t)t] = (float)((tau - 1.0) / next);
            tau = next;
        }
    }
    // dual warm start: iteration t reads w from Wm[t % 2] and writes Wm[(t + 1) % 2];
    // the solve leaves its last w in Wm[0]
    T* Wm[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    if (warm) {
        T* wb = reinterpret_cast<T*>(w + L.warm);
        Wm[0][0] = wb;
        Wm[0][1] = wb + N;
        Wm[1][0] = wb + 2 * N;
        Wm[1][1] = wb + 3 * N;
        if (A.prm.init) launch_zero(Wm[0][0], (size_t)2 * N * sizeof(T), s);
    }
    int wpar = 0;
    if (A.prm.init) {
        launch_adjoint<T>(A.y, A.bits, g, theta, s);
        ++nk;
        if (A.admm) launch_zero(u, (size_t)N * sizeof(T), s);
    } else if (!f32) {
        launch_cast<float, T>(A.theta, theta, N, s);
        ++nk;
        if (A.admm) { launch_cast<float, T>(A.u, u, N, s); ++nk; }
    }
    const int T_outer = A.prm.outer_iters, S = A.prm.inner_iters;
    const float lam = A.prm.lambda;
    if (T_outer > 0) { launch_residual_field<T>(theta, u, A.y, A.bits, rinv, g, r, s); ++nk; }
    const std::vector<float> coef = momentum_coeffs(S, A.prm.dual);
    const OuterMode mode = A.admm ? OuterMode::Admm : OuterMode::Gap;
    const int nparts = out_partial_count(g);
    const int K = choose_fuse(A.prm.tv, A.B, S, A.prm.fuse_k, A.prm.tile);
    for (int t = 0; t < T_outer; ++t) {
        const bool last = t == T_outer - 1;
        const bool metric = A.resid != nullptr && A.resid_every > 0 && ((t + 1) % A.resid_every == 0);
        double* resid_slot = metric ? A.resid + ((t + 1) / A.resid_every - 1) : nullptr;
        if (K > 0) {
            // temporally blocked: ceil(S/K) fused launches, then the next residual
            FusedArgs base{};
            base.g = g;
            base.bits = A.bits;
            base.r = r;
            base.warm = warm ? 1 : 0;
            base.cls = A.prm.tile;
            // VTV tiles form the next residual in their last launch (GAP and ADMM)
            const bool fold_r = !last && !A.fista && A.prm.tv == SCI_TV_VTV;
            if (fold_r) {
                base.r_next = r_alt;
                base.y = A.y;
                base.rinv = rinv;
            }
            FusedBufs<T> fb{theta, u, theta_alt, u, xt,
                            {P[0], P[0] + N, P[1], P[1] + N}, {P[2], P[2] + N, P[3], P[3] + N},
                            {Wm[wpar][0], Wm[wpar][1]}, {Wm[wpar ^ 1][0], Wm[wpar ^ 1][1]}};
            wpar ^= 1;
            const int nf = enqueue_fused_prox<T>(kernel_tv(A.prm.tv, A.prm.dual), mode, K, S, lam, coef, base, fb,
                                                 (last && !A.fista) ? A.x_out : nullptr, s);
            if (nf < 0) return -1;
            nk += nf;
            if (A.twist) {
                // theta holds x^(t), theta_alt the TVdenoise output; x^(t+1) overwrites x^(t-1)
                launch_twist_step<T>(xprev, theta, theta_alt, twist_w, N, t == 0, s);
                ++nk;
                T* next = xprev;
                xprev = theta;
                theta = next;
                if (metric) { launch_residual_norm<T>(theta, A.y, A.bits, g, partials, resid_slot, s); nk += 2; }
                if (!last) { launch_residual_field<T>(theta, u, A.y, A.bits, rinv, g, r, s); ++nk; }
                continue;
            }
            std::swap(theta, theta_alt);
            if (fold_r) std::swap(r, r_alt);
            if (A.fista) {
                // theta holds x^(t); the residual metric is of x^(t)
                if (metric) { launch_residual_norm<T>(theta, A.y, A.bits, g, partials, resid_slot, s); nk += 2; }
                if (!last) {
                    launch_fista_momentum<T>(theta, xprev, theta_alt, N, beta[(size_t)t], s);
                    std::swap(theta, theta_alt);
                    launch_residual_field<T>(theta, u, A.y, A.bits, rinv, g, r, s);
                    nk += 2;
                }
                continue;
            }
            if (!last && !fold_r) { launch_residual_field<T>(theta, u, A.y, A.bits, rinv, g, r, s); ++nk; }
            if (metric) { launch_residual_norm<T>(theta, A.y, A.bits, g, partials, resid_slot, s); nk += 2; }
            continue;
        }
        launch_fgp_stream<T>(kernel_tv(A.prm.tv, A.prm.dual), mode, 1, nullptr, theta, r, A.bits, g, lam, 0.f, xt,
                             nullptr, nullptr,
                             P[0], s);
        ++nk;
        int cur = 0, prev = -1;
        for (int it = 1; it < S; ++it) {
            const int out = 3 - cur - (prev < 0 ? (cur == 0 ? 1 : 0) : prev);
            launch_fgp_stream<T>(kernel_tv(A.prm.tv, A.prm.dual), mode, 0, nullptr, theta, r, A.bits, g, lam,
                                 coef[(size_t)it - 1], xt,
                                 P[cur], prev >= 0 ? P[prev] : nullptr, P[out], s);
            ++nk;
            prev = cur;
            cur = out;
        }
        OutArgs oa{};
        oa.mode = mode;
        oa.y = A.y;
        oa.bits = A.bits;
        oa.rinv = rinv;
        oa.r_next = (last || A.fista) ? nullptr : r;
        oa.x_out = (last && f32 && !A.fista) ? A.x_out : nullptr;
        oa.resid_partials = metric ? partials : nullptr;
        if (last && !f32 && A.x_out != nullptr && A.admm) {
            // x = xt - u_old: stage u_old in FP32 through x_out before the output overwrites u
            launch_cast<T, float>(u, A.x_out, N, s);
            ++nk;
        }
        // TwIST keeps x^(t) beside the TVdenoise output
        launch_fgp_out<T>(oa, xt, P[cur], g, lam, A.twist ? theta_alt : theta, u, s);
        ++nk;
        if (last && !f32 && A.x_out != nullptr && !A.fista) {
            launch_xt_minus(xt, A.prm.storage, A.x_out, N, A.admm, s);
            ++nk;
        }
        if (A.twist) {
            launch_twist_step<T>(xprev, theta, theta_alt, twist_w, N, t == 0, s);
            ++nk;
            T* next = xprev;
            xprev = theta;
            theta = next;
            if (metric) { launch_residual_norm<T>(theta, A.y, A.bits, g, partials, resid_slot, s); nk += 2; }
            if (!last) { launch_residual_field<T>(theta, u, A.y, A.bits, rinv, g, r, s); ++nk; }
            continue;
        }
        if (metric) { launch_sum_partials(partials, nparts, resid_slot, s); ++nk; }
        if (A.fista && !last) {
            launch_fista_momentum<T>(theta, xprev, theta_alt, N, beta[(size_t)t], s);
            std::swap(theta, theta_alt);
            launch_residual_field<T>(theta, u, A.y, A.bits, rinv, g, r, s);
            nk += 2;
        }
    }
    if (warm && wpar == 1)
        cudaMemcpyAsync(Wm[0][0], Wm[1][0], (size_t)2 * N * sizeof(T), cudaMemcpyDeviceToDevice, s);
    if (!f32) {
        launch_cast<T, float>(theta, A.theta, N, s);
        ++nk;
        if (A.admm) { launch_cast<T, float>(u, A.u, N, s); ++nk; }
    } else if (theta != theta_home) {
        cudaMemcpyAsync(theta_home, theta, (size_t)N * sizeof(T), cudaMemcpyDeviceToDevice, s);
    }
    // FISTA's and TwIST's estimate is x^(T), held in theta
    if ((T_outer == 0 || A.fista) && A.x_out != nullptr)
        cudaMemcpyAsync(A.x_out, A.theta, (size_t)N * 4, cudaMemcpyDeviceToDevice, s);
    return nk;
}

int enqueue_solve_any(const SolveArgs& A, cudaStream_t s) {
    switch (A.prm.storage) {
        case SCI_BF16: return enqueue_solve<__nv_bfloat16>(A, s);
        case SCI_F16: return enqueue_solve<__half>(A, s);
        default: return enqueue_solve<float>(A, s);
    }
}

thread_local long long g_last_launches = 0;

// ---- CUDA graph cache: one instantiated graph per distinct solve call ----
struct GraphEntry {
    int device;
    SolveArgs args;
    cudaGraphExec_t exec;
    int launches;
};
std::mutex g_mu;
std::list<GraphEntry> g_cache;  // most recent first
constexpr size_t kMaxGraphs = 16;
cudaStream_t g_capture_stream[64] = {};

bool same_args(const SolveArgs& a, const SolveArgs& b) {
    return a.admm == b.admm && a.fista == b.fista && a.twist == b.twist && a.y == b.y && a.bits == b.bits && a.nx == b.nx && a.ny == b.ny &&
           a.B == b.B && std::memcmp(&a.prm, &b.prm, sizeof(sci_params)) == 0 && a.theta == b.theta &&
           a.u == b.u && a.x_out == b.x_out && a.resid == b.resid && a.resid_every == b.resid_every &&
           a.work == b.work;
}

sci_status run_solve(const SolveArgs& A, cudaStream_t stream) {
    if (cudaGetLastError() != cudaSuccess) { /* clear a stale error from earlier calls */ }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return SCI_ERR_CUDA;
    if (!A.prm.use_graph || cap != cudaStreamCaptureStatusNone) {
        const int nk = enqueue_solve_any(A, stream);
        if (nk < 0) return SCI_ERR_CUDA;
        g_last_launches = nk;
        return check_launch();
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SCI_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto it = g_cache.begin(); it != g_cache.end(); ++it) {
        if (it->device == dev && same_args(it->args, A)) {
            g_cache.splice(g_cache.begin(), g_cache, it);
            if (cudaGraphLaunch(g_cache.front().exec, stream) != cudaSuccess) return SCI_ERR_CUDA;
            g_last_launches = g_cache.front().launches;
            return SCI_OK;
        }
    }
    if (g_capture_stream[dev] == nullptr &&
        cudaStreamCreateWithFlags(&g_capture_stream[dev], cudaStreamNonBlocking) != cudaSuccess)
        return SCI_ERR_CUDA;
    cudaStream_t cs = g_capture_stream[dev];
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SCI_ERR_CUDA;
    const int nk = enqueue_solve_any(A, cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t launch_err = cudaGetLastError();
    if (cudaStreamEndCapture(cs, &graph) != cudaSuccess || launch_err != cudaSuccess || nk < 0) {
        if (graph) cudaGraphDestroy(graph);
        return SCI_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return SCI_ERR_CUDA;
    g_cache.push_front(GraphEntry{dev, A, exec, nk});
    while (g_cache.size() > kMaxGraphs) {
        cudaGraphExecDestroy(g_cache.back().exec);
        g_cache.pop_back();
    }
    if (cudaGraphLaunch(exec, stream) != cudaSuccess) return SCI_ERR_CUDA;
    g_last_launches = nk;
    return SCI_OK;
}

sci_status solve_common(bool admm, const float* y, const uint32_t* bits, int nx, int ny, int B,
                        const sci_params* params, float* theta, float* u, float* x_out,
                        double* resid, int resid_every, void* work, size_t work_bytes,
                        sci_stream_t stream, bool fista = false, bool twist = false) {
    if (y == nullptr || bits == nullptr || theta == nullptr || (admm && u == nullptr)) return SCI_ERR_ARG;
    if (!sizes_ok(nx, ny, B)) return SCI_ERR_ARG;
    if (B > 32) return SCI_ERR_SHAPE;
    sci_status st = validate_params(params, admm);
    if (st != SCI_OK) return st;
    if (resid_every < 0 || (resid_every > 0 && resid == nullptr)) return SCI_ERR_ARG;
    if (params->tile != 0 && !fused_class_fits(params->tv, B, params->tile)) return SCI_ERR_ARG;
    // the dual warm start runs on the temporally blocked path of GAP and ADMM only
    if (params->warm_start &&
        (fista || twist || choose_fuse(params->tv, B, params->inner_iters, params->fuse_k, params->tile) == 0))
        return SCI_ERR_ARG;
    const Layout L = solver_layout(nx, ny, B, params->storage, admm, params->warm_start != 0);
    st = validate_work(work, work_bytes, L.total);
    if (st != SCI_OK) return st;
    if (params->check_input) {
        const long long n = (long long)nx * ny, N = n * B;
        const float* arrays[3] = {y, params->init ? nullptr : theta, (params->init || !admm) ? nullptr : u};
        const long long sizes[3] = {n, N, N};
        st = check_inputs_finite(arrays, sizes, 3, reinterpret_cast<unsigned*>(static_cast<char*>(work) + L.lmax + 64),
                                 (cudaStream_t)stream);
        if (st != SCI_OK) return st;
    }
    SolveArgs A{admm, fista || twist, twist, y, bits, nx, ny, B, *params, theta, u, x_out, resid, resid_every, work};
    return run_solve(A, (cudaStream_t)stream);
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* sci_status_str(sci_status s) {
    switch (s) {
        case SCI_OK: return "ok";
        case SCI_ERR_ARG: return "invalid argument";
        case SCI_ERR_SHAPE: return "unsupported shape";
        case SCI_ERR_CUDA: return "CUDA error";
        case SCI_ERR_NONFINITE: return "non-finite argument";
        case SCI_ERR_TIMEOUT: return "device wait timed out";
        case SCI_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    }
    return "unknown status";
}

int sci_version(void) { return kVersion; }

sci_status sci_masks_pack(const uint8_t* masks, int nx, int ny, int B, uint32_t* bits, int* bad_count,
                          sci_stream_t stream) {
    if (masks == nullptr || bits == nullptr || !sizes_ok(nx, ny, B)) return SCI_ERR_ARG;
    if (B > 32) return SCI_ERR_SHAPE;
    launch_pack(masks, Geo{nx, ny, B, (long long)nx * ny}, bits, bad_count, (cudaStream_t)stream);
    return check_launch();
}

sci_status sci_forward(const float* x, const uint32_t* bits, int nx, int ny, int B, float* y,
                       sci_stream_t stream) {
    if (x == nullptr || bits == nullptr || y == nullptr || !sizes_ok(nx, ny, B)) return SCI_ERR_ARG;
    if (B > 32) return SCI_ERR_SHAPE;
    launch_forward(x, bits, Geo{nx, ny, B, (long long)nx * ny}, y, (cudaStream_t)stream);
    return check_launch();
}

sci_status sci_adjoint(const float* y, const uint32_t* bits, int nx, int ny, int B, float* x,
                       sci_stream_t stream) {
    if (x == nullptr || bits == nullptr || y == nullptr || !sizes_ok(nx, ny, B)) return SCI_ERR_ARG;
    if (B > 32) return SCI_ERR_SHAPE;
    launch_adjoint<float>(y, bits, Geo{nx, ny, B, (long long)nx * ny}, x, (cudaStream_t)stream);
    return check_launch();
}

sci_status sci_project(const float* theta, const float* u, const float* y, const uint32_t* bits, int nx,
                       int ny, int B, float rho, float* x, sci_stream_t stream) {
    if (theta == nullptr || y == nullptr || bits == nullptr || x == nullptr || !sizes_ok(nx, ny, B))
        return SCI_ERR_ARG;
    if (B > 32) return SCI_ERR_SHAPE;
    if (!std::isfinite(rho)) return SCI_ERR_NONFINITE;
    if (rho < 0.f || x == theta || (u != nullptr && x == u)) return SCI_ERR_ARG;
    launch_project(theta, u, y, bits, Geo{nx, ny, B, (long long)nx * ny}, rho, x, (cudaStream_t)stream);
    return check_launch();
}

size_t sci_tv_prox_workspace(int nx, int ny, int B, int tv) {
    (void)tv;
    if (!sizes_ok(nx, ny, B)) return 0;
    return prox_layout(nx, ny, B).total;
}

static sci_status tv_prox_impl(const float* x, int nx, int ny, int B, int tv, float lambda, int inner_iters,
                               float* theta, void* work, size_t work_bytes, sci_stream_t stream, int dual) {
    if (x == nullptr || theta == nullptr || x == theta || !sizes_ok(nx, ny, B)) return SCI_ERR_ARG;
    if (tv < SCI_TV_ATV || tv > SCI_TV_VTV || inner_iters < 1) return SCI_ERR_ARG;
    if (dual == SCI_DUAL_CLIP && tv != SCI_TV_ATV) return SCI_ERR_ARG;
    if (!std::isfinite(lambda)) return SCI_ERR_NONFINITE;
    if (!finite_pos(lambda)) return SCI_ERR_ARG;
    const Layout L = prox_layout(nx, ny, B);
    sci_status st = validate_work(work, work_bytes, L.total);
    if (st != SCI_OK) return st;
    const Geo g{nx, ny, B, (long long)nx * ny};
    cudaStream_t s = (cudaStream_t)stream;
    char* w = static_cast<char*>(work);
    float* P[4] = {reinterpret_cast<float*>(w + L.p[0]), reinterpret_cast<float*>(w + L.p[1]),
                   reinterpret_cast<float*>(w + L.p[2]), reinterpret_cast<float*>(w + L.p[3])};
    const std::vector<float> coef = momentum_coeffs(inner_iters, dual);
    const int K = choose_fuse(tv, B, inner_iters, 0);
    if (K > 0) {
        FusedArgs base{};
        base.g = g;
        base.xin = x;
        base.theta_f32 = theta;
        const size_t N = (size_t)B * nx * ny;
        FusedBufs<float> fb{nullptr, nullptr, nullptr, nullptr, nullptr,
                            {P[0], P[0] + N, P[1], P[1] + N}, {P[2], P[2] + N, P[3], P[3] + N}};
        if (enqueue_fused_prox<float>(kernel_tv(tv, dual), OuterMode::Prox, K, inner_iters, lambda, coef, base, fb,
                                      nullptr, s) < 0)
            return SCI_ERR_CUDA;
        return check_launch();
    }
    launch_fgp_stream<float>(kernel_tv(tv, dual), OuterMode::Prox, 1, x, nullptr, nullptr, nullptr, g, lambda, 0.f,
                             nullptr, nullptr, nullptr, P[0], s);
    int cur = 0, prev = -1;
    for (int it = 1; it < inner_iters; ++it) {
        const int out = 3 - cur - (prev < 0 ? (cur == 0 ? 1 : 0) : prev);
        launch_fgp_stream<float>(kernel_tv(tv, dual), OuterMode::Prox, 0, x, nullptr, nullptr, nullptr, g, lambda,
                                 coef[(size_t)it - 1], nullptr, P[cur], prev >= 0 ? P[prev] : nullptr, P[out], s);
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

sci_status sci_tv_prox(const float* x, int nx, int ny, int B, int tv, float lambda, int inner_iters,
                       float* theta, void* work, size_t work_bytes, sci_stream_t stream) {
    return tv_prox_impl(x, nx, ny, B, tv, lambda, inner_iters, theta, work, work_bytes, stream, SCI_DUAL_FGP);
}

sci_status sci_tv_prox_cham(const float* x, int nx, int ny, int B, int tv, float lambda, int inner_iters,
                            float* theta, void* work, size_t work_bytes, sci_stream_t stream) {
    return tv_prox_impl(x, nx, ny, B, tv, lambda, inner_iters, theta, work, work_bytes, stream, SCI_DUAL_CHAM);
}

sci_status sci_tv_prox_clip(const float* x, int nx, int ny, int B, int tv, float lambda, int inner_iters,
                            float* theta, void* work, size_t work_bytes, sci_stream_t stream) {
    return tv_prox_impl(x, nx, ny, B, tv, lambda, inner_iters, theta, work, work_bytes, stream, SCI_DUAL_CLIP);
}

size_t sci_solver_workspace(int nx, int ny, int B, const sci_params* params) {
    if (params == nullptr || !sizes_ok(nx, ny, B)) return 0;
    if (params->storage < SCI_F32 || params->storage > SCI_F16) return 0;
    return solver_layout(nx, ny, B, params->storage, true, params->warm_start != 0).total;
}

sci_status sci_gap_tv(const float* y, const uint32_t* bits, int nx, int ny, int B, const sci_params* params,
                      float* theta, float* x_out, double* resid, int resid_every, void* work,
                      size_t work_bytes, sci_stream_t stream) {
    return solve_common(false, y, bits, nx, ny, B, params, theta, nullptr, x_out, resid, resid_every, work,
                        work_bytes, stream);
}

sci_status sci_admm_tv(const float* y, const uint32_t* bits, int nx, int ny, int B, const sci_params* params,
                       float* theta, float* u, float* x_out, double* resid, int resid_every, void* work,
                       size_t work_bytes, sci_stream_t stream) {
    return solve_common(true, y, bits, nx, ny, B, params, theta, u, x_out, resid, resid_every, work,
                        work_bytes, stream);
}

sci_status sci_fista_tv(const float* y, const uint32_t* bits, int nx, int ny, int B, const sci_params* params,
                        float* theta, float* x_out, double* resid, int resid_every, void* work,
                        size_t work_bytes, sci_stream_t stream) {
    return solve_common(false, y, bits, nx, ny, B, params, theta, nullptr, x_out, resid, resid_every, work,
                        work_bytes, stream, true);
}

sci_status sci_twist_tv(const float* y, const uint32_t* bits, int nx, int ny, int B, const sci_params* params,
                        float* theta, float* x_out, double* resid, int resid_every, void* work,
                        size_t work_bytes, sci_stream_t stream) {
    return solve_common(false, y, bits, nx, ny, B, params, theta, nullptr, x_out, resid, resid_every, work,
                        work_bytes, stream, false, true);
}

void sci_graph_cache_clear(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto& e : g_cache) cudaGraphExecDestroy(e.exec);
    g_cache.clear();
}

long long sci_last_solve_launches(void) { return g_last_launches; }

int sci_fused_updates(int tv, int B, int inner_iters, int fuse_k) {
    if (tv < SCI_TV_ATV || tv > SCI_TV_VTV || B < 1 || inner_iters < 1 || fuse_k < -1) return -1;
    return choose_fuse(tv, B, inner_iters, fuse_k);
}

int sci_fused_updates_tile(int tv, int B, int inner_iters, int fuse_k, int tile) {
    if (tv < SCI_TV_ATV || tv > SCI_TV_VTV || B < 1 || inner_iters < 1 || fuse_k < -1) return -1;
    if (tile != 0 && (B > 32 || !fused_class_fits(tv, B, tile))) return -1;
    return choose_fuse(tv, B, inner_iters, fuse_k, tile);
}

int sci_tile_classes(int tv, int B, int* out, int max) {
    if (tv < SCI_TV_ATV || tv > SCI_TV_VTV || B < 1 || B > 32 || (out == nullptr && max > 0)) return 0;
    const int def = fused_class(tv, B);
    if (def == 0) return 0;
    int n = 0;
    auto put = [&](int c) {
        if (n < max) out[n] = c;
        ++n;
    };
    put(def);
    const int all[8] = {1, 2, 3, 4, 8, 10, 16, 24};
    for (int c : all)
        if (c != def && fused_class_fits(tv, B, c)) put(c);
    return n;
}

size_t sci_reduce_workspace(void) { return (size_t)kReduceParts * sizeof(double); }

sci_status sci_sqdiff_f64(const float* a, const float* b, size_t n, double* out, void* work,
                          size_t work_bytes, sci_stream_t stream) {
    if (a == nullptr || out == nullptr || n == 0) return SCI_ERR_ARG;
    sci_status st = validate_work(work, work_bytes, sci_reduce_workspace());
    if (st != SCI_OK) return st;
    launch_sqdiff(a, b, (long long)n, static_cast<double*>(work), out, (cudaStream_t)stream);
    return check_launch();
}

sci_status sci_residual_f64(const float* theta, const float* y, const uint32_t* bits, int nx, int ny, int B,
                            double* out, void* work, size_t work_bytes, sci_stream_t stream) {
    if (theta == nullptr || y == nullptr || bits == nullptr || out == nullptr || !sizes_ok(nx, ny, B))
        return SCI_ERR_ARG;
    if (B > 32) return SCI_ERR_SHAPE;
    sci_status st = validate_work(work, work_bytes, sci_reduce_workspace());
    if (st != SCI_OK) return st;
    launch_residual_norm<float>(theta, y, bits, Geo{nx, ny, B, (long long)nx * ny},
                                static_cast<double*>(work), out, (cudaStream_t)stream);
    return check_launch();
}

}  // extern "C"
