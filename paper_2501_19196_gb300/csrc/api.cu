// api.cu -- extern "C" entry points of include/raysplats.h: host-side validation, handle
// management (device buffers grown on demand and then reused), camera tables and launches.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rs_host.h"
#include "rs_internal.cuh"
#include "rs_render.h"

namespace rs {

static thread_local char g_err[512] = "";

rs_status set_error(rs_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

rs_status cuda_check(const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(RS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return RS_OK;
}

// Allocation-failure injection (rs_test_fail_alloc): when armed with n > 0, the n-th device
// allocation from then on fails with RS_ERR_OOM instead of calling cudaMalloc, and the hook disarms.
static int64_t g_fail_alloc_in = 0;
static bool injected_alloc_failure() {
    if (g_fail_alloc_in <= 0) return false;
    return --g_fail_alloc_in == 0;
}

rs_status device_realloc(void** p, size_t bytes) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    if (bytes == 0) bytes = 1;
    if (injected_alloc_failure())
        return set_error(RS_ERR_OOM, "injected allocation failure (rs_test_fail_alloc) of %lld bytes",
                         (long long)bytes);
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(RS_ERR_OOM, "cudaMalloc of %lld bytes failed", (long long)bytes);
    }
    return RS_OK;
}

// (re)allocate a device buffer of `count` elements, freeing the previous one
template <typename T>
static rs_status dmalloc(T*& p, int64_t count) {
    void* q = p;
    const rs_status st = device_realloc(&q, sizeof(T) * (size_t)(count > 0 ? count : 1));
    p = static_cast<T*>(q);
    return st;
}

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

static rs_status check_tune(const rs_tune_params* t, bool build) {
    if (!t) return set_error(RS_ERR_INVALID_ARG, "tune params are NULL");
    if (t->tile_w < 1 || t->tile_w > 32 || (32 % t->tile_w) != 0 || t->tile_h != 32 / t->tile_w)
        return set_error(RS_ERR_INVALID_ARG, "tile %dx%d: tile_w * tile_h must be 32", t->tile_w, t->tile_h);
    if (t->kbuf != 8 && t->kbuf != 16 && t->kbuf != 32)
        return set_error(RS_ERR_INVALID_ARG, "kbuf %d: must be 8, 16 or 32", t->kbuf);
    if (build && (t->leaf_size < 1 || t->leaf_size > 32))
        return set_error(RS_ERR_INVALID_ARG, "leaf_size %d: must be 1..32", t->leaf_size);
    if (build && t->morton_bits != 10 && t->morton_bits != 20 && t->morton_bits != 21)
        return set_error(RS_ERR_INVALID_ARG, "morton_bits %d: must be 10, 20 (extended) or 21", t->morton_bits);
    if (t->block_warps < 1 || t->block_warps > 4)
        return set_error(RS_ERR_INVALID_ARG, "block_warps %d: must be 1..4", t->block_warps);
    if (t->smem_nodes < 0 || t->smem_nodes > kMaxSmemNodes)
        return set_error(RS_ERR_INVALID_ARG, "smem_nodes %d: must be 0..%d", t->smem_nodes, kMaxSmemNodes);
    if (t->traversal < 0 || t->traversal > 3)
        return set_error(RS_ERR_INVALID_ARG, "traversal %d: must be 0 (per ray), 1 (warp packet), 2 (best-first "
                         "warp packet) or 3 (best-first warp packet over 4-wide nodes)", t->traversal);
    if (t->hit_list < 0 || t->hit_list > kMaxHitList)
        return set_error(RS_ERR_INVALID_ARG, "hit_list %d: must be 0..%d", t->hit_list, kMaxHitList);
    return RS_OK;
}

static rs_status check_gaussians(const rs_gaussians* g) {
    if (!g) return set_error(RS_ERR_INVALID_ARG, "gaussians are NULL");
    if (g->n < 1 || g->n > (int64_t)INT32_MAX / 4)
        return set_error(RS_ERR_INVALID_ARG, "n = %lld Gaussians: must be in [1, 2^29]", (long long)g->n);
    if (!g->means || !g->quats || !g->scales || !g->opacities || !g->rgb)
        return set_error(RS_ERR_INVALID_ARG, "a Gaussian parameter pointer is NULL");
    return RS_OK;
}

static bool finite(float x) { return std::isfinite(x); }

}  // namespace rs

using namespace rs;

extern "C" {

int32_t rs_abi_version(void) { return RS_ABI_VERSION; }

const char* rs_last_error(void) { return g_err; }

rs_status rs_default_tune(rs_tune_params* out) {
    if (!out) return set_error(RS_ERR_INVALID_ARG, "out is NULL");
    out->tile_w = 8;
    out->tile_h = 4;
    out->kbuf = 32;
    out->leaf_size = 32;
    out->morton_bits = 21;
    out->persistent = 1;
    out->block_warps = 4;
    out->traversal = 2;
    out->smem_nodes = 256;
    out->hit_list = 256;
    return RS_OK;
}

rs_status rs_test_fail_alloc(int64_t n) {
    if (n < 0) return set_error(RS_ERR_INVALID_ARG, "n = %lld must be >= 0", (long long)n);
    g_fail_alloc_in = n;
    return RS_OK;
}

rs_status rs_build_accel(const rs_gaussians* g, float Q_box, const rs_tune_params* tune, rs_accel** inout,
                         void* cuda_stream) {
    g_err[0] = 0;
    rs_status st = check_gaussians(g);
    if (st) return st;
    if ((st = check_tune(tune, true))) return st;
    if (!inout) return set_error(RS_ERR_INVALID_ARG, "accel handle pointer is NULL");
    if (!(Q_box > 0.f) || !finite(Q_box)) return set_error(RS_ERR_INVALID_ARG, "Q_box must be finite and > 0");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    rs_accel* A = *inout;
    if (!A) {
        A = new (std::nothrow) rs_accel();
        if (!A) return set_error(RS_ERR_OOM, "host allocation failed");
        cudaGetDevice(&A->device);
        if ((st = dmalloc(A->bounds, 6)) || (st = dmalloc(A->err, 1)) || (st = dmalloc(A->top, 4 * kMaxSmemNodes))) {
            if (A->bounds) cudaFree(A->bounds);
            if (A->err) cudaFree(A->err);
            if (A->top) cudaFree(A->top);
            delete A;
            return st;
        }
        cudaMemset(A->err, 0, sizeof(int));
        *inout = A;
    }
    const int64_t n = g->n;
    A->n = 0;  // unusable until this build succeeds (a failed (re)allocation leaves buffers missing)
    if (n > A->cap) {
        const int64_t cap = n;
        const int64_t nb = (cap + 2047) / 2048;
        if ((st = dmalloc(A->rec, 4 * cap)) || (st = dmalloc(A->pbox, 6 * cap)) || (st = dmalloc(A->sph, cap)) ||
            (st = dmalloc(A->keys[0], cap)) || (st = dmalloc(A->keys[1], cap)) || (st = dmalloc(A->vals[0], cap)) ||
            (st = dmalloc(A->vals[1], cap)) || (st = dmalloc(A->hist, 256 * nb)) || (st = dmalloc(A->left, cap)) ||
            (st = dmalloc(A->right, cap)) || (st = dmalloc(A->first, cap)) || (st = dmalloc(A->last, cap)) ||
            (st = dmalloc(A->parent, 2 * cap)) || (st = dmalloc(A->nbox, 6 * cap)) ||
            (st = dmalloc(A->counter, cap)) || (st = dmalloc(A->nodes, 4 * cap))) {
            A->cap = 0;
            return st;
        }
        A->cap = cap;
    }
    if (tune->traversal == 3 && (!A->wide || A->wide_cap < n)) {
        if ((st = dmalloc(A->wide, 8 * std::max<int64_t>(1, n)))) {
            A->wide_cap = 0;
            return st;
        }
        A->wide_cap = n;
    }
    A->has_wide = tune->traversal == 3;
    A->n = n;
    A->leaf_size = tune->leaf_size;
    A->morton_bits = tune->morton_bits;
    A->Q_box = Q_box;
    st = build_accel_device(*A, *g, *tune, s);
    if (st) A->n = 0;
    return st;
}

static rs_status render_impl(const rs_gaussians* g, const rs_accel* accel, const rs_camera* cams, int32_t n_cams,
                             const rs_render_params* p, const rs_tune_params* tune, rs_frame* out,
                             rs_fwd_state** inout_state, uint64_t* stats, void* cuda_stream) {
    g_err[0] = 0;
    rs_status st = check_gaussians(g);
    if (st) return st;
    if ((st = check_tune(tune, false))) return st;
    if (!accel || accel->n != g->n) return set_error(RS_ERR_INVALID_ARG, "accel is NULL or built for another n");
    if (tune->traversal == 3 && !accel->has_wide)
        return set_error(RS_ERR_INVALID_ARG, "traversal 3 needs an accel built with traversal 3 (4-wide nodes)");
    if (!cams || n_cams < 1) return set_error(RS_ERR_INVALID_ARG, "need at least one camera");
    if (!p) return set_error(RS_ERR_INVALID_ARG, "render params are NULL");
    if (!(p->Q > 0.f) || !(p->Q <= accel->Q_box))
        return set_error(RS_ERR_INVALID_ARG, "Q = %g must be in (0, Q_box = %g]", p->Q, accel->Q_box);
    if (!(p->eps1 >= 0.f) || !finite(p->eps1) || !(p->t_near >= 0.f) || !finite(p->t_near))
        return set_error(RS_ERR_INVALID_ARG, "eps1 and t_near must be finite and >= 0");
    if (p->k_max < 1) return set_error(RS_ERR_INVALID_ARG, "k_max must be >= 1");
    if (p->depth_mode != 0) return set_error(RS_ERR_UNSUPPORTED, "only depth_mode 0 is implemented");
    if (p->sort_key != 0 && p->sort_key != 1)
        return set_error(RS_ERR_INVALID_ARG, "sort_key %d: must be 0 (entry t1) or 1 (t_m)", p->sort_key);
    if (p->grad_mode != 0 && p->grad_mode != 1)
        return set_error(RS_ERR_INVALID_ARG, "grad_mode %d: must be 0 (exact) or 1 (eps2 estimator)", p->grad_mode);
    if (p->grad_mode == 1 && !(p->eps2 > 0.f && finite(p->eps2)))
        return set_error(RS_ERR_INVALID_ARG, "eps2 must be finite and > 0 with grad_mode 1");
    for (int k = 0; k < 3; ++k)
        if (!finite(p->background[k])) return set_error(RS_ERR_INVALID_ARG, "background must be finite");
    if (!out || !out->rgb || !out->alpha) return set_error(RS_ERR_INVALID_ARG, "output rgb/alpha are NULL");
    if (!inout_state) return set_error(RS_ERR_INVALID_ARG, "state handle pointer is NULL");
    // camera table
    const int tw = tune->tile_w, th = tune->tile_h;
    std::vector<DevCam> table((size_t)n_cams);
    int64_t tiles = 0, pix = 0;
    for (int c = 0; c < n_cams; ++c) {
        const rs_camera& C = cams[c];
        if (C.width < 1 || C.height < 1 || (int64_t)C.width * C.height >= ((int64_t)1 << 31))
            return set_error(RS_ERR_INVALID_ARG, "camera %d: bad size %dx%d", c, C.width, C.height);
        bool ok = finite(C.fx) && finite(C.fy) && finite(C.cx) && finite(C.cy) && C.fx != 0.f && C.fy != 0.f;
        for (int k = 0; k < 9; ++k) ok = ok && finite(C.R_wc[k]);
        for (int k = 0; k < 3; ++k) ok = ok && finite(C.pos[k]);
        if (!ok) return set_error(RS_ERR_INVALID_ARG, "camera %d: non-finite or zero-focal parameters", c);
        DevCam& D = table[(size_t)c];
        memcpy(D.R, C.R_wc, sizeof(D.R));
        memcpy(D.pos, C.pos, sizeof(D.pos));
        D.fx = C.fx;
        D.fy = C.fy;
        D.cx = C.cx;
        D.cy = C.cy;
        D.W = C.width;
        D.H = C.height;
        D.tiles_x = (C.width + tw - 1) / tw;
        D.tiles_y = (C.height + th - 1) / th;
        D.tile_base = tiles;
        D.pix_base = pix;
        tiles += (int64_t)D.tiles_x * D.tiles_y;
        pix += (int64_t)C.width * C.height;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    rs_fwd_state* S = *inout_state;
    if (!S) {
        S = new (std::nothrow) rs_fwd_state();
        if (!S) return set_error(RS_ERR_OOM, "host allocation failed");
        cudaGetDevice(&S->device);
        if ((st = dmalloc(S->queue, 4)) || (st = dmalloc(S->err, 1))) {
            if (S->queue) cudaFree(S->queue);
            if (S->err) cudaFree(S->err);
            delete S;
            return st;
        }
        cudaMemset(S->err, 0, sizeof(int));
        *inout_state = S;
    }
    S->n_pix = 0;  // holds no render until this forward is launched
    if (pix > S->cap_pix) {
        if ((st = dmalloc(S->sT, pix)) || (st = dmalloc(S->skey, pix)) || (st = dmalloc(S->sn, pix))) {
            S->cap_pix = 0;
            return st;
        }
        S->cap_pix = pix;
    }
    if (p->grad_mode == 1 && pix > S->cap_sS) {
        if ((st = dmalloc(S->sS, pix))) {
            S->cap_sS = 0;
            return st;
        }
        S->cap_sS = pix;
    }
    const int64_t n_ids = pix * tune->hit_list;
    if (n_ids > S->cap_ids) {
        if ((st = dmalloc(S->ids, n_ids))) {
            S->cap_ids = 0;
            return st;
        }
        S->cap_ids = n_ids;
    }
    if (n_cams > S->cap_cams) {
        if (S->cams_pinned) cudaFreeHost(S->cams_pinned);
        S->cams_pinned = nullptr;
        if (cudaMallocHost(&S->cams_pinned, sizeof(DevCam) * (size_t)n_cams) != cudaSuccess) {
            cudaGetLastError();
            S->cap_cams = 0;
            return set_error(RS_ERR_OOM, "pinned camera staging allocation failed");
        }
        if ((st = dmalloc(S->cams_dev, n_cams))) {
            S->cap_cams = 0;
            return st;
        }
        S->cap_cams = n_cams;
        S->cams_host.clear();
    }
    const bool same = S->cams_host.size() == table.size() &&
                      memcmp(S->cams_host.data(), table.data(), sizeof(DevCam) * table.size()) == 0;
    if (!same) {
        // the staging buffer may still feed an earlier in-flight upload
        if (!S->cams_host.empty()) cudaStreamSynchronize(s);
        memcpy(S->cams_pinned, table.data(), sizeof(DevCam) * table.size());
        if (cudaMemcpyAsync(S->cams_dev, S->cams_pinned, sizeof(DevCam) * table.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return cuda_check("camera upload");
        S->cams_host = table;
    }
    S->n_cams = n_cams;
    S->total_tiles = tiles;
    S->tile_w = tw;
    S->kbuf = tune->kbuf;
    S->block_warps = tune->block_warps;
    S->persistent = tune->persistent;
    S->accel = accel;
    S->n_gauss = g->n;
    TraceParams P;
    P.Q = p->Q;
    P.eps1 = p->eps1;
    P.t_near = p->t_near;
    P.bg[0] = p->background[0];
    P.bg[1] = p->background[1];
    P.bg[2] = p->background[2];
    P.k_max = p->k_max;
    P.max_rounds = (int32_t)std::min<int64_t>(INT32_MAX, g->n / tune->kbuf + 3);
    P.max_visits = (int32_t)std::min<int64_t>(INT32_MAX, 2 * g->n + 16);
    P.n_gauss = (int32_t)g->n;
    P.n_nodes = (int32_t)std::max<int64_t>(1, g->n - 1);
    P.list_cap = tune->hit_list;
    P.sort_key = p->sort_key;
    P.grad_mode = p->grad_mode;
    P.eps2 = p->eps2;
    P.sS = p->grad_mode == 1 ? S->sS : nullptr;
    P.ids = tune->hit_list > 0 ? S->ids : nullptr;
    S->P = P;

    FwdArgs A{};
    A.rec = accel->rec;
    A.sph = accel->sph;
    A.nodes = accel->nodes;
    A.top = accel->top;
    A.n_top = accel->n_top;
    A.wide = accel->wide;
    A.cams = S->cams_dev;
    A.n_cams = n_cams;
    A.tile_w = tw;
    A.P = P;
    A.rgb = out->rgb;
    A.alpha = out->alpha;
    A.depth = out->depth;
    A.sT = S->sT;
    A.skey = S->skey;
    A.sn = S->sn;
    A.queue = S->queue;
    A.err = accel->err;
    A.stats = reinterpret_cast<unsigned long long*>(stats);
    const int block = 32 * tune->block_warps;
    const bool count = stats != nullptr;
    if (tune->persistent) {
        A.cam_single = -1;
        A.total_tiles = tiles;
        if (cudaMemsetAsync(S->queue, 0, sizeof(unsigned long long), s) != cudaSuccess) return cuda_check("queue reset");
        const int grid = (int)std::min<int64_t>(
            persistent_grid_fwd(tune->kbuf, block, count, p->grad_mode == 1 ? 2 : tune->traversal, A.n_top,
                                sm_count()),
            (tiles + tune->block_warps - 1) / tune->block_warps);
        const cudaError_t e = launch_forward(A, tune->kbuf, true, count, tune->traversal, std::max(grid, 1),
                                             block, s);
        if (e != cudaSuccess) return set_error(RS_ERR_CUDA, "render launch: %s", cudaGetErrorString(e));
    } else {
        for (int c = 0; c < n_cams; ++c) {
            A.cam_single = c;
            A.total_tiles = (int64_t)table[(size_t)c].tiles_x * table[(size_t)c].tiles_y;
            const int grid = (int)((A.total_tiles + tune->block_warps - 1) / tune->block_warps);
            const cudaError_t e = launch_forward(A, tune->kbuf, false, count, tune->traversal, grid, block, s);
            if (e != cudaSuccess) return set_error(RS_ERR_CUDA, "render launch: %s", cudaGetErrorString(e));
        }
    }
    S->n_pix = pix;
    return RS_OK;
}

rs_status rs_render(const rs_gaussians* g, const rs_accel* accel, const rs_camera* cams, int32_t n_cams,
                    const rs_render_params* params, const rs_tune_params* tune, rs_frame* out,
                    rs_fwd_state** inout_state, void* cuda_stream) {
    return render_impl(g, accel, cams, n_cams, params, tune, out, inout_state, nullptr, cuda_stream);
}

rs_status rs_render_counted(const rs_gaussians* g, const rs_accel* accel, const rs_camera* cams, int32_t n_cams,
                            const rs_render_params* params, const rs_tune_params* tune, rs_frame* out,
                            rs_fwd_state** inout_state, uint64_t* stats_device, void* cuda_stream) {
    if (!stats_device) return set_error(RS_ERR_INVALID_ARG, "stats_device is NULL");
    return render_impl(g, accel, cams, n_cams, params, tune, out, inout_state, stats_device, cuda_stream);
}

static rs_status backward_impl(const rs_gaussians* g, const rs_accel* accel, const rs_fwd_state* state,
                               const rs_frame_grad* dl, const rs_tune_params* tune, rs_gaussian_grads* out,
                               uint64_t* stats, void* cuda_stream) {
    g_err[0] = 0;
    rs_status st = check_gaussians(g);
    if (st) return st;
    if ((st = check_tune(tune, false))) return st;
    if (!state || state->n_pix <= 0) return set_error(RS_ERR_INVALID_ARG, "state is NULL or holds no render");
    if (!accel || accel != state->accel || accel->n != g->n || state->n_gauss != g->n)
        return set_error(RS_ERR_INVALID_ARG, "accel / scene differ from the forward pass");
    if (tune->traversal == 3 && !accel->has_wide)
        return set_error(RS_ERR_INVALID_ARG, "traversal 3 needs an accel built with traversal 3 (4-wide nodes)");
    if (tune->tile_w != state->tile_w)
        return set_error(RS_ERR_INVALID_ARG, "tile shape differs from the forward pass");
    if (!dl || !dl->d_rgb) return set_error(RS_ERR_INVALID_ARG, "upstream gradient d_rgb is NULL");
    if (!out) return set_error(RS_ERR_INVALID_ARG, "gradient outputs are NULL");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    rs_fwd_state* S = const_cast<rs_fwd_state*>(state);
    if (g->n > S->cap_gauss) {
        if ((st = dmalloc(S->gtmp, 4 * g->n))) {
            S->cap_gauss = 0;
            return st;
        }
        S->cap_gauss = g->n;
    }
    const bool list = S->P.list_cap > 0;  // the forward recorded hit lists
    if (list && S->total_tiles > S->cap_ovf) {
        if ((st = dmalloc(S->ovf, S->total_tiles))) {
            S->cap_ovf = 0;
            return st;
        }
        S->cap_ovf = S->total_tiles;
    }
    if (cudaMemsetAsync(S->gtmp, 0, sizeof(float4) * 4 * (size_t)g->n, s) != cudaSuccess)
        return cuda_check("gradient scratch reset");
    FwdArgs A{};
    A.rec = accel->rec;
    A.sph = accel->sph;
    A.nodes = accel->nodes;
    A.top = accel->top;
    A.n_top = accel->n_top;
    A.wide = accel->wide;
    A.cams = S->cams_dev;
    A.n_cams = S->n_cams;
    A.tile_w = S->tile_w;
    A.P = S->P;
    A.sT = S->sT;
    A.skey = S->skey;
    A.sn = S->sn;
    A.queue = S->queue;
    A.err = accel->err;
    A.stats = reinterpret_cast<unsigned long long*>(stats);
    const bool count = stats != nullptr;
    BwdArgs B{dl->d_rgb, dl->d_alpha, dl->d_depth, S->gtmp, list ? S->ovf : nullptr, list ? S->cap_ovf : 0};
    const int block = 32 * tune->block_warps;
    if (cudaMemsetAsync(S->queue + 1, 0, 3 * sizeof(unsigned long long), s) != cudaSuccess)
        return cuda_check("queue reset");
    if (list) {
        // 1. replay every ray whose hits fit in its list; collect the tiles that overflow
        if (tune->persistent) {
            A.cam_single = -1;
            A.total_tiles = S->total_tiles;
            const int grid = (int)std::min<int64_t>(list_replay_grid(count, block, sm_count(), dl->d_depth != nullptr),
                                                    (S->total_tiles + tune->block_warps - 1) / tune->block_warps);
            const cudaError_t e = launch_list_replay(A, B, true, count, std::max(grid, 1), block, s);
            if (e != cudaSuccess) return set_error(RS_ERR_CUDA, "list replay launch: %s", cudaGetErrorString(e));
        } else {
            for (int c = 0; c < S->n_cams; ++c) {
                const DevCam& D = S->cams_host[(size_t)c];
                A.cam_single = c;
                A.total_tiles = (int64_t)D.tiles_x * D.tiles_y;
                const int grid = (int)((A.total_tiles + tune->block_warps - 1) / tune->block_warps);
                const cudaError_t e = launch_list_replay(A, B, false, count, grid, block, s);
                if (e != cudaSuccess) return set_error(RS_ERR_CUDA, "list replay launch: %s", cudaGetErrorString(e));
            }
        }
        // 2. re-traverse the overflow tiles (a persistent launch over the device-side list)
        A.cam_single = -1;
        A.total_tiles = S->total_tiles;
        const int grid = (int)std::min<int64_t>(
            persistent_grid_bwd(tune->kbuf, block, count, tune->traversal, A.n_top, sm_count(), dl->d_depth != nullptr),
            (S->total_tiles + tune->block_warps - 1) / tune->block_warps);
        const cudaError_t e = launch_backward(A, B, tune->kbuf, true, count, tune->traversal, std::max(grid, 1),
                                              block, s);
        if (e != cudaSuccess) return set_error(RS_ERR_CUDA, "backward launch: %s", cudaGetErrorString(e));
    } else if (tune->persistent) {
        A.cam_single = -1;
        A.total_tiles = S->total_tiles;
        const int grid = (int)std::min<int64_t>(
            persistent_grid_bwd(tune->kbuf, block, count, tune->traversal, A.n_top, sm_count(), dl->d_depth != nullptr),
            (S->total_tiles + tune->block_warps - 1) / tune->block_warps);
        const cudaError_t e = launch_backward(A, B, tune->kbuf, true, count, tune->traversal, std::max(grid, 1),
                                              block, s);
        if (e != cudaSuccess) return set_error(RS_ERR_CUDA, "backward launch: %s", cudaGetErrorString(e));
    } else {
        for (int c = 0; c < S->n_cams; ++c) {
            const DevCam& D = S->cams_host[(size_t)c];
            A.cam_single = c;
            A.total_tiles = (int64_t)D.tiles_x * D.tiles_y;
            const int grid = (int)((A.total_tiles + tune->block_warps - 1) / tune->block_warps);
            const cudaError_t e =
                launch_backward(A, B, tune->kbuf, false, count, tune->traversal, grid, block, s);
            if (e != cudaSuccess) return set_error(RS_ERR_CUDA, "backward launch: %s", cudaGetErrorString(e));
        }
    }
    const cudaError_t e = launch_finalize(S->gtmp, accel->rec, accel->vals[0], g->quats, g->scales, g->n, *out, s);
    if (e != cudaSuccess) return set_error(RS_ERR_CUDA, "finalize launch: %s", cudaGetErrorString(e));
    return RS_OK;
}

rs_status rs_render_backward(const rs_gaussians* g, const rs_accel* accel, const rs_fwd_state* state,
                             const rs_frame_grad* dl, const rs_tune_params* tune, rs_gaussian_grads* out,
                             void* cuda_stream) {
    return backward_impl(g, accel, state, dl, tune, out, nullptr, cuda_stream);
}

rs_status rs_render_backward_counted(const rs_gaussians* g, const rs_accel* accel, const rs_fwd_state* state,
                                     const rs_frame_grad* dl, const rs_tune_params* tune, rs_gaussian_grads* out,
                                     uint64_t* stats_device, void* cuda_stream) {
    if (!stats_device) return set_error(RS_ERR_INVALID_ARG, "stats_device is NULL");
    return backward_impl(g, accel, state, dl, tune, out, stats_device, cuda_stream);
}

rs_status rs_accel_destroy(rs_accel* A) {
    if (!A) return RS_OK;
    cudaDeviceSynchronize();
    void* ptrs[] = {A->rec,  A->pbox,  A->sph, A->keys[0], A->keys[1], A->vals[0], A->vals[1], A->hist,   A->bounds,
                    A->left, A->right, A->first,   A->last,    A->parent,  A->nbox,    A->counter, A->nodes,
                    A->top,  A->wide, A->err};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete A;
    return cuda_check("rs_accel_destroy");
}

rs_status rs_state_destroy(rs_fwd_state* S) {
    if (!S) return RS_OK;
    cudaDeviceSynchronize();
    void* ptrs[] = {S->cams_dev, S->sT, S->skey, S->sn, S->ids, S->sS, S->gtmp, S->ovf, S->queue, S->err};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (S->cams_pinned) cudaFreeHost(S->cams_pinned);
    delete S;
    return cuda_check("rs_state_destroy");
}

rs_status rs_check_device(const rs_accel* accel, const rs_fwd_state* state, void* cuda_stream) {
    g_err[0] = 0;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check("stream synchronize");
    int words[2] = {0, 0};
    if (accel && accel->err) {
        cudaMemcpy(&words[0], accel->err, sizeof(int), cudaMemcpyDeviceToHost);
        cudaMemset(accel->err, 0, sizeof(int));
    }
    if (state && state->err) {
        cudaMemcpy(&words[1], state->err, sizeof(int), cudaMemcpyDeviceToHost);
        cudaMemset(state->err, 0, sizeof(int));
    }
    rs_status st = cuda_check("device error word read");
    if (st) return st;
    const int w = words[0] | words[1];
    if (w) {
        return set_error(RS_ERR_INTERNAL, "device check failed (bits 0x%x:%s%s%s%s%s%s)", w,
                         (w & kErrReplayMismatch) ? " replay-mismatch" : "", (w & kErrBadScene) ? " bad-scene" : "",
                         (w & kErrStack) ? " stack-overflow" : "", (w & kErrLoopGuard) ? " loop-guard" : "",
                         (w & kErrIndex) ? " index-out-of-range" : "",
                         (w & kErrListOverflow) ? " id-list-overflow" : "");
    }
    return RS_OK;
}

rs_status rs_accel_export(const rs_accel* A, int64_t* n_out, uint64_t* codes, uint32_t* perm, int32_t* first,
                          int32_t* last, int32_t* split, float* boxes, float* prim_boxes, float* lo_hi) {
    g_err[0] = 0;
    if (!A) return set_error(RS_ERR_INVALID_ARG, "accel is NULL");
    if (A->n < 1) return set_error(RS_ERR_INVALID_ARG, "accel holds no successful build");
    if (cudaDeviceSynchronize() != cudaSuccess) return cuda_check("synchronize");
    const int64_t n = A->n;
    if (n_out) *n_out = n;
    if (codes) cudaMemcpy(codes, A->keys[0], sizeof(uint64_t) * n, cudaMemcpyDeviceToHost);
    if (perm) cudaMemcpy(perm, A->vals[0], sizeof(uint32_t) * n, cudaMemcpyDeviceToHost);
    if (n > 1) {
        if (first) cudaMemcpy(first, A->first, sizeof(int32_t) * (n - 1), cudaMemcpyDeviceToHost);
        if (last) cudaMemcpy(last, A->last, sizeof(int32_t) * (n - 1), cudaMemcpyDeviceToHost);
        if (split) {
            // split = the last position of the left child
            std::vector<int32_t> l((size_t)(n - 1)), f((size_t)(n - 1)), la((size_t)(n - 1));
            cudaMemcpy(l.data(), A->left, sizeof(int32_t) * (n - 1), cudaMemcpyDeviceToHost);
            for (int64_t i = 0; i < n - 1; ++i) split[i] = l[(size_t)i] < 0 ? ~l[(size_t)i] : l[(size_t)i];
        }
        if (boxes) cudaMemcpy(boxes, A->nbox, sizeof(float) * 6 * (n - 1), cudaMemcpyDeviceToHost);
    }
    if (prim_boxes) cudaMemcpy(prim_boxes, A->pbox, sizeof(float) * 6 * n, cudaMemcpyDeviceToHost);
    if (lo_hi) {
        unsigned b[6];
        cudaMemcpy(b, A->bounds, sizeof(b), cudaMemcpyDeviceToHost);
        for (int k = 0; k < 6; ++k) {
            const unsigned u = b[k];
            const unsigned bits = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
            memcpy(&lo_hi[k], &bits, 4);
        }
    }
    return cuda_check("rs_accel_export");
}

rs_status rs_debug_rays(const rs_camera* cams, int32_t n_cams, int64_t n_rays, const int32_t* cam_idx,
                        const int32_t* px, const int32_t* py, float* o, float* d, void* cuda_stream) {
    g_err[0] = 0;
    if (!cams || n_cams < 1 || n_rays < 0 || (n_rays > 0 && (!cam_idx || !px || !py || !o || !d)))
        return set_error(RS_ERR_INVALID_ARG, "bad arguments");
    if (n_rays == 0) return RS_OK;
    std::vector<DevCam> table((size_t)n_cams);
    for (int c = 0; c < n_cams; ++c) {
        memcpy(table[(size_t)c].R, cams[c].R_wc, sizeof(float) * 9);
        memcpy(table[(size_t)c].pos, cams[c].pos, sizeof(float) * 3);
        table[(size_t)c].fx = cams[c].fx;
        table[(size_t)c].fy = cams[c].fy;
        table[(size_t)c].cx = cams[c].cx;
        table[(size_t)c].cy = cams[c].cy;
        table[(size_t)c].W = cams[c].width;
        table[(size_t)c].H = cams[c].height;
    }
    DevCam* dc = nullptr;
    rs_status st = dmalloc(dc, n_cams);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaMemcpyAsync(dc, table.data(), sizeof(DevCam) * table.size(), cudaMemcpyHostToDevice, s);
    const cudaError_t e = launch_debug_rays(dc, n_rays, cam_idx, px, py, o, d, s);
    cudaStreamSynchronize(s);
    cudaFree(dc);
    if (e != cudaSuccess) return set_error(RS_ERR_CUDA, "debug rays: %s", cudaGetErrorString(e));
    return cuda_check("rs_debug_rays");
}

rs_status rs_debug_hits(const rs_accel* accel, int64_t n_pairs, const float* ray_o, const float* ray_d,
                        const int32_t* sorted_j, float Q, float t_near, float* out, void* cuda_stream) {
    g_err[0] = 0;
    if (!accel || accel->n < 1 || n_pairs < 0 || (n_pairs > 0 && (!ray_o || !ray_d || !sorted_j || !out)))
        return set_error(RS_ERR_INVALID_ARG, "bad arguments (or an accel without a successful build)");
    if (n_pairs == 0) return RS_OK;
    const cudaError_t e =
        launch_debug_hits(accel->rec, accel->n, n_pairs, ray_o, ray_d, sorted_j, Q, t_near, out, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return set_error(RS_ERR_CUDA, "debug hits: %s", cudaGetErrorString(e));
    return RS_OK;
}

rs_status rs_tune(const rs_gaussians* g, float Q_box, const rs_camera* cams, int32_t n_cams,
                  const rs_render_params* params, const rs_tune_params* candidates, int32_t n_candidates,
                  int32_t reps, rs_frame* scratch, const rs_frame_grad* dl, rs_gaussian_grads* scratch_grads,
                  rs_tune_params* best, float* ms_out, void* cuda_stream) {
    g_err[0] = 0;
    if (!candidates || n_candidates < 1 || reps < 1 || !best || !scratch)
        return set_error(RS_ERR_INVALID_ARG, "rs_tune: need candidates, reps >= 1, best and scratch");
    if (dl && !scratch_grads) return set_error(RS_ERR_INVALID_ARG, "rs_tune: dl given without scratch_grads");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_check("rs_tune event create");
    }
    float best_ms = -1.f;
    rs_status last = RS_ERR_INVALID_ARG;
    char first_err[512] = "";
    for (int c = 0; c < n_candidates; ++c) {
        const rs_tune_params& t = candidates[c];
        rs_accel* A = nullptr;
        rs_fwd_state* S = nullptr;
        float ms = -1.f;
        auto one = [&]() -> rs_status {
            rs_status st = rs_build_accel(g, Q_box, &t, &A, cuda_stream);
            if (st) return st;
            if ((st = rs_render(g, A, cams, n_cams, params, &t, scratch, &S, cuda_stream))) return st;
            if (dl) st = rs_render_backward(g, A, S, dl, &t, scratch_grads, cuda_stream);
            return st;
        };
        rs_status st = one();  // warm-up (allocates)
        if (!st) {
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && !st; ++r) st = one();
            cudaEventRecord(e1, s);
            if (!st && cudaEventSynchronize(e1) == cudaSuccess) {
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= (float)reps;
                if (!st) st = rs_check_device(A, S, cuda_stream);
            } else if (!st) {
                st = cuda_check("rs_tune timing");
            }
        }
        if (st) {
            if (!first_err[0]) snprintf(first_err, sizeof(first_err), "candidate %d: %s", c, g_err);
            last = st;
            ms = -1.f;
        }
        cudaStreamSynchronize(s);
        rs_state_destroy(S);
        rs_accel_destroy(A);
        if (ms_out) ms_out[c] = ms;
        if (ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
            best_ms = ms;
            *best = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms < 0.f) return set_error(last ? last : RS_ERR_INVALID_ARG, "rs_tune: no candidate ran (%s)", first_err);
    g_err[0] = 0;
    return RS_OK;
}

}  // extern "C"
