// render_fwd.cu -- the forward render kernels (a7-a9) and their launchers, plus the debug
// kernels that expose the FP32 ray and hit-test sequences to the tests.
#include <algorithm>

#include "trace.cuh"

namespace rs {

// The best-first forward (traversal 2, and the eps2 estimator) with K = 32 keeps its pending hits
// in shared memory (SmemKbuf) instead of registers: 85 registers instead of 128, so 6 CTAs of 4
// warps per SM instead of 4.  It does not stage top nodes (the rings take that shared memory).
constexpr bool kFwdSmemKbuf = true;

// dynamic shared memory of a forward launch: staged top nodes, or the warps' k-buffer rings
template <int K>
static size_t ring_smem_bytes(int block) { return (size_t)(block / 32) * K * 32 * sizeof(int64_t); }

template <int K, bool PERSIST, bool COUNT, int MODE, bool EPS2 = false, bool SMEMK = false>
__global__ void __launch_bounds__(128, SMEMK ? 6 : 4) k_render_fwd(FwdArgs A) {
    extern __shared__ float4 s_top[];
    if (MODE != 3 && !SMEMK)
        for (int i = threadIdx.x; i < 4 * A.n_top; i += blockDim.x) s_top[i] = A.top[i];
    __syncthreads();
    const NodeSrc ns{A.nodes, s_top, (MODE != 3 && !SMEMK && A.n_top > 0) ? kTopRef : 0, A.wide, A.P.n_nodes, A.n_top,
                     A.P.n_gauss, A.err};
    const int lane = threadIdx.x & 31;
    int64_t* kb_col = nullptr;  // this lane's column of its warp's ring block
    if (SMEMK) kb_col = reinterpret_cast<int64_t*>(s_top) + (threadIdx.x >> 5) * (K * 32) + lane;
    int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    Counters cnt;
    uint32_t rays = 0;
    while (true) {
        if (PERSIST) {
            unsigned long long t = 0;
            if (lane == 0) t = atomicAdd(A.queue, 1ull);
            tile = (int64_t)__shfl_sync(0xffffffffu, t, 0);
        }
        if (tile >= A.total_tiles) break;
        DevCam cam;
        int px, py;
        int64_t pix;
        const bool valid = tile_pixel(A, tile, lane, cam, px, py, pix);
        float C0, C1, C2, T, depth;
        int64_t last_key;
        int count;
        float3 o, d;
        camera_ray(cam, px, py, o, d);
        if (MODE == 3)
            trace_forward_bf<K, COUNT, 4>(A.rec, A.sph, ns, A.P, pix, valid, o, d, C0, C1, C2, T, depth, last_key, count,
                                          cnt, A.err);
        else if (MODE == 2 && SMEMK)
            trace_forward_bf<K, COUNT, 2, EPS2, false, true>(A.rec, A.sph, ns, A.P, pix, valid, o, d, C0, C1, C2, T, depth,
                                                             last_key, count, cnt, A.err,
                                                             SegRange{0.f, kEmptyKey, 0, true}, kb_col);
        else if (MODE == 2)
            trace_forward_bf<K, COUNT, 2, EPS2>(A.rec, A.sph, ns, A.P, pix, valid, o, d, C0, C1, C2, T, depth, last_key, count,
                                          cnt, A.err);
        else if (MODE == 1)
            trace_forward_packet<K, COUNT>(A.rec, A.sph, ns, A.P, pix, valid, o, d, C0, C1, C2, T, depth, last_key, count,
                                           cnt, A.err);
        else if (valid)
            trace_forward<K, COUNT>(A.rec, A.sph, ns, A.P, pix, o, d, C0, C1, C2, T, depth, last_key, count, cnt, A.err);
        if (valid) {
            A.rgb[3 * pix + 0] = fmaf(T, A.P.bg[0], C0);
            A.rgb[3 * pix + 1] = fmaf(T, A.P.bg[1], C1);
            A.rgb[3 * pix + 2] = fmaf(T, A.P.bg[2], C2);
            A.alpha[pix] = 1.f - T;
            if (A.depth) A.depth[pix] = depth;
            A.sT[pix] = T;
            A.skey[pix] = last_key;
            A.sn[pix] = count;
            if (COUNT) ++rays;
        }
        if (!PERSIST) break;
    }
    if (COUNT) {
        unsigned long long v[kNumStats] = {rays, cnt.nodes, cnt.tests, cnt.hits, cnt.rounds,
                                           cnt.inserted, 0, 0, cnt.wnodes, cnt.wleaf};
#pragma unroll
        for (int k = 0; k < kNumStats; ++k) {
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], s);
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < kNumStats; ++k)
                if (v[k]) atomicAdd(A.stats + k, v[k]);
        }
    }
}

__global__ void k_debug_rays(const DevCam* cams, int64_t n, const int32_t* ci, const int32_t* px, const int32_t* py,
                             float* o, float* d) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    float3 oo, dd;
    camera_ray(cams[ci[r]], px[r], py[r], oo, dd);
    o[3 * r] = oo.x; o[3 * r + 1] = oo.y; o[3 * r + 2] = oo.z;
    d[3 * r] = dd.x; d[3 * r + 1] = dd.y; d[3 * r + 2] = dd.z;
}

__global__ void k_debug_hits(const float4* rec, int64_t n_gauss, int64_t n_pairs, const float* ro, const float* rd,
                             const int32_t* sj, float Q, float t_near, float* out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_pairs) return;
    float* o = out + 8 * k;
    const int j = sj[k];
    if (j < 0 || j >= n_gauss) {  // out-of-range id: report NaN instead of reading
        for (int c = 0; c < 8; ++c) o[c] = __int_as_float(0x7fc00000);
        return;
    }
    Hit h;
    ray_ellipsoid<false>(make_float3(ro[3 * k], ro[3 * k + 1], ro[3 * k + 2]),
                         make_float3(rd[3 * k], rd[3 * k + 1], rd[3 * k + 2]), rec[4 * j], rec[4 * j + 1],
                         rec[4 * j + 2], Q, t_near, h);
    o[0] = h.D2;
    o[1] = h.t1;
    o[2] = h.hit ? 1.f : 0.f;
    o[3] = response_alpha(rec[4 * j + 3].x, h.D2);
    // the ordering keys' sub-ulp residuals, decoded to units of ulp of their high half: the
    // centre of the residual's bin (sort key 0: t1; sort key 1: max(t_m, t1))
    const int jb = key_id_bits((int)n_gauss), sb = 32 - jb;
    const uint32_t smask = (1u << sb) - 1u;
    const double bins = (double)(1ull << sb);
    const uint32_t sub = h.hit ? (uint32_t)((uint64_t)hit_key(h, 0, j, jb) >> jb) & smask : 0u;
    const uint32_t subm = h.hit ? (uint32_t)((uint64_t)hit_key(h, 1, j, jb) >> jb) & smask : 0u;
    o[4] = h.hit ? (float)(((double)sub + 0.5) / bins - 0.5) : 0.f;
    o[5] = (float)sb;
    o[6] = hit_key_t(h, 1);
    o[7] = h.hit ? (float)(((double)subm + 0.5) / bins - 0.5) : 0.f;
}


// ---------------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------------
static size_t smem_bytes(int n_top) { return (size_t)n_top * 4 * sizeof(float4); }

template <int K, bool COUNT, int MODE>
static int occupancy_fwd(int block, size_t smem) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_fwd<K, true, COUNT, MODE>, block, smem);
    return nb;
}

template <int K, bool COUNT>
static int occupancy_fwd_m(int block, int mode, size_t smem) {
    if (mode == 3) return occupancy_fwd<K, COUNT, 3>(block, 0);
    if constexpr (kFwdSmemKbuf && K == 32) {
        if (mode == 2) {  // the eps2 estimator's kernel has the same footprint
            int nb = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_fwd<K, true, COUNT, 2, false, true>, block,
                                                          ring_smem_bytes<K>(block));
            return nb;
        }
    }
    if (mode == 2) return occupancy_fwd<K, COUNT, 2>(block, smem);
    if (mode == 1) return occupancy_fwd<K, COUNT, 1>(block, smem);
    return occupancy_fwd<K, COUNT, 0>(block, smem);
}

int persistent_grid_fwd(int K, int block, bool count, int mode, int n_top, int sms) {
    const size_t sm = smem_bytes(n_top);
    int nb = 1;
    if (K == 8) nb = count ? occupancy_fwd_m<8, true>(block, mode, sm) : occupancy_fwd_m<8, false>(block, mode, sm);
    else if (K == 16) nb = count ? occupancy_fwd_m<16, true>(block, mode, sm) : occupancy_fwd_m<16, false>(block, mode, sm);
    else nb = count ? occupancy_fwd_m<32, true>(block, mode, sm) : occupancy_fwd_m<32, false>(block, mode, sm);
    return std::max(1, nb) * sms;
}

template <int K, bool PERSIST, bool COUNT>
static void launch_fwd_mode(const FwdArgs& A, int mode, int grid, int block, cudaStream_t st) {
    const size_t sm = smem_bytes(A.n_top);
    // the eps2 estimator's phase 2 is built into the best-first traversal only (every traversal
    // order gives the same result, so the order is a free choice)
    if constexpr (kFwdSmemKbuf && K == 32) {
        if (A.P.grad_mode == 1) {
            k_render_fwd<K, PERSIST, COUNT, 2, true, true><<<grid, block, ring_smem_bytes<K>(block), st>>>(A);
            return;
        }
        if (mode == 2) {
            k_render_fwd<K, PERSIST, COUNT, 2, false, true><<<grid, block, ring_smem_bytes<K>(block), st>>>(A);
            return;
        }
    }
    if (A.P.grad_mode == 1) k_render_fwd<K, PERSIST, COUNT, 2, true><<<grid, block, sm, st>>>(A);
    else if (mode == 3) k_render_fwd<K, PERSIST, COUNT, 3><<<grid, block, 0, st>>>(A);
    else if (mode == 2) k_render_fwd<K, PERSIST, COUNT, 2><<<grid, block, sm, st>>>(A);
    else if (mode == 1) k_render_fwd<K, PERSIST, COUNT, 1><<<grid, block, sm, st>>>(A);
    else k_render_fwd<K, PERSIST, COUNT, 0><<<grid, block, sm, st>>>(A);
}

template <int K>
static void launch_fwd_k(const FwdArgs& A, bool persistent, bool count, int mode, int grid, int block, cudaStream_t st) {
    if (persistent) {
        if (count) launch_fwd_mode<K, true, true>(A, mode, grid, block, st);
        else launch_fwd_mode<K, true, false>(A, mode, grid, block, st);
    } else {
        if (count) launch_fwd_mode<K, false, true>(A, mode, grid, block, st);
        else launch_fwd_mode<K, false, false>(A, mode, grid, block, st);
    }
}

cudaError_t launch_forward(const FwdArgs& A, int K, bool persistent, bool count, int mode, int grid, int block,
                           cudaStream_t st) {
    if (K == 8) launch_fwd_k<8>(A, persistent, count, mode, grid, block, st);
    else if (K == 16) launch_fwd_k<16>(A, persistent, count, mode, grid, block, st);
    else if (K == 32) launch_fwd_k<32>(A, persistent, count, mode, grid, block, st);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_debug_rays(const DevCam* cams, int64_t n, const int32_t* ci, const int32_t* px, const int32_t* py,
                              float* o, float* d, cudaStream_t st) {
    k_debug_rays<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(cams, n, ci, px, py, o, d);
    return cudaGetLastError();
}

cudaError_t launch_debug_hits(const float4* rec, int64_t n_gauss, int64_t n, const float* ro, const float* rd,
                              const int32_t* sj, float Q, float t_near, float* out, cudaStream_t st) {
    k_debug_hits<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(rec, n_gauss, n, ro, rd, sj, Q, t_near, out);
    return cudaGetLastError();
}

}  // namespace rs
