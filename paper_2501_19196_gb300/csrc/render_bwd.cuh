// render_bwd.cuh -- the adjoint kernels (a10) and their templated launchers, shared by
// render_bwd.cu (DEPTH = false, and the entry points) and render_bwd_depth.cu (DEPTH = true):
// the two halves of the kernel instantiations compile in parallel.
#pragma once
#include <algorithm>

#include "trace.cuh"

namespace rs {

// List replay (adjoint, first launch): one warp per ray tile of the forward pass; every ray
// whose hits all fit in its hit list is replayed from it (replay_list).  A tile holding a ray
// with more hits is appended to the overflow list, which k_render_bwd re-traverses next.
// Dynamic shared memory: the threads' gradient staging slots (list_stage_bytes).
static size_t list_stage_bytes(int block) { return (size_t)block * BulkScatter::kFloat4 * sizeof(float4); }

template <bool PERSIST, bool COUNT, bool DEPTH>
__global__ void __launch_bounds__(128, 8) k_replay_list(FwdArgs A, BwdArgs B) {
    extern __shared__ float4 s_stage[];
    BulkScatter sc(s_stage + BulkScatter::kFloat4 * threadIdx.x);
    const int lane = threadIdx.x & 31;
    int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    Counters cnt;
    uint32_t rays = 0;
    uint64_t listed = 0;
    while (true) {
        if (PERSIST) {
            unsigned long long t = 0;
            if (lane == 0) t = atomicAdd(A.queue + 1, 1ull);
            tile = (int64_t)__shfl_sync(0xffffffffu, t, 0);
        }
        if (tile >= A.total_tiles) break;
        DevCam cam;
        int px, py;
        int64_t pix;
        const bool valid = tile_pixel(A, tile, lane, cam, px, py, pix);
        const int n = valid ? A.sn[pix] : 0;
        const int nl = n <= A.P.list_cap ? n : 0;
        float3 o, d;
        camera_ray(cam, px, py, o, d);
        Upstream g{{0.f, 0.f, 0.f}, 0.f, 0.f, {0.f, 0.f, 0.f, -1.f}};
        float Tf = 1.f;
        if (nl > 0) {
            g.c[0] = B.d_rgb[3 * pix];
            g.c[1] = B.d_rgb[3 * pix + 1];
            g.c[2] = B.d_rgb[3 * pix + 2];
            g.a = B.d_alpha ? B.d_alpha[pix] : 0.f;
            g.d = DEPTH ? B.d_depth[pix] : 0.f;
            if (A.P.grad_mode == 1) {
                const float4 o = A.P.sS[pix];
                g.o[0] = o.x;
                g.o[1] = o.y;
                g.o[2] = o.z;
                g.o[3] = o.w;
            }
            Tf = A.sT[pix];
        }
        if (COUNT && n > 0) ++rays;
        if (COUNT) listed += nl;
        replay_list<COUNT, DEPTH>(A.rec, A.P, pix, o, d, Tf, nl, g, B.gtmp, cnt, A.err, sc);
        if (__any_sync(0xffffffffu, n > A.P.list_cap) && lane == 0) {
            const int64_t global = A.cam_single < 0 ? tile : A.cams[A.cam_single].tile_base + tile;
            const unsigned long long slot = atomicAdd(A.queue + 3, 1ull);
            if (slot < (unsigned long long)B.ovf_cap) B.ovf[slot] = (int)global;
            else atomicOr(A.err, kErrIndex);
        }
        if (!PERSIST) break;
    }
    sc.drain();
    if (COUNT) {
        unsigned long long v[kNumStats] = {rays, 0, 0, cnt.hits, 0, 0, 0, listed, 0, 0};
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

// The best-first re-traversal with K = 32 keeps its pending hits in shared-memory rings, as the
// forward does (SmemKbuf, descending): the register buffer held 64 of its 167 registers (3 CTAs
// of 4 warps per SM).  With the rings it runs 4 CTAs per SM at 123 registers without spills
// (measured 1.7x faster than the register buffer; 5 and 6 CTAs per SM spill and were slower).
// Each lane also keeps a list of 16 finalised keys in shared memory, replayed densely (48 KB per
// CTA with both).  It does not stage top nodes (the rings take that shared memory).
constexpr bool kBwdSmemKbuf = true;

// rings of K pending keys and lists of 16 finalised keys per lane
template <int K>
static size_t bwd_ring_smem_bytes(int block) { return (size_t)(block / 32) * (K + 16) * 32 * sizeof(int64_t); }

template <int K, bool PERSIST, bool COUNT, int MODE, bool DEPTH, bool SMEMK = false>
__global__ void __launch_bounds__(128, SMEMK ? 4 : 1) k_render_bwd(FwdArgs A, BwdArgs B) {
    extern __shared__ float4 s_top[];
    if (B.ovf && A.queue[3] == 0) return;  // every ray was replayed from its hit list
    if (MODE != 3 && !SMEMK)
        for (int i = threadIdx.x; i < 4 * A.n_top; i += blockDim.x) s_top[i] = A.top[i];
    __syncthreads();
    const NodeSrc ns{A.nodes, s_top, (MODE != 3 && !SMEMK && A.n_top > 0) ? kTopRef : 0, A.wide, A.P.n_nodes,
                     A.n_top, A.P.n_gauss, A.err};
    const int lane = threadIdx.x & 31;
    int64_t* kb_col = nullptr;  // this lane's column of its warp's ring block
    int64_t* fin_col = nullptr;  // this lane's column of its warp's finalised-key block
    if (SMEMK) {
        kb_col = reinterpret_cast<int64_t*>(s_top) + (threadIdx.x >> 5) * (K * 32) + lane;
        fin_col = reinterpret_cast<int64_t*>(s_top) + (blockDim.x >> 5) * (K * 32) + (threadIdx.x >> 5) * (16 * 32) + lane;
    }
    // with a hit list, only the tiles the list replay found overflowing are re-traversed
    const int64_t n_tiles = B.ovf ? (int64_t)min((unsigned long long)B.ovf_cap, A.queue[3]) : A.total_tiles;
    int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    Counters cnt;
    uint32_t rays = 0, retraced = 0;
    while (true) {
        if (PERSIST) {
            unsigned long long t = 0;
            if (lane == 0) t = atomicAdd(A.queue + 2, 1ull);
            tile = (int64_t)__shfl_sync(0xffffffffu, t, 0);
        }
        if (tile >= n_tiles) break;
        if (B.ovf) tile = B.ovf[tile];
        DevCam cam;
        int px, py;
        int64_t pix;
        const bool valid = tile_pixel(A, tile, lane, cam, px, py, pix);
        const int n = valid ? A.sn[pix] : 0;
        const int nt = n > A.P.list_cap ? n : 0;  // rays the hit list cannot replay
        float3 o, d;
        camera_ray(cam, px, py, o, d);
        Upstream g{{0.f, 0.f, 0.f}, 0.f, 0.f, {0.f, 0.f, 0.f, -1.f}};
        float Tf = 1.f;
        int64_t lk = -1;
        if (nt > 0) {
            g.c[0] = B.d_rgb[3 * pix];
            g.c[1] = B.d_rgb[3 * pix + 1];
            g.c[2] = B.d_rgb[3 * pix + 2];
            g.a = B.d_alpha ? B.d_alpha[pix] : 0.f;
            g.d = DEPTH ? B.d_depth[pix] : 0.f;
            if (A.P.grad_mode == 1) {
                const float4 o = A.P.sS[pix];
                g.o[0] = o.x;
                g.o[1] = o.y;
                g.o[2] = o.z;
                g.o[3] = o.w;
            }
            Tf = A.sT[pix];
            lk = A.skey[pix];
            if (COUNT) {
                ++retraced;
                if (A.P.list_cap == 0) ++rays;
            }
        }
        if (MODE == 3)
            trace_backward_bf<K, COUNT, 4, DEPTH>(A.rec, A.sph, ns, A.P, o, d, Tf, lk, nt, g, B.gtmp, cnt, A.err);
        else if (MODE == 2 && SMEMK)
            trace_backward_bf<K, COUNT, 2, DEPTH, true>(A.rec, A.sph, ns, A.P, o, d, Tf, lk, nt, g, B.gtmp, cnt, A.err,
                                                        kb_col, fin_col);
        else if (MODE == 2)
            trace_backward_bf<K, COUNT, 2, DEPTH>(A.rec, A.sph, ns, A.P, o, d, Tf, lk, nt, g, B.gtmp, cnt, A.err);
        else if (MODE == 1)
            trace_backward_packet<K, COUNT, DEPTH>(A.rec, A.sph, ns, A.P, o, d, Tf, lk, nt, g, B.gtmp, cnt, A.err);
        else if (nt > 0)
            trace_backward<K, COUNT, DEPTH>(A.rec, A.sph, ns, A.P, o, d, Tf, lk, nt, g, B.gtmp, cnt, A.err);
        if (!PERSIST) break;
    }
    if (COUNT) {
        unsigned long long v[kNumStats] = {rays,     cnt.nodes, cnt.tests, cnt.hits,   cnt.rounds,
                                           cnt.inserted, retraced, 0,        cnt.wnodes, cnt.wleaf};
#pragma unroll
        for (int k = 0; k < kNumStats; ++k) {
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], s);
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < kNumStats; ++k) atomicAdd(A.stats + k, v[k]);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------------
static size_t smem_bytes(int n_top) { return (size_t)n_top * 4 * sizeof(float4); }

template <int K, bool COUNT, int MODE, bool DEPTH>
static int occupancy_bwd(int block, size_t smem) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_bwd<K, true, COUNT, MODE, DEPTH>, block, smem);
    return nb;
}

template <int K, bool COUNT, bool DEPTH>
static int occupancy_bwd_m(int block, int mode, size_t smem) {
    if (mode == 3) return occupancy_bwd<K, COUNT, 3, DEPTH>(block, 0);
    if constexpr (kBwdSmemKbuf && K == 32) {
        if (mode == 2) {
            int nb = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_bwd<K, true, COUNT, 2, DEPTH, true>, block,
                                                          bwd_ring_smem_bytes<K>(block));
            return nb;
        }
    }
    if (mode == 2) return occupancy_bwd<K, COUNT, 2, DEPTH>(block, smem);
    if (mode == 1) return occupancy_bwd<K, COUNT, 1, DEPTH>(block, smem);
    return occupancy_bwd<K, COUNT, 0, DEPTH>(block, smem);
}

template <int K, bool DEPTH>
static int occupancy_bwd_k(int block, bool count, int mode, size_t smem) {
    return count ? occupancy_bwd_m<K, true, DEPTH>(block, mode, smem) : occupancy_bwd_m<K, false, DEPTH>(block, mode, smem);
}


template <int K, bool PERSIST, bool COUNT, bool DEPTH>
static void launch_bwd_mode(const FwdArgs& A, const BwdArgs& B, int mode, int grid, int block, cudaStream_t st) {
    const size_t sm = smem_bytes(A.n_top);
    if constexpr (kBwdSmemKbuf && K == 32) {
        if (mode == 2) {
            k_render_bwd<K, PERSIST, COUNT, 2, DEPTH, true><<<grid, block, bwd_ring_smem_bytes<K>(block), st>>>(A, B);
            return;
        }
    }
    if (mode == 3) k_render_bwd<K, PERSIST, COUNT, 3, DEPTH><<<grid, block, 0, st>>>(A, B);
    else if (mode == 2) k_render_bwd<K, PERSIST, COUNT, 2, DEPTH><<<grid, block, sm, st>>>(A, B);
    else if (mode == 1) k_render_bwd<K, PERSIST, COUNT, 1, DEPTH><<<grid, block, sm, st>>>(A, B);
    else k_render_bwd<K, PERSIST, COUNT, 0, DEPTH><<<grid, block, sm, st>>>(A, B);
}

template <int K, bool DEPTH>
static void launch_bwd_k(const FwdArgs& A, const BwdArgs& B, bool persistent, bool count, int mode, int grid, int block,
                         cudaStream_t st) {
    if (persistent) {
        if (count) launch_bwd_mode<K, true, true, DEPTH>(A, B, mode, grid, block, st);
        else launch_bwd_mode<K, true, false, DEPTH>(A, B, mode, grid, block, st);
    } else {
        if (count) launch_bwd_mode<K, false, true, DEPTH>(A, B, mode, grid, block, st);
        else launch_bwd_mode<K, false, false, DEPTH>(A, B, mode, grid, block, st);
    }
}

template <bool DEPTH>
static cudaError_t launch_bwd_d(const FwdArgs& A, const BwdArgs& B, int K, bool persistent, bool count, int mode,
                                int grid, int block, cudaStream_t st) {
    if (K == 8) launch_bwd_k<8, DEPTH>(A, B, persistent, count, mode, grid, block, st);
    else if (K == 16) launch_bwd_k<16, DEPTH>(A, B, persistent, count, mode, grid, block, st);
    else if (K == 32) launch_bwd_k<32, DEPTH>(A, B, persistent, count, mode, grid, block, st);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}


template <bool PERSIST, bool COUNT, bool DEPTH>
static int list_occupancy(int block) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_replay_list<PERSIST, COUNT, DEPTH>, block,
                                                  list_stage_bytes(block));
    return nb;
}


template <bool DEPTH>
static void launch_list_d(const FwdArgs& A, const BwdArgs& B, bool persistent, bool count, int grid, int block,
                          cudaStream_t st) {
    if (persistent) {
        if (count) k_replay_list<true, true, DEPTH><<<grid, block, list_stage_bytes(block), st>>>(A, B);
        else k_replay_list<true, false, DEPTH><<<grid, block, list_stage_bytes(block), st>>>(A, B);
    } else {
        if (count) k_replay_list<false, true, DEPTH><<<grid, block, list_stage_bytes(block), st>>>(A, B);
        else k_replay_list<false, false, DEPTH><<<grid, block, list_stage_bytes(block), st>>>(A, B);
    }
}

// the per-DEPTH halves of the entry points (render_bwd.cu dispatches on DEPTH)
template <bool DEPTH>
static int persistent_grid_bwd_d(int K, int block, bool count, int mode, int n_top, int sms) {
    const size_t sm = smem_bytes(n_top);
    int nb = 1;
    if (K == 8) nb = occupancy_bwd_k<8, DEPTH>(block, count, mode, sm);
    else if (K == 16) nb = occupancy_bwd_k<16, DEPTH>(block, count, mode, sm);
    else nb = occupancy_bwd_k<32, DEPTH>(block, count, mode, sm);
    return std::max(1, nb) * sms;
}

template <bool DEPTH>
static int list_replay_grid_d(bool count, int block, int sms) {
    const int nb = count ? list_occupancy<true, true, DEPTH>(block) : list_occupancy<true, false, DEPTH>(block);
    return std::max(1, nb) * sms;
}

// DEPTH = true, compiled in render_bwd_depth.cu
int persistent_grid_bwd_depth(int K, int block, bool count, int mode, int n_top, int sms);
cudaError_t launch_backward_depth(const FwdArgs& A, const BwdArgs& B, int K, bool persistent, bool count, int mode,
                                  int grid, int block, cudaStream_t st);
int list_replay_grid_depth(bool count, int block, int sms);
void launch_list_replay_depth(const FwdArgs& A, const BwdArgs& B, bool persistent, bool count, int grid, int block,
                              cudaStream_t st);

}  // namespace rs
