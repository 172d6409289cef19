// rs_render.h -- kernel argument blocks and launchers of render.cu (host + device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "rs_internal.cuh"

namespace rs {

struct FwdArgs {
    const float4* rec;
    const float4* sph;    // bounding spheres (Morton order)
    const float4* nodes;
    const float4* top;    // staged top nodes (n_top of them; root = kTopRef when n_top > 0)
    int n_top;
    const float4* wide;   // 4-wide nodes (traversal 3), 8 float4 per binary node index
    const DevCam* cams;
    int n_cams;
    int cam_single;       // >= 0: plain launch of this camera only; -1: persistent over all
    int64_t total_tiles;  // tiles of the launch (one camera, or all cameras)
    int tile_w;           // tile_h = 32 / tile_w
    TraceParams P;
    float* rgb;
    float* alpha;
    float* depth;
    float* sT;        // per pixel: final transmittance
    int64_t* skey;    // per pixel: (t1, sorted id) key of the last composited hit
    int* sn;          // per pixel: composited hits
    unsigned long long* queue;  // [0] forward tiles, [1] list-replay tiles, [2] re-traversal tiles,
                                // [3] overflow tiles appended by the list replay
    int* err;
    unsigned long long* stats;
};

struct BwdArgs {
    const float* d_rgb;
    const float* d_alpha;
    const float* d_depth;  // may be NULL
    float4* gtmp;  // 4 per Gaussian (Morton order): (dM row k, dm_k) k = 0..2, (dop, drgb)
    int* ovf;      // tiles (global ids) holding a ray with more hits than its hit list; NULL:
                   // the re-traversing adjoint covers every tile
    int64_t ovf_cap;
};

int persistent_grid_fwd(int K, int block, bool count, int mode, int n_top, int sms);
int persistent_grid_bwd(int K, int block, bool count, int mode, int n_top, int sms, bool depth);
int list_replay_grid(bool count, int block, int sms, bool depth);
cudaError_t launch_list_replay(const FwdArgs& A, const BwdArgs& B, bool persistent, bool count, int grid, int block,
                               cudaStream_t st);
cudaError_t launch_forward(const FwdArgs& A, int K, bool persistent, bool count, int mode, int grid, int block,
                           cudaStream_t st);
cudaError_t launch_backward(const FwdArgs& A, const BwdArgs& B, int K, bool persistent, bool count, int mode,
                            int grid, int block, cudaStream_t st);
cudaError_t launch_finalize(const float4* gtmp, const float4* rec, const uint32_t* perm, const float* quats,
                            const float* scales, int64_t n, const rs_gaussian_grads& out, cudaStream_t st);
cudaError_t launch_debug_rays(const DevCam* cams, int64_t n, const int32_t* ci, const int32_t* px,
                              const int32_t* py, float* o, float* d, cudaStream_t st);
cudaError_t launch_debug_hits(const float4* rec, int64_t n_gauss, int64_t n, const float* ro, const float* rd,
                              const int32_t* sj, float Q, float t_near, float* out, cudaStream_t st);

}  // namespace rs

struct rs_fwd_state {
    int device = 0;
    int64_t n_pix = 0, cap_pix = 0;
    int64_t cap_gauss = 0;
    int n_cams = 0, cap_cams = 0;
    std::vector<rs::DevCam> cams_host;  // last uploaded table
    rs::DevCam* cams_dev = nullptr;
    rs::DevCam* cams_pinned = nullptr;  // staging for the upload
    float* sT = nullptr;
    int64_t* skey = nullptr;
    int* sn = nullptr;
    int* ids = nullptr;                 // hit lists (hit_list ids per pixel)
    int64_t cap_ids = 0;
    float4* sS = nullptr;               // eps2 estimator: colour / alpha behind the last hit
    int64_t cap_sS = 0;
    float4* gtmp = nullptr;
    int* ovf = nullptr;                 // overflow tile list of the adjoint
    int64_t cap_ovf = 0;
    unsigned long long* queue = nullptr;
    int* err = nullptr;
    // what the forward recorded
    rs::TraceParams P{};
    int64_t total_tiles = 0;
    int tile_w = 8, kbuf = 16, block_warps = 4;
    int persistent = 1;
    int traversal = 1;
    const rs_accel* accel = nullptr;
    int64_t n_gauss = 0;
};
