// fixed_scratch.cu -- rs_render_fixed_scratch: a build + forward render that allocates nothing.
//
// Some callers cannot call cudaMalloc: plug-ins whose host application owns every device
// allocation (the plug-in gets buffers, never an allocator), and tools that run under a fixed
// device-memory budget and must not grow the process's footprint.  This entry point serves
// them: it takes the caller's scene, cameras and output buffers and keeps every intermediate
// (render records, boxes, sort buffers, tree, nodes, camera table, work counter, per-ray state)
// in one file-scope __device__ array of fixed size, shared by all calls on a device.
//
// Limits: n <= RS_FIXED_MAX_GAUSSIANS, sum of W*H <= RS_FIXED_MAX_PIXELS, n_cams <=
// RS_FIXED_MAX_CAMERAS; the array is about 12 MB and every GPU that loads the library holds
// it until the process exits.  The first call on a device resolves the array's device address
// (cudaGetSymbolAddress with that device current) and caches it for the life of the process;
// do not call the entry point again on a device after cudaDeviceReset (the cached address
// belongs to the context that was reset).
// Calls share the array and keep the previous call's contents, so calls that overlap on the
// GPU (different streams, or different host threads on the same device) race; the entry point
// itself clears everything that must start at zero.  The camera table travels as a kernel
// argument, so no host memory is read after the call returns.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "rs_host.h"
#include "rs_internal.cuh"
#include "rs_render.h"

namespace rs {
namespace fixed {

constexpr int64_t kN = RS_FIXED_MAX_GAUSSIANS;
constexpr int64_t kPix = RS_FIXED_MAX_PIXELS;
constexpr int kCams = RS_FIXED_MAX_CAMERAS;
constexpr int64_t kSortTile = 2048;
constexpr int64_t kBlocks = (kN + kSortTile - 1) / kSortTile;

constexpr int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }

// byte offsets of each region inside the array
constexpr int64_t oRec = 0;
constexpr int64_t oPbox = align256(oRec + 16 * 4 * kN);
constexpr int64_t oSph = align256(oPbox + 4 * 6 * kN);
constexpr int64_t oKeys0 = align256(oSph + 16 * kN);
constexpr int64_t oKeys1 = align256(oKeys0 + 8 * kN);
constexpr int64_t oVals0 = align256(oKeys1 + 8 * kN);
constexpr int64_t oVals1 = align256(oVals0 + 4 * kN);
constexpr int64_t oHist = align256(oVals1 + 4 * kN);
constexpr int64_t oBounds = align256(oHist + 4 * 256 * kBlocks);
constexpr int64_t oLeft = align256(oBounds + 4 * 6);
constexpr int64_t oRight = align256(oLeft + 4 * kN);
constexpr int64_t oFirst = align256(oRight + 4 * kN);
constexpr int64_t oLast = align256(oFirst + 4 * kN);
constexpr int64_t oParent = align256(oLast + 4 * kN);
constexpr int64_t oNbox = align256(oParent + 4 * 2 * kN);
constexpr int64_t oCounter = align256(oNbox + 4 * 6 * kN);
constexpr int64_t oNodes = align256(oCounter + 4 * kN);
constexpr int64_t oTop = align256(oNodes + 16 * 4 * kN);
constexpr int64_t oErr = align256(oTop + 16 * 4 * kMaxSmemNodes);
constexpr int64_t oCams = align256(oErr + 4);
constexpr int64_t oQueue = align256(oCams + (int64_t)sizeof(DevCam) * kCams);
constexpr int64_t oST = align256(oQueue + 16);
constexpr int64_t oSKey = align256(oST + 4 * kPix);
constexpr int64_t oSN = align256(oSKey + 8 * kPix);
constexpr int64_t kBytes = align256(oSN + 4 * kPix);

static __device__ __align__(256) unsigned char g_scratch[kBytes];

constexpr int kMaxDevices = 64;
static unsigned char* g_base[kMaxDevices] = {};
static std::mutex g_mu;

// The camera table, passed by value to a one-block kernel that writes it into the array.
struct CamTable {
    DevCam c[kCams];
};
static_assert(sizeof(CamTable) <= 4000, "the camera table must fit in a kernel's parameters");

__global__ void k_upload_cams(const CamTable t, int n, DevCam* __restrict__ dst) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = t.c[i];
}

// device address of g_scratch on the current device (resolved once per device)
static rs_status scratch_base(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_check("cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(RS_ERR_UNSUPPORTED, "device %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return set_error(RS_ERR_CUDA, "cudaGetSymbolAddress of the fixed scratch failed: %s", cudaGetErrorString(e));
        }
        g_base[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_base[dev];
    return RS_OK;
}

}  // namespace fixed
}  // namespace rs

using namespace rs;

extern "C" rs_status rs_render_fixed_scratch(const rs_gaussians* g, const rs_camera* cams, int32_t n_cams,
                                             const rs_render_params* p, const rs_tune_params* tune, rs_frame* out,
                                             void* cuda_stream) {
    using namespace rs::fixed;
    if (!g || !cams || !p || !tune || !out || !out->rgb || !out->alpha)
        return set_error(RS_ERR_INVALID_ARG, "rs_render_fixed_scratch: NULL argument");
    if (!g->means || !g->quats || !g->scales || !g->opacities || !g->rgb)
        return set_error(RS_ERR_INVALID_ARG, "a Gaussian parameter pointer is NULL");
    if (g->n < 1 || g->n > kN)
        return set_error(RS_ERR_INVALID_ARG, "n = %lld Gaussians: the fixed scratch holds 1..%lld", (long long)g->n,
                         (long long)kN);
    if (n_cams < 1 || n_cams > kCams)
        return set_error(RS_ERR_INVALID_ARG, "%d cameras: the fixed scratch holds 1..%d", n_cams, kCams);
    if (tune->tile_w < 1 || tune->tile_w > 32 || (32 % tune->tile_w) != 0 || tune->tile_h != 32 / tune->tile_w ||
        (tune->kbuf != 8 && tune->kbuf != 16 && tune->kbuf != 32) || tune->leaf_size < 1 || tune->leaf_size > 32 ||
        (tune->morton_bits != 10 && tune->morton_bits != 20 && tune->morton_bits != 21) || tune->block_warps < 1 ||
        tune->block_warps > 4 || tune->traversal < 0 || tune->traversal > 2 || tune->smem_nodes < 0 ||
        tune->smem_nodes > kMaxSmemNodes)
        return set_error(RS_ERR_INVALID_ARG, "bad tune parameters");
    if (!(p->Q > 0.f) || !std::isfinite(p->Q) || !(p->eps1 >= 0.f) || !std::isfinite(p->eps1) ||
        !(p->t_near >= 0.f) || !std::isfinite(p->t_near) || p->k_max < 1)
        return set_error(RS_ERR_INVALID_ARG, "bad render parameters");
    if (p->depth_mode != 0) return set_error(RS_ERR_UNSUPPORTED, "only depth_mode 0 is implemented");
    if (p->sort_key != 0 && p->sort_key != 1) return set_error(RS_ERR_INVALID_ARG, "sort_key must be 0 or 1");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(p->background[k])) return set_error(RS_ERR_INVALID_ARG, "background must be finite");
    CamTable table;
    memset(&table, 0, sizeof(table));
    int64_t tiles = 0, pix = 0;
    for (int c = 0; c < n_cams; ++c) {
        const rs_camera& C = cams[c];
        // each camera on its own first, so that no running total can overflow
        if (C.width < 1 || C.height < 1 || C.width > kPix || C.height > kPix ||
            (int64_t)C.width * C.height > kPix - pix)
            return set_error(RS_ERR_INVALID_ARG,
                             "camera %d: %dx%d pixels (after %lld): the fixed scratch holds at most %lld pixels", c,
                             C.width, C.height, (long long)pix, (long long)kPix);
        bool ok = std::isfinite(C.fx) && std::isfinite(C.fy) && std::isfinite(C.cx) && std::isfinite(C.cy) &&
                  C.fx != 0.f && C.fy != 0.f;
        for (int k = 0; k < 9; ++k) ok = ok && std::isfinite(C.R_wc[k]);
        for (int k = 0; k < 3; ++k) ok = ok && std::isfinite(C.pos[k]);
        if (!ok) return set_error(RS_ERR_INVALID_ARG, "camera %d: non-finite or zero-focal parameters", c);
        DevCam& D = table.c[c];
        memcpy(D.R, C.R_wc, sizeof(D.R));
        memcpy(D.pos, C.pos, sizeof(D.pos));
        D.fx = C.fx;
        D.fy = C.fy;
        D.cx = C.cx;
        D.cy = C.cy;
        D.W = C.width;
        D.H = C.height;
        D.tiles_x = (C.width + tune->tile_w - 1) / tune->tile_w;
        D.tiles_y = (C.height + tune->tile_h - 1) / tune->tile_h;
        D.tile_base = tiles;
        D.pix_base = pix;
        tiles += (int64_t)D.tiles_x * D.tiles_y;
        pix += (int64_t)C.width * C.height;
    }

    unsigned char* base = nullptr;
    rs_status st = scratch_base(&base);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // the acceleration structure, pointing into the array
    rs_accel A;
    A.n = g->n;
    A.cap = kN;
    A.leaf_size = tune->leaf_size;
    A.morton_bits = tune->morton_bits;
    A.Q_box = p->Q;
    A.rec = reinterpret_cast<float4*>(base + oRec);
    A.pbox = reinterpret_cast<float*>(base + oPbox);
    A.sph = reinterpret_cast<float4*>(base + oSph);
    A.keys[0] = reinterpret_cast<uint64_t*>(base + oKeys0);
    A.keys[1] = reinterpret_cast<uint64_t*>(base + oKeys1);
    A.vals[0] = reinterpret_cast<uint32_t*>(base + oVals0);
    A.vals[1] = reinterpret_cast<uint32_t*>(base + oVals1);
    A.hist = reinterpret_cast<uint32_t*>(base + oHist);
    A.bounds = reinterpret_cast<unsigned*>(base + oBounds);
    A.left = reinterpret_cast<int*>(base + oLeft);
    A.right = reinterpret_cast<int*>(base + oRight);
    A.first = reinterpret_cast<int*>(base + oFirst);
    A.last = reinterpret_cast<int*>(base + oLast);
    A.parent = reinterpret_cast<int*>(base + oParent);
    A.nbox = reinterpret_cast<float*>(base + oNbox);
    A.counter = reinterpret_cast<int*>(base + oCounter);
    A.nodes = reinterpret_cast<float4*>(base + oNodes);
    A.top = reinterpret_cast<float4*>(base + oTop);
    A.err = reinterpret_cast<int*>(base + oErr);
    if (cudaMemsetAsync(A.err, 0, sizeof(int), s) != cudaSuccess) return cuda_check("fixed scratch: reset");
    if ((st = build_accel_device(A, *g, *tune, s))) return st;

    DevCam* cams_dev = reinterpret_cast<DevCam*>(base + oCams);
    k_upload_cams<<<1, 32, 0, s>>>(table, n_cams, cams_dev);
    if ((st = cuda_check("fixed scratch: camera upload"))) return st;
    unsigned long long* queue = reinterpret_cast<unsigned long long*>(base + oQueue);
    if (cudaMemsetAsync(queue, 0, 16, s) != cudaSuccess) return cuda_check("fixed scratch: queue reset");

    FwdArgs F{};
    F.rec = A.rec;
    F.sph = A.sph;
    F.nodes = A.nodes;
    F.top = A.top;
    F.n_top = A.n_top;
    F.cams = cams_dev;
    F.n_cams = n_cams;
    F.cam_single = -1;
    F.total_tiles = tiles;
    F.tile_w = tune->tile_w;
    F.P.Q = p->Q;
    F.P.eps1 = p->eps1;
    F.P.t_near = p->t_near;
    F.P.bg[0] = p->background[0];
    F.P.bg[1] = p->background[1];
    F.P.bg[2] = p->background[2];
    F.P.k_max = p->k_max;
    F.P.max_rounds = (int32_t)(g->n / tune->kbuf + 3);
    F.P.max_visits = (int32_t)(2 * g->n + 16);
    F.P.n_gauss = (int32_t)g->n;
    F.P.n_nodes = (int32_t)std::max<int64_t>(1, g->n - 1);
    F.P.list_cap = 0;  // forward only: no hit list
    F.P.ids = nullptr;
    F.P.sort_key = p->sort_key;
    F.P.grad_mode = 0;  // forward only: the gradient mode does not change the image
    F.P.eps2 = 1.f;
    F.P.sS = nullptr;
    F.rgb = out->rgb;
    F.alpha = out->alpha;
    F.depth = out->depth;
    F.sT = reinterpret_cast<float*>(base + oST);
    F.skey = reinterpret_cast<int64_t*>(base + oSKey);
    F.sn = reinterpret_cast<int*>(base + oSN);
    F.queue = queue;
    F.err = A.err;
    F.stats = nullptr;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int block = 32 * tune->block_warps;
    const int grid = (int)std::min<int64_t>(persistent_grid_fwd(tune->kbuf, block, false, tune->traversal, F.n_top, sms),
                                            (tiles + tune->block_warps - 1) / tune->block_warps);
    const cudaError_t e = launch_forward(F, tune->kbuf, true, false, tune->traversal, std::max(grid, 1), block, s);
    if (e != cudaSuccess) return set_error(RS_ERR_CUDA, "fixed scratch render launch: %s", cudaGetErrorString(e));
    return RS_OK;
}
