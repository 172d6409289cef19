// rs_host.h -- host-side internals of the C ABI: handles, error reporting, launch helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/raysplats.h"

struct rs_accel {
    int64_t n = 0;    // Gaussians in the current build
    int64_t cap = 0;  // capacity of the device buffers (Gaussians)
    int leaf_size = 4;
    int morton_bits = 21;
    float Q_box = 0.f;
    int device = 0;
    // records and boxes in Morton order
    float4* rec = nullptr;   // 4 per Gaussian
    float* pbox = nullptr;   // 6 per Gaussian
    float4* sph = nullptr;   // 1 per Gaussian: bounding sphere (mean, padded radius^2)
    // sort
    uint64_t* keys[2] = {nullptr, nullptr};
    uint32_t* vals[2] = {nullptr, nullptr};
    uint32_t* hist = nullptr;
    unsigned* bounds = nullptr;  // 6 ordered uints
    // tree (internal nodes [0, n-1))
    int* left = nullptr;
    int* right = nullptr;
    int* first = nullptr;
    int* last = nullptr;
    int* parent = nullptr;   // 2n - 1
    float* nbox = nullptr;   // 6 per internal node
    int* counter = nullptr;
    float4* nodes = nullptr; // 4 per internal node (>= 1 node)
    float4* top = nullptr;   // 4 per staged node (kMaxSmemNodes), remapped copies of the top nodes
    float4* wide = nullptr;  // 8 per internal node: 4-wide nodes (built when traversal == 3)
    int has_wide = 0;
    int64_t wide_cap = 0;
    int n_top = 0;           // staged nodes (0: no staging; the root is then node 0)
    int* err = nullptr;      // device error word
};

namespace rs {

using Accel = rs_accel;

// thread-local last-error message and status helpers (api.cu)
rs_status set_error(rs_status st, const char* fmt, ...);
rs_status cuda_check(const char* what);

rs_status build_accel_device(Accel& A, const rs_gaussians& g, const rs_tune_params& tp, cudaStream_t st);

// Free *p (if any) and allocate `bytes` of device memory into it (at least 1 byte).  Honours
// the allocation-failure injection of rs_test_fail_alloc; on failure *p is NULL and RS_ERR_OOM
// is returned with a message.
rs_status device_realloc(void** p, size_t bytes);

}  // namespace rs
