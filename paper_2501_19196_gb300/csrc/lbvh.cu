// lbvh.cu -- device LBVH builder over the scene's Gaussians, rebuilt every training step.
//
// Steps (all stream ordered, no host synchronisation):
//   bounds   min/max of the means (exact, order independent)
//   morton   FP32 quantisation with a fixed operation sequence + bit interleave (x high)
//   sort     stable LSD radix sort of (code, id), 8-bit digits, per-pass histogram / scan /
//            scatter; stability inside a tile from warp-ordered match ranks
//   records  per sorted Gaussian: M = S^-1 R^T with R from the quaternion (App. A.6,
//            s = 2/|q|^2), mean, opacity, colour, conservative ellipsoid box
//   karras   binary radix tree over the keys made unique as (code, position) (Karras 2012)
//   refit    bottom-up box union with per-node arrival counters; the second thread to reach
//            a node writes its traversal node (both child boxes + child references), with
//            subtrees of <= leaf_size Gaussians collapsed into leaves.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rs_internal.cuh"
#include "rs_host.h"

namespace rs {

// ---------------------------------------------------------------------------------------------
// bounds
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned f2ord(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void k_bounds_init(unsigned* b) {
    if (threadIdx.x < 3) b[threadIdx.x] = 0xffffffffu;      // min
    else if (threadIdx.x < 6) b[threadIdx.x] = 0u;          // max
}

__global__ void k_bounds(const float* __restrict__ means, int64_t n, unsigned* __restrict__ b) {
    unsigned lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const unsigned u = f2ord(means[3 * i + k]);
            lo[k] = min(lo[k], u);
            hi[k] = max(hi[k], u);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], s));
            hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], s));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicMin(&b[k], lo[k]);
            atomicMax(&b[3 + k], hi[k]);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// morton
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread3(uint64_t x) {  // 21 bits -> every third bit
    x &= 0x1fffffull;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// bits = 10 / 21: plain 30 / 63-bit codes.  bits = 20: extended 63-bit code
// [x y z interleave of cell bits 19..16][3-bit size class][interleave of bits 15..0] with
// class = clamp(E(max scale) - E(max scene extent) + 11, 0, 7), E = biased FP32 exponent, so
// that large Gaussians gather in their own subtrees instead of inflating their neighbours'.
__global__ void k_morton(const float* __restrict__ means, const float* __restrict__ scales, int64_t n,
                         const unsigned* __restrict__ b, int bits, uint64_t* __restrict__ keys,
                         uint32_t* __restrict__ vals) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float scale = (float)(1u << bits);
    const unsigned cmax = (1u << bits) - 1u;
    uint64_t cell[3];
    float ext_max = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = ord2f(b[k]), hi = ord2f(b[3 + k]);
        float ext = __fsub_rn(hi, lo);
        if (!(ext > 0.f)) ext = 1.f;
        ext_max = fmaxf(ext_max, ext);
        const float u = __fdiv_rn(__fsub_rn(means[3 * i + k], lo), ext);
        const float f = floorf(__fmul_rn(u, scale));
        cell[k] = f <= 0.f ? 0u : (f >= (float)cmax ? cmax : (unsigned)f);
    }
    uint64_t code;
    if (bits == 20) {
        const uint64_t hi3 = (spread3(cell[0] >> 16) << 2) | (spread3(cell[1] >> 16) << 1) | spread3(cell[2] >> 16);
        const uint64_t lo3 = (spread3(cell[0] & 0xffffu) << 2) | (spread3(cell[1] & 0xffffu) << 1) |
                             spread3(cell[2] & 0xffffu);
        const float smax = fmaxf(fmaxf(scales[3 * i], scales[3 * i + 1]), scales[3 * i + 2]);
        int c = (int)((__float_as_uint(smax) >> 23) & 0xffu) - (int)((__float_as_uint(ext_max) >> 23) & 0xffu) + 11;
        c = c < 0 ? 0 : (c > 7 ? 7 : c);
        code = (hi3 << 51) | ((uint64_t)c << 48) | lo3;
    } else {
        code = (spread3(cell[0]) << 2) | (spread3(cell[1]) << 1) | spread3(cell[2]);
    }
    keys[i] = code;
    vals[i] = (uint32_t)i;
}

// ---------------------------------------------------------------------------------------------
// radix sort: 8-bit digits, tiles of kSortThreads * kSortItems keys
// ---------------------------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048
constexpr int kSortWarps = kSortThreads / 32;

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                            int shift, uint32_t* __restrict__ hist,
                                                            int nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const int64_t i = base + it * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of m entries, single CTA of 1024 threads
__global__ void __launch_bounds__(1024) k_scan(uint32_t* __restrict__ a, int64_t m) {
    __shared__ uint32_t part[1024];
    const int64_t chunk = (m + 1023) / 1024;
    const int64_t b0 = threadIdx.x * chunk, b1 = min(m, b0 + chunk);
    uint32_t s = 0;
    for (int64_t i = b0; i < b1; ++i) s += a[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (int64_t i = b0; i < b1; ++i) {
        const uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint64_t* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin,
                                                               uint64_t* __restrict__ kout,
                                                               uint32_t* __restrict__ vout, int64_t n,
                                                               int shift,
                                                               const uint32_t* __restrict__ offs,
                                                               int nblocks) {
    // per-warp digit counters (+1 bucket for out-of-range keys)
    __shared__ uint32_t wc[kSortWarps][257];
    __shared__ uint32_t goff[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = lane; d < 257; d += 32) wc[warp][d] = 0;
    goff[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    __syncwarp();
    // warp w owns keys [base + w*256, base + w*256 + 256) of the tile, lane-strided
    const int64_t base = (int64_t)blockIdx.x * kSortTile + warp * (32 * kSortItems);
    uint64_t k[kSortItems];
    uint32_t v[kSortItems], rank[kSortItems];
    int dig[kSortItems];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const int64_t i = base + it * 32 + lane;
        const bool ok = i < n;
        k[it] = ok ? kin[i] : 0ull;
        v[it] = ok ? vin[i] : 0u;
        dig[it] = ok ? (int)((unsigned)(k[it] >> shift) & 0xffu) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, dig[it]);
        const uint32_t before = wc[warp][dig[it]];
        rank[it] = before + __popc(peers & lt);
        __syncwarp();
        if ((peers & lt) == 0) wc[warp][dig[it]] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps, per digit
    {
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = wc[w][d];
            wc[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        if (dig[it] < 256) {
            const uint32_t pos = goff[dig[it]] + wc[warp][dig[it]] + rank[it];
            kout[pos] = k[it];
            vout[pos] = v[it];
        }
    }
}

// ---------------------------------------------------------------------------------------------
// records + primitive boxes (sorted order)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void quat_rot(float fa, float fb, float fc, float fd, double R[9]) {
    // App. A.6: s = 2/|q|^2, R = I + s K(q), in FP64
    const double qa = fa, qb = fb, qc = fc, qd = fd;
    const double s = 2.0 / (qa * qa + qb * qb + qc * qc + qd * qd);
    const double bs = qb * s, cs = qc * s, ds = qd * s;
    const double ab = qa * bs, ac = qa * cs, ad = qa * ds;
    const double bb = qb * bs, bc = qb * cs, bd = qb * ds;
    const double cc = qc * cs, cd = qc * ds, dd = qd * ds;
    R[0] = 1.0 - cc - dd; R[1] = bc - ad;       R[2] = bd + ac;
    R[3] = bc + ad;       R[4] = 1.0 - bb - dd; R[5] = cd - ab;
    R[6] = bd - ac;       R[7] = cd + ab;       R[8] = 1.0 - bb - cc;
}

__global__ void k_records(const float* __restrict__ means, const float* __restrict__ quats,
                          const float* __restrict__ scales, const float* __restrict__ opac,
                          const float* __restrict__ rgb, const uint32_t* __restrict__ perm, int64_t n,
                          float Q, float4* __restrict__ rec, float* __restrict__ pbox, float4* __restrict__ sph,
                          int* err) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t i = perm[j];
    const float4 q = *reinterpret_cast<const float4*>(quats + 4 * i);
    const float s[3] = {scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]};
    const float m[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    // The whitening M = S^-1 R^T (Sec. 3, App. A.6) is evaluated in FP64 and each entry rounded
    // once to FP32, so a record carries only its own rounding.  Measured against an FP64
    // evaluation of the same Gaussian, the largest FP32 error of the hit tests' D2, t1 and t_m
    // drops by about half (the FP64 pass costs under 0.1 ms per rebuild of 1M Gaussians).
    double Rd[9];
    quat_rot(q.x, q.y, q.z, q.w, Rd);
    float R[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = __double2float_rn(Rd[k]);
    bool bad = !(s[0] > 0.f && s[1] > 0.f && s[2] > 0.f) || !(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w > 0.f);
    float M[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double inv = 1.0 / (double)s[k];
#pragma unroll
        for (int l = 0; l < 3; ++l) M[3 * k + l] = __double2float_rn(Rd[3 * l + k] * inv);
    }
    rec[4 * j + 0] = make_float4(M[0], M[1], M[2], m[0]);
    rec[4 * j + 1] = make_float4(M[3], M[4], M[5], m[1]);
    rec[4 * j + 2] = make_float4(M[6], M[7], M[8], m[2]);
    rec[4 * j + 3] = make_float4(opac[i], rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2]);
    // conservative box of {x : |M (x - m)|^2 <= Q} = m + R S (ball of radius sqrt(Q)):
    // half extent along world axis a = sqrt(Q) * |row a of R S|, padded.
    const float sq = sqrtf(Q);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float r0 = R[3 * a] * s[0], r1 = R[3 * a + 1] * s[1], r2 = R[3 * a + 2] * s[2];
        float ext = sq * sqrtf(r0 * r0 + r1 * r1 + r2 * r2);
        ext = ext * (1.f + 1e-5f) + 1e-5f * fabsf(m[a]) + 1e-30f;
        bad |= !(ext < 3.0e38f) || !(fabsf(m[a]) < 3.0e38f);
        pbox[6 * j + a] = m[a] - ext;
        pbox[6 * j + 3 + a] = m[a] + ext;
    }
    // bounding sphere of the ellipsoid: radius sqrt(Q) * max scale, padded like the box
    const float smax = fmaxf(fmaxf(s[0], s[1]), s[2]);
    const float r = (sq * smax) * (1.f + 1e-5f) + 1e-30f;
    sph[j] = make_float4(m[0], m[1], m[2], r * r);
    if (bad) atomicOr(err, kErrBadScene);
}

// ---------------------------------------------------------------------------------------------
// Karras 2012 hierarchy over keys (code, position)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int delta(const uint64_t* __restrict__ c, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    const uint64_t a = c[i], b = c[j];
    if (a != b) return __clzll((long long)(a ^ b));
    return 64 + __clz((int)((uint32_t)i ^ (uint32_t)j));
}

__global__ void k_karras(const uint64_t* __restrict__ codes, int64_t n, int* __restrict__ left,
                         int* __restrict__ right, int* __restrict__ first, int* __restrict__ last,
                         int* __restrict__ parent) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int dsgn = (delta(codes, n, i, i + 1) - delta(codes, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(codes, n, i, i - dsgn);
    int64_t lmax = 2;
    while (delta(codes, n, i, i + lmax * dsgn) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(codes, n, i, i + (l + t) * dsgn) > dmin) l += t;
    const int64_t j = i + l * dsgn;
    const int dnode = delta(codes, n, i, j);
    int64_t s = 0;
    int64_t t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(codes, n, i, i + (s + t) * dsgn) > dnode) s += t;
    } while (t > 1);
    const int64_t gamma = i + s * dsgn + min(dsgn, 0);
    const int64_t lo = min(i, j), hi = max(i, j);
    const int lc = (lo == gamma) ? ~(int)gamma : (int)gamma;
    const int rc = (hi == gamma + 1) ? ~(int)(gamma + 1) : (int)(gamma + 1);
    left[i] = lc;
    right[i] = rc;
    first[i] = (int)lo;
    last[i] = (int)hi;
    // parents: internal nodes at [0, n-1), leaves at [n-1, 2n-1)
    parent[lc >= 0 ? lc : (n - 1) + ~lc] = (int)i;
    parent[rc >= 0 ? rc : (n - 1) + ~rc] = (int)i;
    if (i == 0) parent[0] = -1;
}

// ---------------------------------------------------------------------------------------------
// refit + traversal node emission
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void child_info(int c, const int* first, const int* last,
                                           const float* pbox, const float* nbox, int leaf_size,
                                           float b[6], int& ref, int& cnt) {
    if (c < 0) {
        const int leaf = ~c;
#pragma unroll
        for (int k = 0; k < 6; ++k) b[k] = __ldcg(pbox + 6 * leaf + k);
        ref = ~leaf;
        cnt = 1;
    } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) b[k] = __ldcg(nbox + 6 * c + k);
        const int f = __ldcg(first + c), l = __ldcg(last + c);
        const int sz = l - f + 1;
        if (sz <= leaf_size) {
            ref = ~f;
            cnt = sz;
        } else {
            ref = c;
            cnt = 0;
        }
    }
}

__global__ void k_refit(int64_t n, const int* __restrict__ left, const int* __restrict__ right,
                        const int* __restrict__ first, const int* __restrict__ last,
                        const int* __restrict__ parent, const float* __restrict__ pbox,
                        float* __restrict__ nbox, int* __restrict__ counter, float4* __restrict__ nodes,
                        int leaf_size, int* err) {
    const int64_t leaf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (leaf >= n) return;
    int p = parent[(n - 1) + leaf];
    for (int level = 0; p >= 0; ++level) {
        if (level > 2 * kStackSize) {  // deeper than any radix tree over 96-bit keys: corrupt
            atomicOr(err, kErrLoopGuard);
            return;
        }
        __threadfence();
        if (atomicAdd(&counter[p], 1) == 0) return;  // first arrival: the sibling finishes p
        __threadfence();
        float b0[6], b1[6];
        int r0, r1, c0, c1;
        child_info(left[p], first, last, pbox, nbox, leaf_size, b0, r0, c0);
        child_info(right[p], first, last, pbox, nbox, leaf_size, b1, r1, c1);
        float u[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            u[k] = fminf(b0[k], b1[k]);
            u[3 + k] = fmaxf(b0[3 + k], b1[3 + k]);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) __stcg(nbox + 6 * p + k, u[k]);
        const int sz = last[p] - first[p] + 1;
        if (sz > leaf_size || p == 0) {
            nodes[4 * p + 0] = make_float4(b0[0], b0[3], b0[1], b0[4]);
            nodes[4 * p + 1] = make_float4(b1[0], b1[3], b1[1], b1[4]);
            nodes[4 * p + 2] = make_float4(b0[2], b0[5], b1[2], b1[5]);
            nodes[4 * p + 3] = make_float4(__int_as_float(r0), __int_as_float(r1), __int_as_float(c0),
                                           __int_as_float(c1));
        }
        p = parent[p];
    }
}

// Breadth-first staging of the top `m` nodes for the render kernels' shared memory.  Slots are
// assigned level by level in node order (deterministic: a block scan over the children
// counts); each staged copy refers to its staged children as kTopRef + slot.  One CTA.
__global__ void __launch_bounds__(kMaxSmemNodes) k_stage_top(const float4* __restrict__ nodes, int m,
                                                             float4* __restrict__ top) {
    __shared__ int cur[kMaxSmemNodes], nxt[kMaxSmemNodes], pos[kMaxSmemNodes];
    __shared__ int n_cur, n_next, base_next;
    const int t = threadIdx.x;
    if (t == 0) {
        cur[0] = 0;
        n_cur = 1;
    }
    __syncthreads();
    int base = 0;  // slot of cur[0]
    while (true) {
        const int nc = n_cur;
        if (nc == 0) break;
        float4 n0, n1, n2, n3;
        int cnt = 0;
        if (t < nc) {
            const int node = cur[t];
            n0 = nodes[4 * node];
            n1 = nodes[4 * node + 1];
            n2 = nodes[4 * node + 2];
            n3 = nodes[4 * node + 3];
            cnt = (__float_as_int(n3.x) >= 0) + (__float_as_int(n3.y) >= 0);
        }
        pos[t] = cnt;
        __syncthreads();
        for (int off = 1; off < kMaxSmemNodes; off <<= 1) {  // inclusive scan of the counts
            const int v = t >= off ? pos[t - off] : 0;
            __syncthreads();
            pos[t] += v;
            __syncthreads();
        }
        if (t == 0) {
            base_next = base + nc;
            n_next = min(pos[kMaxSmemNodes - 1], max(0, m - (base + nc)));
        }
        __syncthreads();
        if (t < nc) {
            int r[2] = {__float_as_int(n3.x), __float_as_int(n3.y)};
            int p = pos[t] - cnt;  // exclusive position of this node's first internal child
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (r[c] >= 0) {
                    if (p < n_next) {
                        nxt[p] = r[c];
                        r[c] = kTopRef + base_next + p;
                    }
                    ++p;
                }
            }
            const int slot = base + t;
            top[4 * slot] = n0;
            top[4 * slot + 1] = n1;
            top[4 * slot + 2] = n2;
            top[4 * slot + 3] = make_float4(__int_as_float(r[0]), __int_as_float(r[1]), n3.z, n3.w);
        }
        __syncthreads();
        if (t < n_next) cur[t] = nxt[t];
        if (t == 0) n_cur = n_next;
        base = base_next;
        __syncthreads();
    }
}

// 4-wide nodes: for every emitted binary node p, its children are p's grandchildren (a leaf
// child stays a child).  Descending into an internal grandchild g then uses g's own wide node,
// so a traversal of the wide nodes visits every other level of the binary tree.  Layout per
// node (8 float4): lo.x, hi.x, lo.y, hi.y, lo.z, hi.z of the four children, refs, counts;
// unused slots have ref kEmptyRef.  Only emitted nodes (size > leaf_size, or the root) are
// read: their child references are valid by construction.
__global__ void k_wide(const float4* __restrict__ nodes, const int* __restrict__ first, const int* __restrict__ last,
                       int64_t n_int, int leaf_size, float4* __restrict__ wide) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n_int) return;
    if (first && p != 0 && (last[p] - first[p] + 1) <= leaf_size) return;  // not emitted (n == 1: first is NULL)
    float lo[3][4], hi[3][4];
    int ref[4], cnt[4];
    int m = 0;
    auto add = [&](const float4 a, const float4 b, const float4 z, int side, int r, int c) {
        // box of child `side` of a binary node (a = side 0 xy, b = side 1 xy, z = both z)
        const float4 xy = side ? b : a;
        lo[0][m] = xy.x; hi[0][m] = xy.y; lo[1][m] = xy.z; hi[1][m] = xy.w;
        lo[2][m] = side ? z.z : z.x; hi[2][m] = side ? z.w : z.y;
        ref[m] = r;
        cnt[m] = c;
        ++m;
    };
    const float4 n0 = nodes[4 * p], n1 = nodes[4 * p + 1], n2 = nodes[4 * p + 2], n3 = nodes[4 * p + 3];
    const int r[2] = {__float_as_int(n3.x), __float_as_int(n3.y)};
    const int c[2] = {__float_as_int(n3.z), __float_as_int(n3.w)};
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        if (r[side] >= 0) {
            const int g = r[side];
            const float4 g0 = nodes[4 * g], g1 = nodes[4 * g + 1], g2 = nodes[4 * g + 2], g3 = nodes[4 * g + 3];
            add(g0, g1, g2, 0, __float_as_int(g3.x), __float_as_int(g3.z));
            add(g0, g1, g2, 1, __float_as_int(g3.y), __float_as_int(g3.w));
        } else {
            add(n0, n1, n2, side, r[side], c[side]);
        }
    }
    for (; m < 4; ++m) {
        lo[0][m] = lo[1][m] = lo[2][m] = 3.0e38f;
        hi[0][m] = hi[1][m] = hi[2][m] = -3.0e38f;
        ref[m] = kEmptyRef;
        cnt[m] = 0;
    }
    float4* w = wide + 8 * p;
    w[0] = make_float4(lo[0][0], lo[0][1], lo[0][2], lo[0][3]);
    w[1] = make_float4(hi[0][0], hi[0][1], hi[0][2], hi[0][3]);
    w[2] = make_float4(lo[1][0], lo[1][1], lo[1][2], lo[1][3]);
    w[3] = make_float4(hi[1][0], hi[1][1], hi[1][2], hi[1][3]);
    w[4] = make_float4(lo[2][0], lo[2][1], lo[2][2], lo[2][3]);
    w[5] = make_float4(hi[2][0], hi[2][1], hi[2][2], hi[2][3]);
    w[6] = make_float4(__int_as_float(ref[0]), __int_as_float(ref[1]), __int_as_float(ref[2]), __int_as_float(ref[3]));
    w[7] = make_float4(__int_as_float(cnt[0]), __int_as_float(cnt[1]), __int_as_float(cnt[2]), __int_as_float(cnt[3]));
}

// single Gaussian: a root whose first child is the leaf and whose second child is empty
__global__ void k_single_root(const float* __restrict__ pbox, float4* __restrict__ nodes) {
    const float* b = pbox;
    nodes[0] = make_float4(b[0], b[3], b[1], b[4]);
    nodes[1] = make_float4(b[0], b[3], b[1], b[4]);
    nodes[2] = make_float4(b[2], b[5], b[2], b[5]);
    nodes[3] = make_float4(__int_as_float(~0), __int_as_float(~0), __int_as_float(1), __int_as_float(0));
}

// ---------------------------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------------------------
static inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

rs_status build_accel_device(Accel& A, const rs_gaussians& g, const rs_tune_params& tp, cudaStream_t st) {
    const int64_t n = A.n;
    const int bits = tp.morton_bits;
    k_bounds_init<<<1, 32, 0, st>>>(A.bounds);
    {
        const unsigned grid = (unsigned)std::min<int64_t>(grid_for(n, 256), 4 * 152);
        k_bounds<<<grid, 256, 0, st>>>(g.means, n, A.bounds);
    }
    k_morton<<<grid_for(n, 256), 256, 0, st>>>(g.means, g.scales, n, A.bounds, bits, A.keys[0], A.vals[0]);
    const int nblocks = (int)((n + kSortTile - 1) / kSortTile);
    const int passes = bits == 10 ? 4 : 8;
    for (int ps = 0; ps < passes; ++ps) {
        const int src = ps & 1, dst = src ^ 1;
        k_sort_hist<<<nblocks, kSortThreads, 0, st>>>(A.keys[src], n, 8 * ps, A.hist, nblocks);
        k_scan<<<1, 1024, 0, st>>>(A.hist, (int64_t)256 * nblocks);
        k_sort_scatter<<<nblocks, kSortThreads, 0, st>>>(A.keys[src], A.vals[src], A.keys[dst], A.vals[dst], n,
                                                         8 * ps, A.hist, nblocks);
    }
    // passes is even: the sorted (code, id) pairs are back in buffer 0
    k_records<<<grid_for(n, 256), 256, 0, st>>>(g.means, g.quats, g.scales, g.opacities, g.rgb, A.vals[0], n,
                                               A.Q_box, A.rec, A.pbox, A.sph, A.err);
    if (n == 1) {
        k_single_root<<<1, 1, 0, st>>>(A.pbox, A.nodes);
    } else {
        k_karras<<<grid_for(n - 1, 256), 256, 0, st>>>(A.keys[0], n, A.left, A.right, A.first, A.last, A.parent);
        cudaMemsetAsync(A.counter, 0, sizeof(int) * (size_t)(n - 1), st);
        k_refit<<<grid_for(n, 256), 256, 0, st>>>(n, A.left, A.right, A.first, A.last, A.parent, A.pbox, A.nbox,
                                                 A.counter, A.nodes, tp.leaf_size, A.err);
    }
    // at most one node per internal node can be staged (n - 1 internal nodes, one for n == 1)
    A.n_top = (int)std::min<int64_t>(std::min(tp.smem_nodes, kMaxSmemNodes), std::max<int64_t>(1, n - 1));
    if (tp.smem_nodes <= 0) A.n_top = 0;
    if (A.n_top > 0) k_stage_top<<<1, kMaxSmemNodes, 0, st>>>(A.nodes, A.n_top, A.top);
    if (A.has_wide) {
        const int64_t n_int = std::max<int64_t>(1, n - 1);
        k_wide<<<grid_for(n_int, 256), 256, 0, st>>>(A.nodes, n == 1 ? nullptr : A.first, n == 1 ? nullptr : A.last,
                                                    n_int, tp.leaf_size, A.wide);
    }
    return cuda_check("rs_build_accel launch");
}

}  // namespace rs
