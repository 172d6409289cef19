// trace.cuh -- the device side of the rendering path shared by the forward and adjoint kernels
// (render_fwd.cu, render_bwd.cu): ray/box and ray/ellipsoid tests, k-buffers, the warp
// node queue, the per-ray and warp-packet traversals, and the per-hit adjoint.
//
// Forward (a7-a9): each lane traces one camera ray.  A pass traverses the LBVH (by default
// best first over warp packets) with a buffer of pending hits ordered by their (t, residual,
// id) key beyond the last composited key; a pending hit is composited front to back (Eq. 3)
// with alpha = opacity * exp(-D2/2) (Prop. 2) as soon as no unvisited box can hold an earlier
// hit, and the ray stops after the hit that brings T below eps1 or at k_max hits (Sec. 3).  A
// buffer that overflows caps the pass and a further pass resumes after the last composited
// key.  Per ray it stores T_final, the last composited key and the hit count (16 B), and the
// ids of its first hit_list composited hits.
//
// Adjoint (a10): from the hit list, or by the same traversal mirrored (a descending buffer of
// pending hits below an upper key), the composited hits are replayed back to front.  The
// transmittance before each hit is recovered as T_i = T_{i+1} / (1 - alpha_i) from the stored
// T_final (the forward's (1 - alpha_i) is recomputed bit for bit, so the rounding cancels),
// and the colour behind a hit follows U_{i-1} = alpha_i c_i + (1 - alpha_i) U_i, giving
// dC/dalpha_i = T_i (c_i - U_i) without the division of App. A.4/A.5.  The chain through D2
// (App. A.6) uses the envelope form dD2/dM = 2 p v^T, dD2/dm = -2 M^T p; per-hit contributions
// go to a 16-float-per-Gaussian accumulator with float4 atomics, and a finalize kernel maps
// dL/dM to the quaternion and scales through M = S^-1 R(q)^T.
//
// Launch modes: plain (one launch per camera, one warp per 32-ray tile) and persistent (one
// launch over every camera's tiles, warps pull tiles from a device counter).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "rs_internal.cuh"

#include "rs_render.h"

namespace rs {

__device__ __forceinline__ float safe_rcp(float x) {
    const float ax = fabsf(x);
    return __frcp_rn(ax > 1e-30f ? x : copysignf(1e-30f, x));
}

// Cheap conservative rejection before the full ray/ellipsoid solve: the ray must pass within
// the Gaussian's bounding sphere (radius sqrt(Q) * max scale, padded).  The squared distance
// |w|^2 - <w, d>^2 is widened by 1e-6 |w|^2 to absorb its rounding, so a ray the solve would
// accept is never rejected here.
__device__ __forceinline__ bool sphere_may_hit(const float3 o, const float3 d, const float4 sp) {
    const float wx = sp.x - o.x, wy = sp.y - o.y, wz = sp.z - o.z;
    const float tc = fmaf(wz, d.z, fmaf(wy, d.y, wx * d.x));
    const float w2 = fmaf(wz, wz, fmaf(wy, wy, wx * wx));
    return fmaf(-tc, tc, w2) <= fmaf(1e-6f, w2, sp.w);
}

// Where nodes come from: the staged top nodes (shared memory, references kTopRef + slot) or
// the node array in global memory.  `root` is kTopRef when the top is staged, else 0.
struct NodeSrc {
    const float4* __restrict__ g;
    const float4* s;
    int root;
    const float4* __restrict__ w;  // 4-wide nodes (8 float4 each), indexed like the binary nodes
    int n_nodes, n_top, n_gauss;   // bounds of node references, staged slots and leaf ranges
    int* err;
};

// a leaf's Gaussian count after the range check (a corrupt range reads nothing and is reported)
__device__ __forceinline__ int leaf_count(const NodeSrc& ns, int start, int cnt) {
    if (start >= 0 && cnt >= 0 && cnt <= 32 && start <= ns.n_gauss - cnt) return cnt;
    atomicOr(ns.err, kErrIndex);
    return 0;
}

// Bounding-sphere pre-test of one leaf for the whole warp: the leaf's spheres are loaded once
// (lane i holds Gaussian start + i) and broadcast by shuffles.  Bit g of the result is set when
// this lane wants the leaf and its ray may hit Gaussian start + g.  num <= 32 (leaf_size <= 32).
__device__ __forceinline__ uint32_t leaf_sphere_mask(const float4* __restrict__ sph, int start, int num, bool want,
                                                     const float3 o, const float3 d) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float4 mine = make_float4(0.f, 0.f, 0.f, -1.f);
    if (lane < num) mine = __ldg(sph + start + lane);
    uint32_t mask = 0;
    for (int g = 0; g < num; ++g) {
        float4 sp;
        sp.x = __shfl_sync(FULL, mine.x, g);
        sp.y = __shfl_sync(FULL, mine.y, g);
        sp.z = __shfl_sync(FULL, mine.z, g);
        sp.w = __shfl_sync(FULL, mine.w, g);
        if (want && sphere_may_hit(o, d, sp)) mask |= 1u << g;
    }
    return mask;
}

// the hardware's approximate square root (relative error below 2^-22)
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The rays of a warp that share one origin (a camera's tile) as a cone: axis, cos and sin of
// the half-angle, widened so that rounding cannot make it narrower than the rays.
struct RayCone {
    float3 ax;
    float cth, sth;
    bool ok;  // every lane has the same origin
};

__device__ __forceinline__ RayCone warp_ray_cone(const float3 o, const float3 d) {
    const unsigned FULL = 0xffffffffu;
    RayCone c;
    const float ox = __shfl_sync(FULL, o.x, 0), oy = __shfl_sync(FULL, o.y, 0), oz = __shfl_sync(FULL, o.z, 0);
    c.ok = __all_sync(FULL, o.x == ox && o.y == oy && o.z == oz);
    float sx = d.x, sy = d.y, sz = d.z;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        sx += __shfl_xor_sync(FULL, sx, m);
        sy += __shfl_xor_sync(FULL, sy, m);
        sz += __shfl_xor_sync(FULL, sz, m);
    }
    const float il = rsqrtf(fmaxf(sx * sx + sy * sy + sz * sz, 1e-30f));
    c.ax = make_float3(sx * il, sy * il, sz * il);
    // per lane: cos and sin of the angle to the axis (the sine from the cross product, which
    // keeps its accuracy for narrow cones)
    const float cs = d.x * c.ax.x + d.y * c.ax.y + d.z * c.ax.z;
    const float cx = d.y * c.ax.z - d.z * c.ax.y, cy = d.z * c.ax.x - d.x * c.ax.z, cz = d.x * c.ax.y - d.y * c.ax.x;
    const float sn = sqrtf(cx * cx + cy * cy + cz * cz);
    float mc = cs;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) mc = fminf(mc, __shfl_xor_sync(FULL, mc, m));
    c.cth = fmaxf(mc - 1e-5f, -1.f);
    c.sth = fminf(__uint_as_float(__reduce_max_sync(FULL, __float_as_uint(sn))) + 1e-5f, 1.f);
    c.ok = c.ok && c.cth > 0.f;  // narrower than a half space
    return c;
}

// The leaf pre-test of rays that share an origin: lane g tests sphere start + g against the
// warp's ray cone, and the spheres the cone may reach go straight to the full test of every lane
// that wants the leaf (the full test decides, so the result is the same as with a per-lane
// sphere test; that test, four shuffles and a sphere/ray test per candidate, cost more than
// the full tests it saved).  A sphere (c, r) can meet a ray of the cone at t >= 0 only if the
// origin lies inside it, or its centre is ahead (<w, axis> > -r) and its distance to the cone's
// surface, |w x axis| cos - <w, axis> sin, is at most r.
__device__ __forceinline__ uint32_t leaf_sphere_mask_cone(const float4* __restrict__ sph, int start, int num,
                                                          bool want, const float3 o, const float3 d,
                                                          const RayCone& cone) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float4 mine = make_float4(0.f, 0.f, 0.f, -1.f);
    bool reach = false;
    if (lane < num) {
        mine = __ldg(sph + start + lane);
        const float wx = mine.x - o.x, wy = mine.y - o.y, wz = mine.z - o.z;
        const float L2 = wx * wx + wy * wy + wz * wz;
        const float r = sqrt_approx(mine.w) * 1.0001f + 1e-6f * sqrt_approx(L2);
        const float t = wx * cone.ax.x + wy * cone.ax.y + wz * cone.ax.z;
        const float cx = wy * cone.ax.z - wz * cone.ax.y, cy = wz * cone.ax.x - wx * cone.ax.z;
        const float cz = wx * cone.ax.y - wy * cone.ax.x;
        const float dperp = sqrt_approx(cx * cx + cy * cy + cz * cz);
        reach = L2 <= r * r || (t > -r && dperp * cone.cth - t * cone.sth <= r);
    }
    const uint32_t cand = __ballot_sync(FULL, reach);
    return want ? cand : 0u;
}

// The children of one node as seen by the traversal: W = 2 reads a binary node (possibly staged
// in shared memory), W = 4 a wide node (the node's grandchildren; empty slots have ref kEmptyRef).
template <int W>
struct Children {
    float lo[3][W], hi[3][W];
    int ref[W], cnt[W];
};

// STAGED = false: the caller stages no nodes (no shared-memory branch)
template <bool STAGED = true>
__device__ __forceinline__ void fetch_node(const NodeSrc& ns, int node, float4& n0, float4& n1, float4& n2,
                                           float4& n3) {
    const bool ok = (STAGED && node >= kTopRef) ? (node - kTopRef) < ns.n_top : (node >= 0 && node < ns.n_nodes);
    if (!ok) {  // corrupt reference: report, and present a node without children
        atomicOr(ns.err, kErrIndex);
        n0 = n1 = n2 = make_float4(0.f, 0.f, 0.f, 0.f);
        n3 = make_float4(__int_as_float(kEmptyRef), __int_as_float(kEmptyRef), __int_as_float(0), __int_as_float(0));
        return;
    }
    if (STAGED && node >= kTopRef) {
        const float4* p = ns.s + 4 * (node - kTopRef);
        n0 = p[0];
        n1 = p[1];
        n2 = p[2];
        n3 = p[3];
    } else {
        n0 = __ldg(ns.g + 4 * node + 0);
        n1 = __ldg(ns.g + 4 * node + 1);
        n2 = __ldg(ns.g + 4 * node + 2);
        n3 = __ldg(ns.g + 4 * node + 3);
    }
}

template <int W, bool STAGED = true>
__device__ __forceinline__ void fetch_children(const NodeSrc& ns, int node, Children<W>& ch);

template <bool STAGED>
__device__ __forceinline__ void fetch_children2(const NodeSrc& ns, int node, Children<2>& ch) {
    float4 n0, n1, n2, n3;
    fetch_node<STAGED>(ns, node, n0, n1, n2, n3);
    ch.lo[0][0] = n0.x; ch.hi[0][0] = n0.y; ch.lo[1][0] = n0.z; ch.hi[1][0] = n0.w;
    ch.lo[0][1] = n1.x; ch.hi[0][1] = n1.y; ch.lo[1][1] = n1.z; ch.hi[1][1] = n1.w;
    ch.lo[2][0] = n2.x; ch.hi[2][0] = n2.y; ch.lo[2][1] = n2.z; ch.hi[2][1] = n2.w;
    ch.ref[0] = __float_as_int(n3.x); ch.ref[1] = __float_as_int(n3.y);
    ch.cnt[0] = __float_as_int(n3.z); ch.cnt[1] = __float_as_int(n3.w);
}

template <>
__device__ __forceinline__ void fetch_children<2, true>(const NodeSrc& ns, int node, Children<2>& ch) {
    fetch_children2<true>(ns, node, ch);
}

template <>
__device__ __forceinline__ void fetch_children<2, false>(const NodeSrc& ns, int node, Children<2>& ch) {
    fetch_children2<false>(ns, node, ch);
}

template <>
__device__ __forceinline__ void fetch_children<4, true>(const NodeSrc& ns, int node, Children<4>& ch) {
    if (node < 0 || node >= ns.n_nodes) {
        atomicOr(ns.err, kErrIndex);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            ch.ref[c] = kEmptyRef;
            ch.cnt[c] = 0;
            ch.lo[0][c] = ch.lo[1][c] = ch.lo[2][c] = ch.hi[0][c] = ch.hi[1][c] = ch.hi[2][c] = 0.f;
        }
        return;
    }
    const float4* p = ns.w + 8 * node;
    const float4 lx = __ldg(p + 0), hx = __ldg(p + 1), ly = __ldg(p + 2), hy = __ldg(p + 3);
    const float4 lz = __ldg(p + 4), hz = __ldg(p + 5), rf = __ldg(p + 6), ct = __ldg(p + 7);
    const float a[8][4] = {{lx.x, lx.y, lx.z, lx.w}, {hx.x, hx.y, hx.z, hx.w}, {ly.x, ly.y, ly.z, ly.w},
                           {hy.x, hy.y, hy.z, hy.w}, {lz.x, lz.y, lz.z, lz.w}, {hz.x, hz.y, hz.z, hz.w},
                           {rf.x, rf.y, rf.z, rf.w}, {ct.x, ct.y, ct.z, ct.w}};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        ch.lo[0][c] = a[0][c]; ch.hi[0][c] = a[1][c];
        ch.lo[1][c] = a[2][c]; ch.hi[1][c] = a[3][c];
        ch.lo[2][c] = a[4][c]; ch.hi[2][c] = a[5][c];
        ch.ref[c] = __float_as_int(a[6][c]);
        ch.cnt[c] = __float_as_int(a[7][c]);
    }
}

// entry / exit of child c's box, widened by 1e-6 relative (as slab2)
template <int W>
__device__ __forceinline__ void slab_child(const Children<W>& ch, int c, const float3 o, const float3 inv, float& en,
                                           float& ex) {
    const float a0 = (ch.lo[0][c] - o.x) * inv.x, b0 = (ch.hi[0][c] - o.x) * inv.x;
    const float a1 = (ch.lo[1][c] - o.y) * inv.y, b1 = (ch.hi[1][c] - o.y) * inv.y;
    const float a2 = (ch.lo[2][c] - o.z) * inv.z, b2 = (ch.hi[2][c] - o.z) * inv.z;
    const float e = fmaxf(fmaxf(fminf(a0, b0), fminf(a1, b1)), fminf(a2, b2));
    const float x = fminf(fminf(fmaxf(a0, b0), fmaxf(a1, b1)), fmaxf(a2, b2));
    en = fmaf(-1e-6f, fabsf(e), e);
    ex = fmaf(1e-6f, fabsf(x), x);
}

// Entry and exit parameters of both children's boxes, widened by 1e-6 relative so that rounding
// can never drop a box that holds a hit (the boxes themselves are padded too).
__device__ __forceinline__ void slab2(const float4 n0, const float4 n1, const float4 n2, const float3 o,
                                      const float3 inv, float& en0, float& ex0, float& en1, float& ex1) {
    {
        const float a0 = (n0.x - o.x) * inv.x, b0 = (n0.y - o.x) * inv.x;
        const float a1 = (n0.z - o.y) * inv.y, b1 = (n0.w - o.y) * inv.y;
        const float a2 = (n2.x - o.z) * inv.z, b2 = (n2.y - o.z) * inv.z;
        const float en = fmaxf(fmaxf(fminf(a0, b0), fminf(a1, b1)), fminf(a2, b2));
        const float ex = fminf(fminf(fmaxf(a0, b0), fmaxf(a1, b1)), fmaxf(a2, b2));
        en0 = fmaf(-1e-6f, fabsf(en), en);
        ex0 = fmaf(1e-6f, fabsf(ex), ex);
    }
    {
        const float a0 = (n1.x - o.x) * inv.x, b0 = (n1.y - o.x) * inv.x;
        const float a1 = (n1.z - o.y) * inv.y, b1 = (n1.w - o.y) * inv.y;
        const float a2 = (n2.z - o.z) * inv.z, b2 = (n2.w - o.z) * inv.z;
        const float en = fmaxf(fmaxf(fminf(a0, b0), fminf(a1, b1)), fminf(a2, b2));
        const float ex = fminf(fminf(fmaxf(a0, b0), fmaxf(a1, b1)), fmaxf(a2, b2));
        en1 = fmaf(-1e-6f, fabsf(en), en);
        ex1 = fmaf(1e-6f, fabsf(ex), ex);
    }
}

// ascending buffer: keys[0] nearest; insert `key` (< keys[K-1]) by one bubble pass
template <int K>
__device__ __forceinline__ void kbuf_insert_asc(int64_t (&keys)[K], int64_t key) {
    keys[K - 1] = key;
#pragma unroll
    for (int s = K - 1; s > 0; --s) {
        const int64_t ka = keys[s - 1], kb = keys[s];
        keys[s - 1] = min(ka, kb);
        keys[s] = max(ka, kb);
    }
}

// descending buffer: keys[0] farthest; insert `key` (> keys[K-1])
template <int K>
__device__ __forceinline__ void kbuf_insert_desc(int64_t (&keys)[K], int64_t key) {
    keys[K - 1] = key;
#pragma unroll
    for (int s = K - 1; s > 0; --s) {
        const int64_t ka = keys[s - 1], kb = keys[s];
        keys[s - 1] = max(ka, kb);
        keys[s] = min(ka, kb);
    }
}

// drop keys[0] (the hit just composited / replayed)
template <int K>
__device__ __forceinline__ void kbuf_pop_front(int64_t (&keys)[K], int64_t empty) {
#pragma unroll
    for (int s = 0; s < K - 1; ++s) keys[s] = keys[s + 1];
    keys[K - 1] = empty;
}

// Occupancy-aware variants for warp-converged callers.  A lane's buffer holds nk keys in slots
// [0, nk); the rest are empty.  The warp sizes the compare-exchange network by the largest nk
// among the lanes taking part (a uniform choice), so a sparsely filled buffer costs a short
// network instead of all K stages.  Results equal those of the full-width functions above.
template <int K, int C, bool DESC>
__device__ __forceinline__ void kbuf_insert_at(int64_t (&keys)[K], int64_t key) {
    keys[C] = key;  // free for every inserting lane (nk <= C), or the dropped last slot (C = K-1)
#pragma unroll
    for (int s = C; s > 0; --s) {
        const int64_t ka = keys[s - 1], kb = keys[s];
        keys[s - 1] = DESC ? max(ka, kb) : min(ka, kb);
        keys[s] = DESC ? min(ka, kb) : max(ka, kb);
    }
}

// insert `key` where `ins` (all 32 lanes call); a full buffer drops its last key.  DESC: the
// descending buffer of the adjoint.
template <int K, bool DESC = false>
__device__ __forceinline__ void kbuf_insert_warp(int64_t (&keys)[K], int& nk, bool ins, int64_t key) {
    const int m = (int)__reduce_max_sync(0xffffffffu, ins ? (unsigned)nk : 0u);
    if constexpr (K > 8) {
        if (m < 8) {
            if (ins) kbuf_insert_at<K, 8, DESC>(keys, key);
            if (ins) ++nk;
            return;
        }
    }
    if constexpr (K > 16) {
        if (m < 16) {
            if (ins) kbuf_insert_at<K, 16, DESC>(keys, key);
            if (ins) ++nk;
            return;
        }
    }
    if constexpr (K > 24) {
        if (m < 24) {
            if (ins) kbuf_insert_at<K, 24, DESC>(keys, key);
            if (ins) ++nk;
            return;
        }
    }
    if (ins) {
        kbuf_insert_at<K, K - 1, DESC>(keys, key);
        if (nk < K) ++nk;
    }
}

template <int K, int C>
__device__ __forceinline__ void kbuf_pop_upto(int64_t (&keys)[K], int64_t empty) {
#pragma unroll
    for (int s = 0; s < C; ++s) keys[s] = keys[s + 1];
    keys[C] = empty;
}

// drop keys[0] in the lanes of `group` (the calling lanes, converged)
template <int K>
__device__ __forceinline__ void kbuf_pop_warp(int64_t (&keys)[K], int& nk, int64_t empty, unsigned group) {
    const int m = (int)__reduce_max_sync(group, (unsigned)nk);
    --nk;
    if constexpr (K > 8) {
        if (m <= 8) {
            kbuf_pop_upto<K, 8>(keys, empty);
            return;
        }
    }
    kbuf_pop_front<K>(keys, empty);
}

struct Counters {
    uint32_t nodes = 0, tests = 0, hits = 0, rounds = 0, inserted = 0;
    uint32_t wnodes = 0, wleaf = 0;  // packet modes: node fetches and leaf iterations of whole warps
};

// Running state of one ray's back-to-front replay: the transmittance in front of the next hit
// to replay and the colour / alpha / depth composited behind it (App. A.4-A.5).
struct Adjoint {
    float Tn, U0, U1, U2, UA, UD;
    float O0, O1, O2, OA;  // eps2 estimator: colour / alpha behind the first replayed hit (OA < 0: none)
};



// Upstream gradient of one ray: dL/d(rgb), dL/d(alpha), dL/d(depth); and, for the eps2
// estimator, the colour / alpha behind its last composited hit (o[3] < 0: none).
struct Upstream {
    float c[3], a, d;
    float o[4];
};

// Start the back-to-front replay of one ray.
__device__ __forceinline__ Adjoint adjoint_start(const TraceParams& P, float T_final, const Upstream& g) {
    return Adjoint{T_final, P.bg[0], P.bg[1], P.bg[2], 0.f, 0.f, g.o[0], g.o[1], g.o[2], g.o[3]};
}

// The adjoint of one composited hit (sorted Gaussian j), given the hits behind it: recovers
// T_i = T_{i+1} / (1 - alpha_i), forms dL/dalpha_i = T_i (sum_ch g_ch (c_ch - U_ch) +
// g_A (1 - U_A) + g_D (t_i - U_D)), advances U, and returns the 16-float contribution
// (dM rows + dm, dopacity + drgb) in v.  alpha comes from the same solve as in the forward
// pass, so it has the same bits.  The depth term also moves the hit's key t_i:
//   t_m = -<o',d'>/a:  dt_m/dM = -(d' v^T + p d^T)/a,  dt_m/dm = M^T d'/a;
//   t1 = t_m - r, r = sqrt((Q - D2)/a):
//                      dt1/dM = (-d' v^T - p d^T + p v^T / r + r d' d^T)/a,
//                      dt1/dm = M^T (d' - p/r)/a,
// with d' = M d, p = M v and v the closest point minus the mean.
template <bool DEPTH>
__device__ __forceinline__ void adjoint_hit(const float4* __restrict__ rec, int j, const float3 o, const float3 d,
                                            const TraceParams& P, Adjoint& s, const Upstream& g,
                                            float4 (&v)[4]) {
    const float4 g0 = __ldg(rec + 4 * j + 0);
    const float4 g1 = __ldg(rec + 4 * j + 1);
    const float4 g2 = __ldg(rec + 4 * j + 2);
    const float4 sh = __ldg(rec + 4 * j + 3);
    Hit h;
    ray_ellipsoid<false>(o, d, g0, g1, g2, P.Q, P.t_near, h);
    closest_point_accurate(o, d, g0, g1, g2, h.tm, h.p, h.v);
    const float tk = DEPTH ? hit_key_t(h, P.sort_key) : 0.f;
    const float e = expf(__fmul_rn(-0.5f, h.D2));
    const float a = __fmul_rn(sh.x, e);
    const float om = __fsub_rn(1.f, a);
    const float Ti = __fdiv_rn(s.Tn, om);
    const float w = Ti * a;
    // the eps2 estimator replaces what the first replayed (last composited) hit sees behind it
    const bool over = s.OA >= 0.f;
    const float B0 = over ? s.O0 : s.U0, B1 = over ? s.O1 : s.U1, B2 = over ? s.O2 : s.U2;
    const float BA = over ? s.OA : s.UA;
    s.OA = -1.f;
    float dLda = Ti * (g.c[0] * (sh.y - B0) + g.c[1] * (sh.z - B1) + g.c[2] * (sh.w - B2) + g.a * (1.f - BA));
    if (DEPTH) dLda = fmaf(Ti, g.d * (tk - s.UD), dLda);
    s.U0 = fmaf(a, sh.y, om * s.U0);
    s.U1 = fmaf(a, sh.z, om * s.U1);
    s.U2 = fmaf(a, sh.w, om * s.U2);
    s.UA = fmaf(om, s.UA, a);
    if (DEPTH) s.UD = fmaf(a, tk, om * s.UD);
    s.Tn = Ti;
    const float gD2 = -0.5f * a * dLda;
    const float q0 = 2.f * gD2 * h.p[0], q1 = 2.f * gD2 * h.p[1], q2 = 2.f * gD2 * h.p[2];
    const float dm0 = -(g0.x * q0 + g1.x * q1 + g2.x * q2);  // dL/dm = -M^T (2 gD2 p)
    const float dm1 = -(g0.y * q0 + g1.y * q1 + g2.y * q2);
    const float dm2 = -(g0.z * q0 + g1.z * q1 + g2.z * q2);
    v[0] = make_float4(q0 * h.v[0], q0 * h.v[1], q0 * h.v[2], dm0);
    v[1] = make_float4(q1 * h.v[0], q1 * h.v[1], q1 * h.v[2], dm1);
    v[2] = make_float4(q2 * h.v[0], q2 * h.v[1], q2 * h.v[2], dm2);
    v[3] = make_float4(dLda * e, g.c[0] * w, g.c[1] * w, g.c[2] * w);
    const float gt = DEPTH ? g.d * w : 0.f;  // dL/dt_i: depth = sum w_i t_i
    if (DEPTH && gt != 0.f) {
        const float dd[3] = {d.x, d.y, d.z};
        const float4 rows[3] = {g0, g1, g2};
        float dp[3];  // d' = M d
#pragma unroll
        for (int k = 0; k < 3; ++k) dp[k] = rows[k].x * d.x + rows[k].y * d.y + rows[k].z * d.z;
        const float aa = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
        const bool t1key = P.sort_key == 0;
        const float rr = t1key ? sqrtf(fmaxf(P.Q - h.D2, 0.f) / aa) : 0.f;  // half chord
        const float ir = t1key ? 1.f / fmaxf(rr, 1e-20f) : 0.f;
        const float ga = gt / aa;
        float x[3];  // d' - p/r (t1) or d' (t_m): dt/dm = M^T x / a
#pragma unroll
        for (int k = 0; k < 3; ++k) x[k] = dp[k] - h.p[k] * ir;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            // row k of dt/dM: (-d'_k + p_k / r) v^T + (-p_k + r d'_k) d^T
            const float cv = -dp[k] + h.p[k] * ir, cd = -h.p[k] + rr * dp[k];
            v[k].x += ga * (cv * h.v[0] + cd * dd[0]);
            v[k].y += ga * (cv * h.v[1] + cd * dd[1]);
            v[k].z += ga * (cv * h.v[2] + cd * dd[2]);
        }
        v[0].w += ga * (rows[0].x * x[0] + rows[1].x * x[1] + rows[2].x * x[2]);
        v[1].w += ga * (rows[0].y * x[0] + rows[1].y * x[1] + rows[2].y * x[2]);
        v[2].w += ga * (rows[0].z * x[0] + rows[1].z * x[1] + rows[2].z * x[2]);
    }
}

// ---------------------------------------------------------------------------------------------
// Forward: one streaming pass per ray.
//
// Near-first stack traversal; a register buffer holds up to K *pending* hits (found, not yet
// composited) in (t1, id) order.  The stack keeps, per entry, the running minimum of the box
// entries below it, so after each node the smallest entry t_min of every box still to visit is
// known: a pending hit with t1 < t_min can no longer be preceded by an undiscovered hit, and is
// composited at once (Eq. 3); the ray stops traversing as soon as T < eps1 or k_max hits are
// composited (Sec. 3).  If the buffer overflows, the pass keeps exactness with a key cap (no
// hit at or beyond a dropped key is accepted or composited) and a new pass resumes after the
// last composited key -- so the composited sequence is always the exact sorted prefix.
// ---------------------------------------------------------------------------------------------
template <int K, bool COUNT>
__device__ __forceinline__ void trace_forward(const float4* __restrict__ rec, const float4* __restrict__ sph, const NodeSrc& nodes,
                                              const TraceParams& P, int64_t pix, const float3 o, const float3 d, float& C0,
                                              float& C1, float& C2, float& T, float& depth,
                                              int64_t& last_key, int& count, Counters& cnt, int* err) {
    const float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    const int jb = key_id_bits(P.n_gauss);  // id bits of the ordering keys
    const float eps = fmaxf(P.eps1, 1e-30f);
    const float INF = __int_as_float(0x7f800000);
    T = 1.f;
    C0 = C1 = C2 = 0.f;
    depth = 0.f;
    count = 0;
    last_key = -1;
    int64_t lo_key = -1;
    bool done = false;
    int passes = 0;
    int st_node[kStackSize];
    float st_e[kStackSize], st_b[kStackSize];
    while (!done) {
        if (++passes > P.max_rounds) {
            atomicOr(err, kErrLoopGuard);
            break;
        }
        if (COUNT) cnt.rounds++;
        int64_t keys[K];
#pragma unroll
        for (int s = 0; s < K; ++s) {
            keys[s] = kEmptyKey;
        }
        int64_t cap = kEmptyKey;  // hits must have key < cap (tightened on overflow)
        const float tlo = lo_key < 0 ? P.t_near : key_t(lo_key);
        int sp = 0, node = nodes.root, visits = 0;
        auto composite_front = [&]() {
            const int64_t key = keys[0];
            const int j = key_j(key, jb);
            Hit hc;  // the same solve as at insertion time: the same bits
            ray_ellipsoid<false>(o, d, __ldg(rec + 4 * j + 0), __ldg(rec + 4 * j + 1), __ldg(rec + 4 * j + 2), P.Q,
                                 P.t_near, hc);
            const float4 sh = __ldg(rec + 4 * j + 3);
            const float a = response_alpha(sh.x, hc.D2);
            const float w = __fmul_rn(T, a);
            C0 = fmaf(w, sh.y, C0);
            C1 = fmaf(w, sh.z, C1);
            C2 = fmaf(w, sh.w, C2);
            depth = fmaf(w, key_t(key), depth);
            T = __fmul_rn(T, __fsub_rn(1.f, a));
            if (count < P.list_cap) P.ids[pix * P.list_cap + count] = j;  // for the adjoint's list replay
            ++count;
            last_key = key;
            if (COUNT) cnt.hits++;
            if (T < eps || count >= P.k_max) done = true;
            kbuf_pop_front<K>(keys, kEmptyKey);
        };
        while (true) {
            if (++visits > P.max_visits) {
                atomicOr(err, kErrLoopGuard);
                done = true;
                break;
            }
            float4 n0, n1, n2, n3;
            fetch_node(nodes, node, n0, n1, n2, n3);
            if (COUNT) cnt.nodes++;
            float en0, ex0, en1, ex1;
            slab2(n0, n1, n2, o, inv, en0, ex0, en1, ex1);
            const int r0 = __float_as_int(n3.x), r1 = __float_as_int(n3.y);
            const int c0 = __float_as_int(n3.z), c1 = __float_as_int(n3.w);
            float e0 = fmaxf(en0, tlo), e1 = fmaxf(en1, tlo);
            bool h0, h1;
            {
                const float tcap = cap == kEmptyKey ? INF : key_t(cap);
                const bool full = keys[K - 1] != kEmptyKey;
                const float tK = full ? key_t(keys[K - 1]) : INF;
                h0 = e0 <= fminf(ex0, tcap);
                h1 = e1 <= fminf(ex1, tcap);
                if (h0 && e0 > tK) { h0 = false; cap = min(cap, pack_key(e0, 0)); }
                if (h1 && e1 > tK) { h1 = false; cap = min(cap, pack_key(e1, 0)); }
            }
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const bool hs = side ? h1 : h0;
                const int rr = side ? r1 : r0;
                if (hs && rr < 0) {
                    const int start = ~rr, num = leaf_count(nodes, ~rr, side ? c1 : c0);
                    for (int q = start; q < start + num; ++q) {
                        if (!sphere_may_hit(o, d, __ldg(sph + q))) continue;
                        const float4 g0 = __ldg(rec + 4 * q + 0);
                        const float4 g1 = __ldg(rec + 4 * q + 1);
                        const float4 g2 = __ldg(rec + 4 * q + 2);
                        Hit h;
                        ray_ellipsoid<false>(o, d, g0, g1, g2, P.Q, P.t_near, h);
                        if (COUNT) cnt.tests++;
                        if (h.hit) {
                            const int64_t key = hit_key(h, P.sort_key, q, jb);
                            if (key > lo_key && key < cap) {
                                if (key < keys[K - 1]) {
                                    if (keys[K - 1] != kEmptyKey) cap = keys[K - 1];  // evicted
                                    kbuf_insert_asc<K>(keys, key);
                                    if (COUNT) cnt.inserted++;
                                } else {
                                    cap = key;  // rejected: buffer full of nearer hits
                                }
                            }
                        }
                    }
                }
            }
            bool i0 = h0 && r0 >= 0, i1 = h1 && r1 >= 0;
            {
                const float tcap = cap == kEmptyKey ? INF : key_t(cap);
                const bool full = keys[K - 1] != kEmptyKey;
                const float tK = full ? key_t(keys[K - 1]) : INF;
                if (i0 && e0 > tcap) i0 = false;
                if (i1 && e1 > tcap) i1 = false;
                if (i0 && e0 > tK) { i0 = false; cap = min(cap, pack_key(e0, 0)); }
                if (i1 && e1 > tK) { i1 = false; cap = min(cap, pack_key(e1, 0)); }
            }
            const float top = sp > 0 ? st_b[sp - 1] : INF;
            int next = -1;
            float bound = INF;
            if (i0 && i1) {
                const bool first0 = e0 <= e1;
                const int nf = first0 ? r0 : r1, ns = first0 ? r1 : r0;
                const float ef = first0 ? e0 : e1, es = first0 ? e1 : e0;
                if (sp < kStackSize) {
                    st_node[sp] = ns;
                    st_e[sp] = es;
                    st_b[sp] = fminf(es, top);
                    ++sp;
                } else {
                    atomicOr(err, kErrStack);
                }
                next = nf;
                bound = fminf(ef, st_b[sp - 1]);
            } else if (i0) {
                next = r0;
                bound = fminf(e0, top);
            } else if (i1) {
                next = r1;
                bound = fminf(e1, top);
            } else {
                const float tcap = cap == kEmptyKey ? INF : key_t(cap);
                const bool full = keys[K - 1] != kEmptyKey;
                const float tK = full ? key_t(keys[K - 1]) : INF;
                while (sp > 0) {
                    --sp;
                    const float e = st_e[sp];
                    if (e > tcap) continue;
                    if (e > tK) {
                        cap = min(cap, pack_key(e, 0));
                        continue;
                    }
                    next = st_node[sp];
                    bound = fminf(e, sp > 0 ? st_b[sp - 1] : INF);
                    break;
                }
            }
            // composite every pending hit that no unvisited box can precede
            while (!done && keys[0] != kEmptyKey && key_t(keys[0]) < bound) composite_front();
            if (done || next < 0) break;
            node = next;
        }
        while (!done && keys[0] != kEmptyKey) composite_front();
        if (!done) {
            if (cap == kEmptyKey) done = true;  // every hit beyond lo_key was seen
            else lo_key = last_key;             // overflow: resume after the last composited hit
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Adjoint: the mirror image.  Far-first traversal (by box exit), a descending buffer of pending
// hits with key below the upper bound (initially just above the last composited key), and a
// running maximum of the stacked box exits: a pending hit with t1 above it is the farthest
// unprocessed hit and is replayed at once, back to front.  Boxes entering beyond the last
// composited hit are pruned.  Overflow is handled with a key floor and a further pass.
// ---------------------------------------------------------------------------------------------
template <int K, bool COUNT, bool DEPTH>
__device__ __forceinline__ void trace_backward(const float4* __restrict__ rec, const float4* __restrict__ sph, const NodeSrc& nodes,
                                               const TraceParams& P, const float3 o, const float3 d, float T_final,
                                               int64_t last_key, int n_hits, const Upstream& g,
                                               float4* __restrict__ gtmp, Counters& cnt, int* err) {
    if (n_hits <= 0) return;
    const float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    const int jb = key_id_bits(P.n_gauss);  // id bits of the ordering keys
    const float NINF = __int_as_float(0xff800000);
    constexpr uint32_t kFloorJ = kKeyLowMax;  // the largest key at a given t
    int64_t hi_key = last_key + 1;  // exclusive upper bound
    Adjoint adj = adjoint_start(P, T_final, g);
    int remaining = n_hits;
    int passes = 0;
    int st_node[kStackSize];
    float st_x[kStackSize], st_b[kStackSize];
    while (remaining > 0) {
        if (++passes > P.max_rounds) {
            atomicOr(err, kErrLoopGuard);
            break;
        }
        if (COUNT) cnt.rounds++;
        int64_t keys[K];
#pragma unroll
        for (int s = 0; s < K; ++s) {
            keys[s] = kEmptyKeyDesc;
        }
        int64_t floor_key = -1;  // hits must have key > floor_key (raised on overflow)
        const float thi = key_t(hi_key);
        int sp = 0, node = nodes.root, visits = 0;
        bool stop = false;
        auto replay_front = [&]() {
            const int64_t key = keys[0];
            const int j = key_j(key, jb);
            float4 v[4];
            adjoint_hit<DEPTH>(rec, j, o, d, P, adj, g, v);
            float4* gp = gtmp + 4 * j;
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(gp + k, v[k]);
            --remaining;
            hi_key = key;
            if (COUNT) cnt.hits++;
            kbuf_pop_front<K>(keys, kEmptyKeyDesc);
        };
        while (true) {
            if (++visits > P.max_visits) {
                atomicOr(err, kErrLoopGuard);
                stop = true;
                break;
            }
            float4 n0, n1, n2, n3;
            fetch_node(nodes, node, n0, n1, n2, n3);
            if (COUNT) cnt.nodes++;
            float en0, ex0, en1, ex1;
            slab2(n0, n1, n2, o, inv, en0, ex0, en1, ex1);
            const int r0 = __float_as_int(n3.x), r1 = __float_as_int(n3.y);
            const int c0 = __float_as_int(n3.z), c1 = __float_as_int(n3.w);
            bool h0, h1;
            {
                const float tfl = floor_key < 0 ? P.t_near : fmaxf(P.t_near, key_t(floor_key));
                const bool full = keys[K - 1] != kEmptyKeyDesc;
                const float tK = full ? key_t(keys[K - 1]) : NINF;
                h0 = en0 <= thi && ex0 >= tfl && ex0 >= en0;
                h1 = en1 <= thi && ex1 >= tfl && ex1 >= en1;
                if (h0 && ex0 < tK) { h0 = false; floor_key = max(floor_key, pack_key(ex0, kFloorJ)); }
                if (h1 && ex1 < tK) { h1 = false; floor_key = max(floor_key, pack_key(ex1, kFloorJ)); }
            }
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const bool hs = side ? h1 : h0;
                const int rr = side ? r1 : r0;
                if (hs && rr < 0) {
                    const int start = ~rr, num = leaf_count(nodes, ~rr, side ? c1 : c0);
                    for (int q = start; q < start + num; ++q) {
                        if (!sphere_may_hit(o, d, __ldg(sph + q))) continue;
                        const float4 g0 = __ldg(rec + 4 * q + 0);
                        const float4 g1 = __ldg(rec + 4 * q + 1);
                        const float4 g2 = __ldg(rec + 4 * q + 2);
                        Hit h;
                        ray_ellipsoid<false>(o, d, g0, g1, g2, P.Q, P.t_near, h);
                        if (COUNT) cnt.tests++;
                        if (h.hit) {
                            const int64_t key = hit_key(h, P.sort_key, q, jb);
                            if (key < hi_key && key > floor_key) {
                                if (key > keys[K - 1]) {
                                    if (keys[K - 1] != kEmptyKeyDesc) floor_key = keys[K - 1];  // evicted
                                    kbuf_insert_desc<K>(keys, key);
                                    if (COUNT) cnt.inserted++;
                                } else {
                                    floor_key = key;
                                }
                            }
                        }
                    }
                }
            }
            bool i0 = h0 && r0 >= 0, i1 = h1 && r1 >= 0;
            {
                const float tfl = floor_key < 0 ? P.t_near : fmaxf(P.t_near, key_t(floor_key));
                const bool full = keys[K - 1] != kEmptyKeyDesc;
                const float tK = full ? key_t(keys[K - 1]) : NINF;
                if (i0 && ex0 < tfl) i0 = false;
                if (i1 && ex1 < tfl) i1 = false;
                if (i0 && ex0 < tK) { i0 = false; floor_key = max(floor_key, pack_key(ex0, kFloorJ)); }
                if (i1 && ex1 < tK) { i1 = false; floor_key = max(floor_key, pack_key(ex1, kFloorJ)); }
            }
            const float top = sp > 0 ? st_b[sp - 1] : NINF;
            int next = -1;
            float bound = NINF;
            if (i0 && i1) {
                const bool first0 = ex0 >= ex1;
                const int nf = first0 ? r0 : r1, ns = first0 ? r1 : r0;
                const float xf = first0 ? ex0 : ex1, xs = first0 ? ex1 : ex0;
                if (sp < kStackSize) {
                    st_node[sp] = ns;
                    st_x[sp] = xs;
                    st_b[sp] = fmaxf(xs, top);
                    ++sp;
                } else {
                    atomicOr(err, kErrStack);
                }
                next = nf;
                bound = fmaxf(xf, st_b[sp - 1]);
            } else if (i0) {
                next = r0;
                bound = fmaxf(ex0, top);
            } else if (i1) {
                next = r1;
                bound = fmaxf(ex1, top);
            } else {
                const float tfl = floor_key < 0 ? P.t_near : fmaxf(P.t_near, key_t(floor_key));
                const bool full = keys[K - 1] != kEmptyKeyDesc;
                const float tK = full ? key_t(keys[K - 1]) : NINF;
                while (sp > 0) {
                    --sp;
                    const float x = st_x[sp];
                    if (x < tfl) continue;
                    if (x < tK) {
                        floor_key = max(floor_key, pack_key(x, kFloorJ));
                        continue;
                    }
                    next = st_node[sp];
                    bound = fmaxf(x, sp > 0 ? st_b[sp - 1] : NINF);
                    break;
                }
            }
            // replay every pending hit that no unvisited box can follow
            while (remaining > 0 && keys[0] != kEmptyKeyDesc && key_t(keys[0]) > bound) replay_front();
            if (remaining == 0 || next < 0) break;
            node = next;
        }
        if (stop) break;
        while (remaining > 0 && keys[0] != kEmptyKeyDesc) replay_front();
        if (remaining > 0 && floor_key < 0) {
            atomicOr(err, kErrReplayMismatch);  // the forward saw hits that this pass did not
            break;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Warp-aggregated gradient scatter (the depth-first packet adjoint; the whole warp calls it,
// converged; the best-first re-traversal and the list replay use per-lane atomics instead).
// Each lane offers its 16-float contribution (dM rows + dm, dopacity + drgb) to the Gaussian
// in Morton position j (j < 0: nothing).  Lanes holding a Gaussian nobody else holds issue
// their four float4 atomics at once; lanes sharing a Gaussian are summed into the group's
// lowest lane first (shuffles), which then issues one set of atomics for the group.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void scatter_grad_warp(float4* __restrict__ gtmp, int j, const float4 (&v)[4]) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(FULL, j);
    const bool mine = j >= 0;
    const bool single = mine && __popc(peers) == 1;
    if (single) {
        float4* gp = gtmp + 4 * j;
#pragma unroll
        for (int k = 0; k < 4; ++k) atomicAdd(gp + k, v[k]);
    }
    unsigned todo = __ballot_sync(FULL, mine && !single);
    while (todo) {
        const int lead = __ffs(todo) - 1;
        const unsigned grp = __shfl_sync(FULL, peers, lead);
        const bool in = (grp >> lane) & 1u;
        const bool small = __popc(grp) <= 4;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float4 x = in ? v[k] : make_float4(0.f, 0.f, 0.f, 0.f);
            if (small) {
                // gather: the leader adds the other members' values one lane at a time
                unsigned rest = grp & ~(1u << lead);
                float4 acc = x;
                while (rest) {
                    const int src = __ffs(rest) - 1;
                    rest &= rest - 1;
                    acc.x += __shfl_sync(FULL, x.x, src);
                    acc.y += __shfl_sync(FULL, x.y, src);
                    acc.z += __shfl_sync(FULL, x.z, src);
                    acc.w += __shfl_sync(FULL, x.w, src);
                }
                x = acc;
            } else {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    x.x += __shfl_xor_sync(FULL, x.x, off);
                    x.y += __shfl_xor_sync(FULL, x.y, off);
                    x.z += __shfl_xor_sync(FULL, x.z, off);
                    x.w += __shfl_xor_sync(FULL, x.w, off);
                }
            }
            if (lane == lead) atomicAdd(gtmp + 4 * j + k, x);
        }
        todo &= ~grp;
    }
}

// ---------------------------------------------------------------------------------------------
// Gradient scatter through the bulk-copy (TMA) unit: a lane's 64 B contribution to one Gaussian
// (dM rows + dm, dopacity + drgb, see adjoint_hit) goes to one of the lane's two staging slots
// in shared memory and is added to the Gaussian's accumulator by one bulk reduction
// (cp.reduce.async.bulk .add.f32: relaxed atomic additions at GPU scope, element by element).
// The float4 atomics it replaces cost per instruction, not per byte (four per hit); one 64 B
// bulk reduction per hit took 38 % off the list replay.  Each lane tracks its own bulk groups:
// a slot is rewritten only after the reduction that last read it has read it, and drain()
// waits until every reduction of the lane has been performed.  The re-traversal adjoint keeps
// its float4 atomics: it issues them at a fifth of the list replay's rate, below what the L2
// sustains, and the bulk path's extra instructions made it 6 % slower (measured).
// ---------------------------------------------------------------------------------------------
struct BulkScatter {
    static constexpr int kFloat4 = 8;  // staging float4 per thread: two 64 B slots
    float4* stage;  // this thread's kFloat4 staging float4 in shared memory (16 B aligned)
    int buf;
    __device__ __forceinline__ explicit BulkScatter(float4* s) : stage(s), buf(0) {}
    // acc: the Gaussian's 64 B accumulator in global memory (16 B aligned)
    __device__ __forceinline__ void add(float4* acc, const float4 (&v)[4]) {
        float4* st = stage + 4 * buf;
        asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 4; ++q) st[q] = v[q];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the stores, seen by the bulk copy
        const size_t gaddr = __cvta_generic_to_global(acc);
        const uint32_t saddr = (uint32_t)__cvta_generic_to_shared(st);
        asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], 64;"
                     :: "l"(gaddr), "r"(saddr) : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        buf ^= 1;
    }
    __device__ __forceinline__ void drain() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
};

// ---------------------------------------------------------------------------------------------
// List replay (the paper's index-buffer adjoint, Sec. 3 and Sec. 5): the forward pass wrote
// the sorted ids of each ray's first list_cap composited hits; a ray with n <= list_cap hits is
// replayed from that list back to front, with no traversal.  Lanes replay different Gaussians
// at any one step, so each lane scatters its own contributions (BulkScatter; warp aggregation,
// which pays in the packet re-traversal where lanes share Gaussians, costs more here than it
// saves).
// ---------------------------------------------------------------------------------------------
template <bool COUNT, bool DEPTH>
__device__ __forceinline__ void replay_list(const float4* __restrict__ rec, const TraceParams& P, int64_t pix,
                                            const float3 o, const float3 d, float T_final, int n, const Upstream& g, float4* __restrict__ gtmp, Counters& cnt, int* err,
                                            BulkScatter& sc) {
    Adjoint s = adjoint_start(P, T_final, g);
    const int* row = P.ids + (n > 0 ? pix * P.list_cap : 0);
    int k = n > 0 ? n : 0;
    while (__any_sync(0xffffffffu, k > 0)) {
        int jout = -1;
        float4 v[4];
        if (k > 0) {
            --k;
            const int j = __ldg(row + k);
            if (j >= 0 && j < P.n_gauss) {
                adjoint_hit<DEPTH>(rec, j, o, d, P, s, g, v);
                jout = j;
                if (COUNT) cnt.hits++;
            } else {  // a corrupt list: report and stop this ray
                atomicOr(err, kErrIndex);
                k = 0;
            }
        }
        if (jout >= 0) sc.add(gtmp + 4 * jout, v);
    }
}

// ---------------------------------------------------------------------------------------------
// Warp-packet variants.  The 32 lanes of a warp (one ray tile) traverse together: the node
// sequence is shared (uniform loads are broadcast, descent is decided by warp votes: a child
// is visited when any active lane needs it), while each lane keeps its own streaming state --
// pending buffer, key cap, and per-lane stack entries (a lane that does not need a stacked box
// records +inf, so its finalisation bound is unaffected).  The result of every lane is exactly
// that of the per-ray traversal: a lane only tests the boxes and Gaussians it would have
// tested, in an order that does not change what it composites.
// ---------------------------------------------------------------------------------------------
template <int K, bool COUNT>
__device__ __forceinline__ void trace_forward_packet(const float4* __restrict__ rec, const float4* __restrict__ sph, const NodeSrc& nodes,
                                                     const TraceParams& P, int64_t pix, bool valid, const float3 o,
                                                     const float3 d, float& C0, float& C1, float& C2, float& T,
                                                     float& depth, int64_t& last_key, int& count, Counters& cnt,
                                                     int* err) {
    const unsigned FULL = 0xffffffffu;
    const float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    const int jb = key_id_bits(P.n_gauss);  // id bits of the ordering keys
    const float eps = fmaxf(P.eps1, 1e-30f);
    const float INF = __int_as_float(0x7f800000);
    T = 1.f;
    C0 = C1 = C2 = 0.f;
    depth = 0.f;
    count = 0;
    last_key = -1;
    int64_t lo_key = -1;
    bool done = !valid;
    int passes = 0;
    int st_node[kStackSize];
    float st_e[kStackSize], st_b[kStackSize];
    while (__any_sync(FULL, !done)) {
        if (++passes > P.max_rounds) {
            if ((threadIdx.x & 31) == 0) atomicOr(err, kErrLoopGuard);
            break;
        }
        if (COUNT && !done) cnt.rounds++;
        bool active = !done;
        int64_t keys[K];
#pragma unroll
        for (int s = 0; s < K; ++s) {
            keys[s] = kEmptyKey;
        }
        int64_t cap = kEmptyKey;
        const float tlo = lo_key < 0 ? P.t_near : key_t(lo_key);
        int sp = 0, node = nodes.root, visits = 0;
        auto composite_front = [&]() {
            const int64_t key = keys[0];
            const int j = key_j(key, jb);
            Hit hc;  // the same solve as at insertion time: the same bits
            ray_ellipsoid<false>(o, d, __ldg(rec + 4 * j + 0), __ldg(rec + 4 * j + 1), __ldg(rec + 4 * j + 2), P.Q,
                                 P.t_near, hc);
            const float4 sh = __ldg(rec + 4 * j + 3);
            const float a = response_alpha(sh.x, hc.D2);
            const float w = __fmul_rn(T, a);
            C0 = fmaf(w, sh.y, C0);
            C1 = fmaf(w, sh.z, C1);
            C2 = fmaf(w, sh.w, C2);
            depth = fmaf(w, key_t(key), depth);
            T = __fmul_rn(T, __fsub_rn(1.f, a));
            if (count < P.list_cap) P.ids[pix * P.list_cap + count] = j;  // for the adjoint's list replay
            ++count;
            last_key = key;
            if (COUNT) cnt.hits++;
            if (T < eps || count >= P.k_max) done = true;
            kbuf_pop_front<K>(keys, kEmptyKey);
        };
        while (true) {
            if (++visits > P.max_visits) {
                if ((threadIdx.x & 31) == 0) atomicOr(err, kErrLoopGuard);
                done = true;
                break;
            }
            float4 n0, n1, n2, n3;
            fetch_node(nodes, node, n0, n1, n2, n3);
            if (COUNT && active) cnt.nodes++;
            if (COUNT && (threadIdx.x & 31) == 0) cnt.wnodes++;
            float en0, ex0, en1, ex1;
            slab2(n0, n1, n2, o, inv, en0, ex0, en1, ex1);
            const int r0 = __float_as_int(n3.x), r1 = __float_as_int(n3.y);
            const int c0 = __float_as_int(n3.z), c1 = __float_as_int(n3.w);
            const float e0 = fmaxf(en0, tlo), e1 = fmaxf(en1, tlo);
            bool h0 = false, h1 = false;
            if (active) {
                const float tcap = cap == kEmptyKey ? INF : key_t(cap);
                const bool full = keys[K - 1] != kEmptyKey;
                const float tK = full ? key_t(keys[K - 1]) : INF;
                h0 = e0 <= fminf(ex0, tcap);
                h1 = e1 <= fminf(ex1, tcap);
                if (h0 && e0 > tK) { h0 = false; cap = min(cap, pack_key(e0, 0)); }
                if (h1 && e1 > tK) { h1 = false; cap = min(cap, pack_key(e1, 0)); }
            }
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int rr = side ? r1 : r0;
                const bool want = (side ? h1 : h0) && rr < 0;
                if (__any_sync(FULL, want)) {
                    const int start = ~rr, num = leaf_count(nodes, ~rr, side ? c1 : c0);
                    for (int q = start; q < start + num; ++q) {
                        if (COUNT && (threadIdx.x & 31) == 0) cnt.wleaf++;
                        if (want && sphere_may_hit(o, d, __ldg(sph + q))) {
                            const float4 g0 = __ldg(rec + 4 * q + 0);
                            const float4 g1 = __ldg(rec + 4 * q + 1);
                            const float4 g2 = __ldg(rec + 4 * q + 2);
                            Hit h;
                            ray_ellipsoid<false>(o, d, g0, g1, g2, P.Q, P.t_near, h);
                            if (COUNT) cnt.tests++;
                            if (h.hit) {
                                const int64_t key = hit_key(h, P.sort_key, q, jb);
                                if (key > lo_key && key < cap) {
                                    if (key < keys[K - 1]) {
                                        if (keys[K - 1] != kEmptyKey) cap = keys[K - 1];
                                        kbuf_insert_asc<K>(keys, key);
                                        if (COUNT) cnt.inserted++;
                                    } else {
                                        cap = key;
                                    }
                                }
                            }
                        }
                    }
                }
            }
            bool i0 = h0 && r0 >= 0, i1 = h1 && r1 >= 0;
            if (active) {
                const float tcap = cap == kEmptyKey ? INF : key_t(cap);
                const bool full = keys[K - 1] != kEmptyKey;
                const float tK = full ? key_t(keys[K - 1]) : INF;
                if (i0 && e0 > tcap) i0 = false;
                if (i1 && e1 > tcap) i1 = false;
                if (i0 && e0 > tK) { i0 = false; cap = min(cap, pack_key(e0, 0)); }
                if (i1 && e1 > tK) { i1 = false; cap = min(cap, pack_key(e1, 0)); }
            }
            const bool any0 = __any_sync(FULL, i0), any1 = __any_sync(FULL, i1);
            const float top = sp > 0 ? st_b[sp - 1] : INF;
            int next = -1;
            float bound = INF;
            if (any0 && any1) {
                const int v0 = __popc(__ballot_sync(FULL, i0 && (!i1 || e0 <= e1)));
                const int v1 = __popc(__ballot_sync(FULL, i1 && (!i0 || e1 < e0)));
                const bool first0 = v0 >= v1;
                const int nf = first0 ? r0 : r1, ns = first0 ? r1 : r0;
                const bool need_f = first0 ? i0 : i1, need_s = first0 ? i1 : i0;
                const float ef = first0 ? e0 : e1, es = first0 ? e1 : e0;
                if (sp < kStackSize) {
                    st_node[sp] = ns;
                    st_e[sp] = need_s ? es : INF;
                    st_b[sp] = fminf(st_e[sp], top);
                    ++sp;
                } else if ((threadIdx.x & 31) == 0) {
                    atomicOr(err, kErrStack);
                }
                next = nf;
                bound = fminf(need_f ? ef : INF, sp > 0 ? st_b[sp - 1] : INF);
            } else if (any0) {
                next = r0;
                bound = fminf(i0 ? e0 : INF, top);
            } else if (any1) {
                next = r1;
                bound = fminf(i1 ? e1 : INF, top);
            } else {
                while (sp > 0) {
                    --sp;
                    const float e = st_e[sp];
                    bool need = false;
                    if (active && e != INF) {
                        const float tcap = cap == kEmptyKey ? INF : key_t(cap);
                        const bool full = keys[K - 1] != kEmptyKey;
                        const float tK = full ? key_t(keys[K - 1]) : INF;
                        if (e <= tcap) {
                            if (e > tK) cap = min(cap, pack_key(e, 0));
                            else need = true;
                        }
                    }
                    if (__any_sync(FULL, need)) {
                        next = st_node[sp];
                        bound = fminf(need ? e : INF, sp > 0 ? st_b[sp - 1] : INF);
                        break;
                    }
                }
            }
            // (bound is +inf once no node is left: everything pending is composited)
            while (active && !done && keys[0] != kEmptyKey && key_t(keys[0]) < bound) composite_front();
            active = active && !done;
            if (next < 0 || !__any_sync(FULL, active)) break;
            node = next;
        }
        if (active && !done) {
            if (cap == kEmptyKey) done = true;
            else lo_key = last_key;
        }
    }
}

template <int K, bool COUNT, bool DEPTH>
__device__ __forceinline__ void trace_backward_packet(const float4* __restrict__ rec,
                                                      const float4* __restrict__ sph, const NodeSrc& nodes,
                                                      const TraceParams& P,
                                                      const float3 o, const float3 d, float T_final,
                                                      int64_t last_key, int n_hits, const Upstream& g,
                                                      float4* __restrict__ gtmp, Counters& cnt, int* err) {
    const unsigned FULL = 0xffffffffu;
    const float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    const int jb = key_id_bits(P.n_gauss);  // id bits of the ordering keys
    const float NINF = __int_as_float(0xff800000);
    constexpr uint32_t kFloorJ = kKeyLowMax;  // the largest key at a given t
    int64_t hi_key = last_key + 1;
    Adjoint adj = adjoint_start(P, T_final, g);
    int remaining = n_hits > 0 ? n_hits : 0;
    int passes = 0;
    int st_node[kStackSize];
    float st_x[kStackSize], st_b[kStackSize];
    while (__any_sync(FULL, remaining > 0)) {
        if (++passes > P.max_rounds) {
            if ((threadIdx.x & 31) == 0) atomicOr(err, kErrLoopGuard);
            break;
        }
        if (COUNT && remaining > 0) cnt.rounds++;
        bool active = remaining > 0;
        int64_t keys[K];
#pragma unroll
        for (int s = 0; s < K; ++s) {
            keys[s] = kEmptyKeyDesc;
        }
        int64_t floor_key = -1;
        const float thi = key_t(hi_key);
        int sp = 0, node = nodes.root, visits = 0;
        bool stop = false;
        auto replay_contrib = [&](int& jout, float4 (&vout)[4]) {
            const int64_t key = keys[0];
            const int j = key_j(key, jb);
            adjoint_hit<DEPTH>(rec, j, o, d, P, adj, g, vout);
            jout = j;
            --remaining;
            hi_key = key;
            if (COUNT) cnt.hits++;
            kbuf_pop_front<K>(keys, kEmptyKeyDesc);
        };
        // warp-uniform replay: every lane takes part in the aggregated scatter
        auto replay_while = [&](auto cond) {
            while (true) {
                const bool c = cond();
                if (!__any_sync(0xffffffffu, c)) break;
                int jout = -1;
                float4 vout[4];
                if (c) replay_contrib(jout, vout);
                scatter_grad_warp(gtmp, jout, vout);
            }
        };
        while (true) {
            if (++visits > P.max_visits) {
                if ((threadIdx.x & 31) == 0) atomicOr(err, kErrLoopGuard);
                stop = true;
                break;
            }
            float4 n0, n1, n2, n3;
            fetch_node(nodes, node, n0, n1, n2, n3);
            if (COUNT && active) cnt.nodes++;
            if (COUNT && (threadIdx.x & 31) == 0) cnt.wnodes++;
            float en0, ex0, en1, ex1;
            slab2(n0, n1, n2, o, inv, en0, ex0, en1, ex1);
            const int r0 = __float_as_int(n3.x), r1 = __float_as_int(n3.y);
            const int c0 = __float_as_int(n3.z), c1 = __float_as_int(n3.w);
            bool h0 = false, h1 = false;
            if (active) {
                const float tfl = floor_key < 0 ? P.t_near : fmaxf(P.t_near, key_t(floor_key));
                const bool full = keys[K - 1] != kEmptyKeyDesc;
                const float tK = full ? key_t(keys[K - 1]) : NINF;
                h0 = en0 <= thi && ex0 >= tfl && ex0 >= en0;
                h1 = en1 <= thi && ex1 >= tfl && ex1 >= en1;
                if (h0 && ex0 < tK) { h0 = false; floor_key = max(floor_key, pack_key(ex0, kFloorJ)); }
                if (h1 && ex1 < tK) { h1 = false; floor_key = max(floor_key, pack_key(ex1, kFloorJ)); }
            }
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int rr = side ? r1 : r0;
                const bool want = (side ? h1 : h0) && rr < 0;
                if (__any_sync(FULL, want)) {
                    const int start = ~rr, num = leaf_count(nodes, ~rr, side ? c1 : c0);
                    for (int q = start; q < start + num; ++q) {
                        if (COUNT && (threadIdx.x & 31) == 0) cnt.wleaf++;
                        if (want && sphere_may_hit(o, d, __ldg(sph + q))) {
                            const float4 g0 = __ldg(rec + 4 * q + 0);
                            const float4 g1 = __ldg(rec + 4 * q + 1);
                            const float4 g2 = __ldg(rec + 4 * q + 2);
                            Hit h;
                            ray_ellipsoid<false>(o, d, g0, g1, g2, P.Q, P.t_near, h);
                            if (COUNT) cnt.tests++;
                            if (h.hit) {
                                const int64_t key = hit_key(h, P.sort_key, q, jb);
                                if (key < hi_key && key > floor_key) {
                                    if (key > keys[K - 1]) {
                                        if (keys[K - 1] != kEmptyKeyDesc) floor_key = keys[K - 1];
                                        kbuf_insert_desc<K>(keys, key);
                                        if (COUNT) cnt.inserted++;
                                    } else {
                                        floor_key = key;
                                    }
                                }
                            }
                        }
                    }
                }
            }
            bool i0 = h0 && r0 >= 0, i1 = h1 && r1 >= 0;
            if (active) {
                const float tfl = floor_key < 0 ? P.t_near : fmaxf(P.t_near, key_t(floor_key));
                const bool full = keys[K - 1] != kEmptyKeyDesc;
                const float tK = full ? key_t(keys[K - 1]) : NINF;
                if (i0 && ex0 < tfl) i0 = false;
                if (i1 && ex1 < tfl) i1 = false;
                if (i0 && ex0 < tK) { i0 = false; floor_key = max(floor_key, pack_key(ex0, kFloorJ)); }
                if (i1 && ex1 < tK) { i1 = false; floor_key = max(floor_key, pack_key(ex1, kFloorJ)); }
            }
            const bool any0 = __any_sync(FULL, i0), any1 = __any_sync(FULL, i1);
            const float top = sp > 0 ? st_b[sp - 1] : NINF;
            int next = -1;
            float bound = NINF;
            if (any0 && any1) {
                const int v0 = __popc(__ballot_sync(FULL, i0 && (!i1 || ex0 >= ex1)));
                const int v1 = __popc(__ballot_sync(FULL, i1 && (!i0 || ex1 > ex0)));
                const bool first0 = v0 >= v1;
                const int nf = first0 ? r0 : r1, ns = first0 ? r1 : r0;
                const bool need_f = first0 ? i0 : i1, need_s = first0 ? i1 : i0;
                const float xf = first0 ? ex0 : ex1, xs = first0 ? ex1 : ex0;
                if (sp < kStackSize) {
                    st_node[sp] = ns;
                    st_x[sp] = need_s ? xs : NINF;
                    st_b[sp] = fmaxf(st_x[sp], top);
                    ++sp;
                } else if ((threadIdx.x & 31) == 0) {
                    atomicOr(err, kErrStack);
                }
                next = nf;
                bound = fmaxf(need_f ? xf : NINF, sp > 0 ? st_b[sp - 1] : NINF);
            } else if (any0) {
                next = r0;
                bound = fmaxf(i0 ? ex0 : NINF, top);
            } else if (any1) {
                next = r1;
                bound = fmaxf(i1 ? ex1 : NINF, top);
            } else {
                while (sp > 0) {
                    --sp;
                    const float x = st_x[sp];
                    bool need = false;
                    if (active && x != NINF) {
                        const float tfl = floor_key < 0 ? P.t_near : fmaxf(P.t_near, key_t(floor_key));
                        const bool full = keys[K - 1] != kEmptyKeyDesc;
                        const float tK = full ? key_t(keys[K - 1]) : NINF;
                        if (x >= tfl) {
                            if (x < tK) floor_key = max(floor_key, pack_key(x, kFloorJ));
                            else need = true;
                        }
                    }
                    if (__any_sync(FULL, need)) {
                        next = st_node[sp];
                        bound = fmaxf(need ? x : NINF, sp > 0 ? st_b[sp - 1] : NINF);
                        break;
                    }
                }
            }
            // (bound is -inf once no node is left: everything pending is replayed)
            replay_while([&] { return active && remaining > 0 && keys[0] != kEmptyKeyDesc && key_t(keys[0]) > bound; });
            active = active && remaining > 0;
            if (next < 0 || !__any_sync(FULL, active)) break;
            node = next;
        }
        if (__any_sync(FULL, stop)) break;
        if (active && remaining > 0 && floor_key < 0) {
            atomicOr(err, kErrReplayMismatch);
            remaining = 0;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Best-first warp packets.  The warp keeps its unvisited nodes in a priority queue distributed
// over the lanes' registers (kQSlots per lane, 32 * kQSlots entries); a node's priority is the
// smallest box entry (forward) or the largest box exit (adjoint) among the lanes that need it.
// Nodes are expanded in priority order, so the queue's extreme priority is a bound valid for
// every lane: forward, no undiscovered hit of any lane precedes it, and pending hits nearer
// than it are composited at once; the adjoint mirrors this back to front.  Hits therefore
// leave the pending buffer almost as soon as they are found and one pass usually suffices.
// The queue holds 64 nodes (2 slots per lane; 4 slots measured 7 % slower).  A node displaced
// from the full queue goes to a per-warp list and returns later in the same pass; only when
// that list is full too is a node dropped, capping (flooring) the keys of every active lane,
// which keeps the result exact at the cost of a further pass.
// ---------------------------------------------------------------------------------------------
constexpr int kQSlots = 2;

// Each occupied slot holds one 32-bit key: the priority's FP32 bit pattern with its 7 low
// mantissa bits replaced by the slot's warp-wide id (lane * kQSlots + slot).  Priorities are
// >= 0, so the keys order as unsigned integers and one redux.sync finds the extreme slot.
// Forward (min-queue) priorities are rounded down and adjoint (max-queue) priorities up by at
// most 127 ulps: both only make the finalisation bounds more conservative.
struct WarpQueue {
    uint32_t key[kQSlots];
    int nd[kQSlots];
};

template <bool MAXQ>
__device__ __forceinline__ uint32_t wq_empty() {
    return MAXQ ? 0u : 0x7f80007fu;  // min-queue: +inf with no valid slot id (ids < 64)
}

template <bool MAXQ>
__device__ __forceinline__ uint32_t wq_bits(float pr) {
    if (MAXQ) return (__float_as_uint(fmaxf(pr, 1.17549435e-38f)) + 0x7fu) & ~0x7fu;  // round up, > 0
    return __float_as_uint(fmaxf(pr, 0.f)) & ~0x7fu;                                   // round down
}

template <bool MAXQ>
__device__ __forceinline__ void wq_init(WarpQueue& q) {
#pragma unroll
    for (int s = 0; s < kQSlots; ++s) {
        q.key[s] = wq_empty<MAXQ>();
        q.nd[s] = 0;
    }
}

// push a (uniform) entry; false when the queue is full
template <bool MAXQ>
__device__ __forceinline__ bool wq_push(WarpQueue& q, float pr, int node, int lane) {
    const uint32_t bits = wq_bits<MAXQ>(pr);
    int free_slot = -1;  // this lane's first empty slot
#pragma unroll
    for (int s = kQSlots - 1; s >= 0; --s)
        if (q.key[s] == wq_empty<MAXQ>()) free_slot = s;
    const unsigned m = __ballot_sync(0xffffffffu, free_slot >= 0);
    if (!m) return false;
    const int owner = __ffs(m) - 1;
    if (lane == owner) {
#pragma unroll
        for (int s = 0; s < kQSlots; ++s)
            if (free_slot == s) {
                q.key[s] = bits | (uint32_t)(owner * kQSlots + s);
                q.nd[s] = node;
            }
    }
    return true;
}

template <bool MAXQ>
__device__ __forceinline__ uint32_t wq_extreme_key(const WarpQueue& q) {
    uint32_t v = q.key[0];
#pragma unroll
    for (int s = 1; s < kQSlots; ++s) v = MAXQ ? max(v, q.key[s]) : min(v, q.key[s]);
    return MAXQ ? __reduce_max_sync(0xffffffffu, v) : __reduce_min_sync(0xffffffffu, v);
}

// pop the extreme entry, whose key v = wq_extreme_key(q) the caller already holds; returns
// false when empty
template <bool MAXQ>
__device__ __forceinline__ bool wq_pop_known(WarpQueue& q, uint32_t v, float& pr, int& node, int lane) {
    if (v == wq_empty<MAXQ>()) return false;
    const int gid = (int)(v & 0x7fu);
    const int owner = gid / kQSlots, slot = gid % kQSlots;
    int mine = q.nd[0];
#pragma unroll
    for (int s = 1; s < kQSlots; ++s)
        if (slot == s) mine = q.nd[s];
    node = __shfl_sync(0xffffffffu, mine, owner);
    pr = __uint_as_float(v & ~0x7fu);
    if (lane == owner) {
#pragma unroll
        for (int s = 0; s < kQSlots; ++s)
            if (slot == s) q.key[s] = wq_empty<MAXQ>();
    }
    return true;
}

// the priority of extreme key v: +inf (min-queue) / -inf (max-queue) for an empty queue
template <bool MAXQ>
__device__ __forceinline__ float wq_key_priority(uint32_t v) {
    if (MAXQ && v == wq_empty<MAXQ>()) return __int_as_float(0xff800000);  // min-queue: the empty key reads +inf
    return __uint_as_float(v & ~0x7fu);
}

// push with displacement: when the queue is full, the worst entry among the queue and the new
// one (largest priority for the min-queue, smallest for the max-queue) does not stay; returns
// true with its (rounded, conservative) priority and node in out_pr / out_node.
template <bool MAXQ>
__device__ __forceinline__ bool wq_push_displace(WarpQueue& q, float pr, int node, int lane, float& out_pr,
                                                 int& out_node) {
    if (wq_push<MAXQ>(q, pr, node, lane)) return false;
    uint32_t v = q.key[0];
#pragma unroll
    for (int s = 1; s < kQSlots; ++s) v = MAXQ ? min(v, q.key[s]) : max(v, q.key[s]);
    v = MAXQ ? __reduce_min_sync(0xffffffffu, v) : __reduce_max_sync(0xffffffffu, v);  // worst key
    const uint32_t nb = wq_bits<MAXQ>(pr);
    const uint32_t wb = v & ~0x7fu;
    const bool replace = MAXQ ? (wb < nb) : (wb > nb);
    if (!replace) {
        out_pr = __uint_as_float(nb);
        out_node = node;
        return true;
    }
    const int gid = (int)(v & 0x7fu);
    const int owner = gid / kQSlots, slot = gid % kQSlots;
    int mine = q.nd[0];
#pragma unroll
    for (int s = 1; s < kQSlots; ++s)
        if (slot == s) mine = q.nd[s];
    out_node = __shfl_sync(0xffffffffu, mine, owner);
    if (lane == owner) {
#pragma unroll
        for (int s = 0; s < kQSlots; ++s)
            if (slot == s) {
                q.key[s] = nb | (uint32_t)gid;
                q.nd[s] = node;
            }
    }
    out_pr = __uint_as_float(wb);
    return true;
}

// Nodes displaced from a full queue, kept for later in the same pass.  Dropping such a node
// instead caps the pass at its priority, and when no hit lies between the pass's start and
// that priority the pass composites nothing; the next pass then starts at the cap (the
// forward's progress rule), but a cap at the pass's start itself, from nodes all entered at
// that point, would repeat the pass until the loop guard ends it.  Such frontiers arise on rays
// that start among many overlapping boxes (reflected rays inside the cloud).  The list is
// warp-uniform (every lane holds the same entries); only a full list drops a node.  Its
// entries live in local memory (touched only when the queue is full); its fill n and its best
// priority (smallest for the min-queue, largest for the max-queue, +-inf when empty) are kept
// by the caller in registers.
constexpr int kDeferSlots = 448;
struct WarpDefer {
    int node[kDeferSlots];
    float pr[kDeferSlots];
};

template <bool MAXQ>
__device__ __forceinline__ float wd_none() {
    return MAXQ ? __int_as_float(0xff800000) : __int_as_float(0x7f800000);
}

// keep a displaced node; false when the list is full (the caller drops the node then)
template <bool MAXQ>
__device__ __forceinline__ bool wd_add(WarpDefer& w, int& n, float& best, float pr, int node) {
    if (n >= kDeferSlots) return false;
    w.node[n] = node;
    w.pr[n] = pr;
    ++n;
    best = MAXQ ? fmaxf(best, pr) : fminf(best, pr);
    return true;
}

// move kept nodes back into the (empty) queue, as many as fit; returns the queue's extreme key
template <bool MAXQ>
__device__ __forceinline__ uint32_t wd_refill(const WarpDefer& w, int& n, float& best, WarpQueue& q, int lane) {
    while (n > 0 && wq_push<MAXQ>(q, w.pr[n - 1], w.node[n - 1], lane)) --n;
    best = wd_none<MAXQ>();
    for (int i = 0; i < n; ++i) best = MAXQ ? fmaxf(best, w.pr[i]) : fminf(best, w.pr[i]);
    return wq_extreme_key<MAXQ>(q);
}

// warp-wide min / max of non-negative floats (their bit patterns order as unsigned integers)
__device__ __forceinline__ float warp_min_nonneg(float v) {
    return __uint_as_float(__reduce_min_sync(0xffffffffu, __float_as_uint(v)));
}
__device__ __forceinline__ float warp_max_nonneg(float v) {
    return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(v)));
}

// EPS2: the eps2 estimator's phase 2 (Sec. 3): after the eps1 cut, the ray goes on collecting
// hits in order without compositing them, accumulating the colour S and transmittance T2 seen
// behind its last composited hit until T2 < eps2; (S + T2 background, 1 - T2) is stored per
// pixel for the adjoint.
// The pending-hit buffer of the best-first traversals, two layouts with one interface.  Keys are
// kept ascending (forward) or descending (DESC: the adjoint's back-to-front replay); front() is
// the next key to composite / replay (the empty key when none) and last() the K-th (the empty
// key unless the buffer is full).
//
// RegKbuf: K 64-bit keys in registers, compare-exchange networks sized by the warp's fill.
template <int K, bool DESC = false>
struct RegKbuf {
    static constexpr int64_t kEmpty = DESC ? kEmptyKeyDesc : kEmptyKey;
    int64_t keys[K];
    int nk;  // occupied slots [0, nk)
    __device__ __forceinline__ explicit RegKbuf(int64_t*) {}
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int s = 0; s < K; ++s) keys[s] = kEmpty;
        nk = 0;
    }
    __device__ __forceinline__ int64_t front() const { return keys[0]; }
    __device__ __forceinline__ int64_t last() const { return keys[K - 1]; }
    // insert `key` (before last() in the buffer's order) where `ins`; all 32 lanes call, converged
    __device__ __forceinline__ void insert_warp(bool ins, int64_t key) { kbuf_insert_warp<K, DESC>(keys, nk, ins, key); }
    // drop front() in the calling lanes (converged among themselves)
    __device__ __forceinline__ void pop(unsigned group) { kbuf_pop_warp<K>(keys, nk, kEmpty, group); }
    // drop every key at or beyond `bound` (ascending: >= bound; descending: <= bound)
    __device__ __forceinline__ void drop_from(int64_t bound) {
        nk = 0;
#pragma unroll
        for (int s = 0; s < K; ++s) {
            if (DESC ? keys[s] <= bound : keys[s] >= bound) keys[s] = kEmpty;
            nk += keys[s] != kEmpty;
        }
    }
};

// SmemKbuf: a ring of K slots per lane in shared memory, laid out slot-major within the warp
// (slot s of lane l at col[32 s], col = warp base + l), so the 32 lanes of a warp always hit
// 32 distinct 8-byte words whatever their ring positions: no bank conflicts.  Only the head,
// the fill and copies of front() and last() live in registers, which frees the 64 registers
// of the register buffer for occupancy.  An insert shifts the keys after the new one by one
// slot (insertion order is nearly sorted in best-first order, so shifts are short); a pop
// advances the head.
template <int K, bool DESC = false>
struct SmemKbuf {
    static_assert((K & (K - 1)) == 0, "ring size must be a power of two");
    static constexpr int64_t kEmpty = DESC ? kEmptyKeyDesc : kEmptyKey;
    int64_t* col;
    int head, nk;
    int64_t fr, lst;
    __device__ __forceinline__ explicit SmemKbuf(int64_t* c) : col(c) {}
    __device__ __forceinline__ int64_t& at(int i) const { return col[((head + i) & (K - 1)) * 32]; }
    __device__ __forceinline__ void reset() {
        head = 0;
        nk = 0;
        fr = lst = kEmpty;
    }
    __device__ __forceinline__ int64_t front() const { return fr; }
    __device__ __forceinline__ int64_t last() const { return lst; }
    __device__ __forceinline__ void insert_warp(bool ins, int64_t key) {
        if (!ins) return;
        int i = nk < K ? nk : K - 1;  // a full ring drops its last key
        while (i > 0) {
            const int64_t v = at(i - 1);
            if (DESC ? v > key : v < key) break;
            at(i) = v;
            --i;
        }
        at(i) = key;
        if (nk < K) ++nk;
        if (i == 0) fr = key;
        lst = nk == K ? at(K - 1) : kEmpty;
    }
    __device__ __forceinline__ void pop(unsigned) {
        head = (head + 1) & (K - 1);
        --nk;
        fr = nk > 0 ? at(0) : kEmpty;
        lst = kEmpty;
    }
    __device__ __forceinline__ void drop_from(int64_t bound) {
        const int before = nk;
        while (nk > 0 && (DESC ? at(nk - 1) <= bound : at(nk - 1) >= bound)) --nk;
        if (nk == 0) fr = kEmpty;
        if (nk != before) lst = kEmpty;
    }
};

// One segment of a ray that continues a composite already under way (the scene renderer's
// segments between surfaces): hits with entry in [t0, end) where cap0 = pack_key(end, 0)
// (kEmptyKey: no end), ids recorded as id | tag, depth accumulated only when `depth` is set.
struct SegRange {
    float t0;
    int64_t cap0;
    int tag;
    bool depth;
};

// SEG = false: a camera ray from scratch (T = 1, nothing composited, entries from t_near).
// SEG = true: the segment `seg` continues (C, T, depth, count); overflowing ids are reported.
// SMEMK: the pending hits in a shared-memory ring (SmemKbuf; kb_col = this lane's column of
// its warp's 32 K-slot block) instead of registers.
template <int K, bool COUNT, int W, bool EPS2 = false, bool SEG = false, bool SMEMK = false>
__device__ __forceinline__ void trace_forward_bf(const float4* __restrict__ rec, const float4* __restrict__ sph, const NodeSrc& nodes,
                                                 const TraceParams& P, int64_t pix, bool valid, const float3 o, const float3 d,
                                                 float& C0, float& C1, float& C2, float& T, float& depth,
                                                 int64_t& last_key, int& count, Counters& cnt, int* err,
                                                 const SegRange seg = SegRange{0.f, kEmptyKey, 0, true},
                                                 int64_t* kb_col = nullptr) {
    using KB = std::conditional_t<SMEMK, SmemKbuf<K>, RegKbuf<K>>;
    KB kb(kb_col);
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    const int jb = key_id_bits(P.n_gauss);  // id bits of the ordering keys
    // camera rays (and a scene's first segment) share their origin; otherwise cone.ok is false
    const RayCone cone = warp_ray_cone(o, d);
    const float eps = fmaxf(P.eps1, 1e-30f);
    const float INF = __int_as_float(0x7f800000);
    const float tmin = SEG ? seg.t0 : P.t_near;
    const int64_t cap0 = SEG ? seg.cap0 : kEmptyKey;
    if (!SEG) {
        T = 1.f;
        C0 = C1 = C2 = 0.f;
        depth = 0.f;
        count = 0;
    }
    last_key = -1;
    int64_t lo_key = -1;
    int64_t lp_key = -1;  // last key composited or (phase 2) collected
    bool ph2 = false;
    float S0 = 0.f, S1 = 0.f, S2 = 0.f, T2 = 1.f;
    bool done = !valid;
    int passes = 0;
    while (__any_sync(FULL, !done)) {
        if (++passes > P.max_rounds) {
            if (lane == 0) atomicOr(err, kErrLoopGuard);
            break;
        }
        if (COUNT && !done) cnt.rounds++;
        bool active = !done;
        const int64_t pass_last = EPS2 ? lp_key : last_key;  // last key composited before this pass
        kb.reset();
        int64_t cap = cap0;
        const float tlo = lo_key < 0 ? tmin : key_t(lo_key);
        auto composite_front = [&]() {
            const int64_t key = kb.front();
            const int j = key_j(key, jb);
            Hit hc;  // the same solve as at insertion time: the same bits
            ray_ellipsoid<false>(o, d, __ldg(rec + 4 * j + 0), __ldg(rec + 4 * j + 1), __ldg(rec + 4 * j + 2), P.Q,
                                 tmin, hc);
            const float4 sh = __ldg(rec + 4 * j + 3);
            const float a = response_alpha(sh.x, hc.D2);
            if (EPS2 && ph2) {  // phase 2: collect, do not composite
                const float w2 = __fmul_rn(T2, a);
                S0 = fmaf(w2, sh.y, S0);
                S1 = fmaf(w2, sh.z, S1);
                S2 = fmaf(w2, sh.w, S2);
                T2 = __fmul_rn(T2, __fsub_rn(1.f, a));
                lp_key = key;
                if (T2 < P.eps2) done = true;
                kb.pop(__activemask());
                return;
            }
            const float w = __fmul_rn(T, a);
            C0 = fmaf(w, sh.y, C0);
            C1 = fmaf(w, sh.z, C1);
            C2 = fmaf(w, sh.w, C2);
            if (!SEG || seg.depth) depth = fmaf(w, key_t(key), depth);
            T = __fmul_rn(T, __fsub_rn(1.f, a));
            if (count < P.list_cap) P.ids[pix * P.list_cap + count] = SEG ? (j | seg.tag) : j;  // for the adjoint
            else if (SEG) atomicOr(err, kErrListOverflow);
            ++count;
            last_key = key;
            lp_key = key;
            if (COUNT) cnt.hits++;
            if (EPS2 && T < eps) ph2 = true;
            else if (T < eps || count >= P.k_max) done = true;
            kb.pop(__activemask());
        };
        auto drop_cap = [&](float e) {  // a node with packet entry e was dropped (kept list full)
            if (active) {
                cap = min(cap, pack_key(fmaxf(e, 0.f), 0));
                // pending hits at or beyond the new cap may be preceded by hits of the dropped
                // subtree: give them back (the next pass finds them again)
                kb.drop_from(cap);
            }
        };
        WarpQueue q;
        wq_init<false>(q);
        wq_push<false>(q, -INF, nodes.root, lane);
        WarpDefer wd;
        int wd_n = 0;
        float wd_best = wd_none<false>();
        uint32_t qtop = wq_extreme_key<false>(q);  // the queue's minimum key, kept across steps
        int visits = 0;
        while (true) {
            if (qtop == wq_empty<false>() && wd_n > 0) qtop = wd_refill<false>(wd, wd_n, wd_best, q, lane);
            float e_node;
            int node;
            const bool popped = wq_pop_known<false>(q, qtop, e_node, node, lane);
            // a lane needs the node unless its (conservative) entry lies past its bounds
            bool need = false;
            if (popped && active) {
                const float tcap = key_t(cap);
                const int64_t kK = kb.last();
                const float tK = key_t(kK);
                if (e_node <= tcap) {
                    if (e_node > tK) cap = min(cap, pack_key(fmaxf(e_node, 0.f), 0));
                    else need = true;
                }
            }
            if (__any_sync(FULL, need)) {
                if (++visits > P.max_visits) {
                    if (lane == 0) atomicOr(err, kErrLoopGuard);
                    done = true;
                    break;
                }
                Children<W> ch;
                fetch_children<W, !SMEMK>(nodes, node, ch);
                if (COUNT && need) cnt.nodes++;
                if (COUNT && lane == 0) cnt.wnodes++;
                float e[W], x[W];
                bool h[W];
#pragma unroll
                for (int c = 0; c < W; ++c) {
                    float en;
                    slab_child<W>(ch, c, o, inv, en, x[c]);
                    e[c] = fmaxf(en, tlo);
                    h[c] = false;
                }
                if (need) {
                    const float tcap = key_t(cap);
                    const int64_t kK = kb.last();
                    const float tK = key_t(kK);
#pragma unroll
                    for (int c = 0; c < W; ++c) {
                        h[c] = ch.ref[c] != kEmptyRef && e[c] <= fminf(x[c], tcap);
                        if (h[c] && e[c] > tK) {
                            h[c] = false;
                            cap = min(cap, pack_key(e[c], 0));
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < W; ++c) {
                    const int rr = ch.ref[c];
                    const bool want = h[c] && rr < 0;
                    if (__any_sync(FULL, want)) {
                        const int start = ~rr, num = leaf_count(nodes, ~rr, ch.cnt[c]);
                        // sphere pre-test of the whole leaf, then one full test per Gaussian that
                        // some lane may hit (in order: the same inserts as a sequential scan)
                        const uint32_t mask = cone.ok ? leaf_sphere_mask_cone(sph, start, num, want, o, d, cone)
                                                      : leaf_sphere_mask(sph, start, num, want, o, d);
                        uint32_t todo = __reduce_or_sync(FULL, mask);
                        while (todo) {
                            const int g = __ffs(todo) - 1;
                            todo &= todo - 1;
                            const int qq = start + g;
                            if (COUNT && lane == 0) cnt.wleaf++;
                            bool ins = false;
                            int64_t ikey = 0;
                            if ((mask >> g) & 1u) {
                                const float4 g0 = __ldg(rec + 4 * qq + 0);
                                const float4 g1 = __ldg(rec + 4 * qq + 1);
                                const float4 g2 = __ldg(rec + 4 * qq + 2);
                                Hit hh;
                                ray_ellipsoid<false>(o, d, g0, g1, g2, P.Q, tmin, hh);
                                if (COUNT) cnt.tests++;
                                if (hh.hit) {
                                    const int64_t key = hit_key(hh, P.sort_key, qq, jb);
                                    if (key > lo_key && key < cap) {
                                        const int64_t kK = kb.last();
                                        if (key < kK) {
                                            if (kK != kEmptyKey) cap = kK;
                                            ins = true;
                                            ikey = key;
                                            if (COUNT) cnt.inserted++;
                                        } else {
                                            cap = key;
                                        }
                                    }
                                }
                            }
                            if (SMEMK) kb.insert_warp(ins, ikey);  // per lane: no vote needed
                            else if (__any_sync(FULL, ins)) kb.insert_warp(ins, ikey);
                        }
                    }
                }
                bool in[W];
#pragma unroll
                for (int c = 0; c < W; ++c) in[c] = h[c] && ch.ref[c] >= 0;
                if (need) {
                    const float tcap = key_t(cap);
                    const int64_t kK = kb.last();
                    const float tK = key_t(kK);
#pragma unroll
                    for (int c = 0; c < W; ++c) {
                        if (in[c] && e[c] > tcap) in[c] = false;
                        if (in[c] && e[c] > tK) {
                            in[c] = false;
                            cap = min(cap, pack_key(e[c], 0));
                        }
                    }
                }
                float ev;
                int ednode;
#pragma unroll
                for (int c = 0; c < W; ++c) {
                    if (__any_sync(FULL, in[c])) {
                        const float ep = warp_min_nonneg(in[c] ? e[c] : INF);  // e >= tlo >= 0
                        if (wq_push_displace<false>(q, ep, ch.ref[c], lane, ev, ednode) && !wd_add<false>(wd, wd_n, wd_best, ev, ednode))
                            drop_cap(ev);
                    }
                }
            }
            qtop = wq_extreme_key<false>(q);
            // +inf when nothing is left: composite all pending
            const float bound = fminf(wq_key_priority<false>(qtop), wd_best);
            while (active && !done && key_t(kb.front()) < bound) composite_front();
            active = active && !done;
            if (!popped || !__any_sync(FULL, active)) break;
        }
        if (active && !done) {
            if (cap == cap0) {
                done = true;  // nothing was dropped: every hit before the end is in
            } else {
                const int64_t got = EPS2 ? lp_key : last_key;
                // A pass that composited nothing ended with an empty buffer: no hit after lo_key
                // lies below the cap (explored nodes would have given it, dropped or pruned
                // ones hold none below the cap), so the next pass may start at the cap.
                lo_key = got != pass_last ? got : max(lo_key, cap - 1);
            }
        }
    }
    if (EPS2 && valid)
        P.sS[pix] = ph2 ? make_float4(fmaf(T2, P.bg[0], S0), fmaf(T2, P.bg[1], S1), fmaf(T2, P.bg[2], S2), 1.f - T2)
                        : make_float4(0.f, 0.f, 0.f, -1.f);
}

// SMEMK: the pending hits in a descending shared-memory ring (SmemKbuf; kb_col = this lane's
// column of its warp's 32 K-slot block) instead of registers.
template <int K, bool COUNT, int W, bool DEPTH, bool SMEMK = false>
__device__ __forceinline__ void trace_backward_bf(const float4* __restrict__ rec, const float4* __restrict__ sph, const NodeSrc& nodes,
                                                  const TraceParams& P, const float3 o, const float3 d,
                                                  float T_final, int64_t last_key, int n_hits, const Upstream& g,
                                                  float4* __restrict__ gtmp, Counters& cnt, int* err,
                                                  int64_t* kb_col = nullptr, int64_t* fin_col = nullptr) {
    using KB = std::conditional_t<SMEMK, SmemKbuf<K, true>, RegKbuf<K, true>>;
    KB kb(kb_col);
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    const int jb = key_id_bits(P.n_gauss);  // id bits of the ordering keys
    // camera rays share their origin: the leaf pre-test bounds the warp's rays by a cone
    const RayCone cone = warp_ray_cone(o, d);
    const float NINF = __int_as_float(0xff800000);
    const float INF = __int_as_float(0x7f800000);
    constexpr uint32_t kFloorJ = kKeyLowMax;  // the largest key at a given t
    int64_t hi_key = last_key + 1;
    Adjoint adj = adjoint_start(P, T_final, g);
    int remaining = n_hits > 0 ? n_hits : 0;
    int passes = 0;
    while (__any_sync(FULL, remaining > 0)) {
        if (++passes > P.max_rounds) {
            if (lane == 0) atomicOr(err, kErrLoopGuard);
            break;
        }
        if (COUNT && remaining > 0) cnt.rounds++;
        bool active = remaining > 0;
        kb.reset();
        int64_t floor_key = -1;
        const int64_t pass_hi = hi_key;  // where this pass starts (from the back)
        const float thi = key_t(hi_key);
        bool stop = false;
        // SMEMK: a hit whose key passes the bound is finalised (taken from the ring into a
        // per-lane list of up to kFin keys in shared memory, in replay order); the lists are
        // replayed densely, all lanes at once, when one fills or the pass ends
        constexpr int kFin = 16;
        int nf = 0;
        auto fin_at = [&](int i) -> int64_t& { return fin_col[32 * i]; };
        auto replay_fin = [&]() {
            int i = 0;
            while (__any_sync(0xffffffffu, i < nf)) {
                int jout = -1;
                float4 vout[4];
                if (i < nf) {
                    jout = key_j(fin_at(i), jb);
                    adjoint_hit<DEPTH>(rec, jout, o, d, P, adj, g, vout);
                    if (COUNT) cnt.hits++;
                }
                ++i;
                if (jout >= 0) {
                    float4* gp = gtmp + 4 * jout;
#pragma unroll
                    for (int q = 0; q < 4; ++q) atomicAdd(gp + q, vout[q]);
                }
            }
            nf = 0;
        };
        auto finalize_while = [&](auto cond) {
            while (true) {
                while (nf < kFin && cond()) {
                    const int64_t key = kb.front();
                    fin_at(nf++) = key;
                    --remaining;
                    hi_key = key;
                    kb.pop(0u);
                }
                if (!__any_sync(0xffffffffu, nf == kFin && cond())) break;
                replay_fin();
            }
        };
        auto replay_contrib = [&](int& jout, float4 (&vout)[4]) {
            const int64_t key = kb.front();
            const int j = key_j(key, jb);
            adjoint_hit<DEPTH>(rec, j, o, d, P, adj, g, vout);
            jout = j;
            --remaining;
            hi_key = key;
            if (COUNT) cnt.hits++;
            kb.pop(__activemask());
        };
        // replay while any lane can; each lane issues its own float4 atomics (a warp-aggregated
        // scatter, whose match and shuffles stall while lanes rarely share a Gaussian at one
        // step, measured 28 % slower here, as in the list replay)
        auto replay_while = [&](auto cond) {
            while (true) {
                const bool c = cond();
                if (!__any_sync(0xffffffffu, c)) break;
                int jout = -1;
                float4 vout[4];
                if (c) replay_contrib(jout, vout);
                if (jout >= 0) {
                    float4* gp = gtmp + 4 * jout;
#pragma unroll
                    for (int q = 0; q < 4; ++q) atomicAdd(gp + q, vout[q]);
                }
            }
        };
        auto drop_floor = [&](float x) {  // a node with packet exit x was dropped (kept list full)
            if (active) {
                floor_key = max(floor_key, pack_key(fmaxf(x, 0.f), kFloorJ));
                // pending hits at or below the new floor may be followed by hits of the dropped
                // subtree: give them back (the next pass finds them again)
                kb.drop_from(floor_key);
            }
        };
        WarpQueue q;
        wq_init<true>(q);
        wq_push<true>(q, INF, nodes.root, lane);
        WarpDefer wd;
        int wd_n = 0;
        float wd_best = wd_none<true>();
        uint32_t qtop = wq_extreme_key<true>(q);  // the queue's maximum key, kept across steps
        int visits = 0;
        while (true) {
            if (qtop == wq_empty<true>() && wd_n > 0) qtop = wd_refill<true>(wd, wd_n, wd_best, q, lane);
            float x_node;
            int node;
            const bool popped = wq_pop_known<true>(q, qtop, x_node, node, lane);
            bool need = false;
            if (popped && active) {
                const float tfl = floor_key < 0 ? P.t_near : fmaxf(P.t_near, key_t(floor_key));
                const int64_t kK = kb.last();
                const float tK = key_t(kK);  // -inf when the buffer is not full
                if (x_node >= tfl) {
                    if (x_node < tK) floor_key = max(floor_key, pack_key(fmaxf(x_node, 0.f), kFloorJ));
                    else need = true;
                }
            }
            if (__any_sync(FULL, need)) {
                if (++visits > P.max_visits) {
                    if (lane == 0) atomicOr(err, kErrLoopGuard);
                    stop = true;
                    break;
                }
                Children<W> ch;
                fetch_children<W, !SMEMK>(nodes, node, ch);
                if (COUNT && need) cnt.nodes++;
                if (COUNT && lane == 0) cnt.wnodes++;
                float en[W], x[W];
                bool h[W];
#pragma unroll
                for (int c = 0; c < W; ++c) {
                    slab_child<W>(ch, c, o, inv, en[c], x[c]);
                    h[c] = false;
                }
                if (need) {
                    const float tfl = floor_key < 0 ? P.t_near : fmaxf(P.t_near, key_t(floor_key));
                    const int64_t kK = kb.last();
                    const float tK = key_t(kK);  // -inf when the buffer is not full
#pragma unroll
                    for (int c = 0; c < W; ++c) {
                        h[c] = ch.ref[c] != kEmptyRef && en[c] <= thi && x[c] >= tfl && x[c] >= en[c];
                        if (h[c] && x[c] < tK) {
                            h[c] = false;
                            floor_key = max(floor_key, pack_key(x[c], kFloorJ));
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < W; ++c) {
                    const int rr = ch.ref[c];
                    const bool want = h[c] && rr < 0;
                    if (__any_sync(FULL, want)) {
                        const int start = ~rr, num = leaf_count(nodes, ~rr, ch.cnt[c]);
                        const uint32_t mask = cone.ok ? leaf_sphere_mask_cone(sph, start, num, want, o, d, cone)
                                                      : leaf_sphere_mask(sph, start, num, want, o, d);
                        uint32_t todo = __reduce_or_sync(FULL, mask);
                        while (todo) {
                            const int g = __ffs(todo) - 1;
                            todo &= todo - 1;
                            const int qq = start + g;
                            if (COUNT && lane == 0) cnt.wleaf++;
                            bool ins = false;
                            int64_t ikey = 0;
                            if ((mask >> g) & 1u) {
                                const float4 g0 = __ldg(rec + 4 * qq + 0);
                                const float4 g1 = __ldg(rec + 4 * qq + 1);
                                const float4 g2 = __ldg(rec + 4 * qq + 2);
                                Hit hh;
                                ray_ellipsoid<false>(o, d, g0, g1, g2, P.Q, P.t_near, hh);
                                if (COUNT) cnt.tests++;
                                if (hh.hit) {
                                    const int64_t key = hit_key(hh, P.sort_key, qq, jb);
                                    if (key < hi_key && key > floor_key) {
                                        const int64_t kK = kb.last();
                                        if (key > kK) {
                                            if (kK != kEmptyKeyDesc) floor_key = kK;
                                            ins = true;
                                            ikey = key;
                                            if (COUNT) cnt.inserted++;
                                        } else {
                                            floor_key = key;
                                        }
                                    }
                                }
                            }
                            if (SMEMK) kb.insert_warp(ins, ikey);  // per lane: no vote needed
                            else if (__any_sync(FULL, ins)) kb.insert_warp(ins, ikey);
                        }
                    }
                }
                bool in[W];
#pragma unroll
                for (int c = 0; c < W; ++c) in[c] = h[c] && ch.ref[c] >= 0;
                if (need) {
                    const float tfl = floor_key < 0 ? P.t_near : fmaxf(P.t_near, key_t(floor_key));
                    const int64_t kK = kb.last();
                    const float tK = key_t(kK);  // -inf when the buffer is not full
#pragma unroll
                    for (int c = 0; c < W; ++c) {
                        if (in[c] && x[c] < tfl) in[c] = false;
                        if (in[c] && x[c] < tK) {
                            in[c] = false;
                            floor_key = max(floor_key, pack_key(x[c], kFloorJ));
                        }
                    }
                }
                float ev;
                int ednode;
#pragma unroll
                for (int c = 0; c < W; ++c) {
                    if (__any_sync(FULL, in[c])) {
                        const float xp = warp_max_nonneg(in[c] ? x[c] : 0.f);  // x >= tfl >= 0
                        if (wq_push_displace<true>(q, xp, ch.ref[c], lane, ev, ednode) && !wd_add<true>(wd, wd_n, wd_best, ev, ednode))
                            drop_floor(ev);
                    }
                }
            }
            qtop = wq_extreme_key<true>(q);
            // -inf when nothing is left: replay everything pending
            const float bound = fmaxf(wq_key_priority<true>(qtop), wd_best);
            if constexpr (SMEMK) finalize_while([&] { return active && remaining > 0 && key_t(kb.front()) > bound; });
            else replay_while([&] { return active && remaining > 0 && key_t(kb.front()) > bound; });
            active = active && remaining > 0;
            if (!popped || !__any_sync(FULL, active)) break;
        }
        if constexpr (SMEMK) replay_fin();
        if (__any_sync(FULL, stop)) break;
        if (active && remaining > 0 && floor_key < 0) {
            atomicOr(err, kErrReplayMismatch);
            remaining = 0;
        }
        // a pass that replayed nothing ended with an empty buffer: every remaining hit lies at
        // or below its floor, so the next pass may start there (the forward's progress rule)
        if (active && remaining > 0 && hi_key == pass_hi) hi_key = min(hi_key, floor_key + 1);
    }
}

// ---------------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ bool tile_pixel(const FwdArgs& A, int64_t tile, int lane, DevCam& cam, int& px, int& py,
                                           int64_t& pix) {
    int c = A.cam_single;
    int64_t local = tile;
    if (A.cam_single < 0) {
        c = 0;
        while (c + 1 < A.n_cams && A.cams[c + 1].tile_base <= tile) ++c;
        local = tile - A.cams[c].tile_base;
    }
    cam = A.cams[c];
    const int tx = (int)(local % cam.tiles_x), ty = (int)(local / cam.tiles_x);
    px = tx * A.tile_w + (lane % A.tile_w);
    py = ty * (32 / A.tile_w) + (lane / A.tile_w);
    pix = cam.pix_base + (int64_t)py * cam.W + px;
    return px < cam.W && py < cam.H && ty < cam.tiles_y;
}

}  // namespace rs
