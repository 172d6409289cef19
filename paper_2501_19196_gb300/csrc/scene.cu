// scene.cu -- Gaussians together with a triangle mesh: mirror bounces and diffuse surfaces lit by
// a point light through the Gaussians (the paper's mesh / mirror / shadow scenes, Sec. 1 and
// Fig. 1; the paper gives no algorithm, the rules are stated in include/raysplats.h).
//
// Per ray (one lane each, one warp per tile of 32 pixels):
//   segment loop: nearest triangle (mesh BVH per lane, closest hit, ties to the lower triangle
//     id), then the Gaussians with entry in [t_min, t_tri) composited in (t1, id) order by the
//     warp-packet best-first traversal of the camera rays (trace.cuh), which continues each
//     lane's colour, transmittance and count; a mirror reflects the ray, a diffuse triangle
//     leaves a shadow ray (any-hit over the mesh per lane, then the product of (1 - alpha)
//     over the Gaussians it crosses, the warp's shadow rays traced as one packet).
//   Triangle hits, reflections and shadow rays follow fixed FP32 sequences (explicit
//   round-to-nearest intrinsics, no contraction), the same the oracle writes out.
// The adjoint replays the composited hits back to front across the segments from a per-ray
// id list (segment in the top two bits), starting from the environment term, then adds the
// shadow rays' d(prod(1 - alpha)) terms.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "rs_host.h"
#include "trace.cuh"

namespace rs {
namespace {

constexpr int kMeshStack = 64;
constexpr int kSceneK = 32;

struct MeshDev {
    const float4* nodes;  // 2 per node: (lo.xyz, left | first), (hi.xyz, right | -count)
    const float4* tris;   // 3 per triangle in leaf order: v0 (w = id), v1 (w = material), v2
    const float4* albedo; // per triangle id
    int n_nodes;
    int n_tri;
};

struct SceneArgs {
    FwdArgs F;            // Gaussians, cameras, tiles, params, outputs (rgb, alpha, depth)
    MeshDev mesh;
    float3 light;
    int max_bounces;
    float eps_off;
    int list_cap;         // composited ids per ray
    int shadow_cap;       // shadow ids per ray
    // per-ray state for the adjoint
    float* sT;
    int* sn;              // composited hits
    int* ssn;             // shadow hits (-1: no shadow ray)
    float4* sE;           // environment term (xyz)
    float4* seg;          // 2 per segment and ray: origin (w = t_min), direction
    float4* shadow;       // 3 per ray: point (w = distance), direction (w = T_s), albedo
    int* ids;             // list_cap per ray: id | segment << 30
    int* sids;            // shadow_cap per ray
};

// ----------------------------------------------------------------------------------------
// FP32 sequences shared (as definitions) with the oracle
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ float dot3_rn(const float a[3], const float b[3]) {
    return __fadd_rn(__fadd_rn(__fmul_rn(a[0], b[0]), __fmul_rn(a[1], b[1])), __fmul_rn(a[2], b[2]));
}

__device__ __forceinline__ void cross_rn(const float a[3], const float b[3], float c[3]) {
    c[0] = __fsub_rn(__fmul_rn(a[1], b[2]), __fmul_rn(a[2], b[1]));
    c[1] = __fsub_rn(__fmul_rn(a[2], b[0]), __fmul_rn(a[0], b[2]));
    c[2] = __fsub_rn(__fmul_rn(a[0], b[1]), __fmul_rn(a[1], b[0]));
}

// Moller-Trumbore; true and t when tmin < t < tmax
__device__ __forceinline__ bool tri_hit(const float o[3], const float d[3], const float v0[3], const float v1[3],
                                        const float v2[3], float tmin, float tmax, float& t) {
    const float e1[3] = {__fsub_rn(v1[0], v0[0]), __fsub_rn(v1[1], v0[1]), __fsub_rn(v1[2], v0[2])};
    const float e2[3] = {__fsub_rn(v2[0], v0[0]), __fsub_rn(v2[1], v0[1]), __fsub_rn(v2[2], v0[2])};
    float p[3];
    cross_rn(d, e2, p);
    const float det = dot3_rn(e1, p);
    if (fabsf(det) < 1e-12f) return false;
    const float inv = __fdiv_rn(1.0f, det);
    const float s[3] = {__fsub_rn(o[0], v0[0]), __fsub_rn(o[1], v0[1]), __fsub_rn(o[2], v0[2])};
    const float u = __fmul_rn(dot3_rn(s, p), inv);
    if (u < 0.0f || u > 1.0f) return false;
    float q[3];
    cross_rn(s, e1, q);
    const float w = __fmul_rn(dot3_rn(d, q), inv);
    if (w < 0.0f || __fadd_rn(u, w) > 1.0f) return false;
    t = __fmul_rn(dot3_rn(e2, q), inv);
    return t > tmin && t < tmax;
}

__device__ __forceinline__ void load_tri(const MeshDev& M, int k, float v0[3], float v1[3], float v2[3], int& id,
                                         int& mat) {
    const float4 a = __ldg(M.tris + 3 * k), b = __ldg(M.tris + 3 * k + 1), c = __ldg(M.tris + 3 * k + 2);
    v0[0] = a.x; v0[1] = a.y; v0[2] = a.z;
    v1[0] = b.x; v1[1] = b.y; v1[2] = b.z;
    v2[0] = c.x; v2[1] = c.y; v2[2] = c.z;
    id = __float_as_int(a.w);
    mat = __float_as_int(b.w);
}

__device__ __forceinline__ bool box_hit(const float4 lo, const float4 hi, const float3 o, const float3 inv, float tmin,
                                        float tmax, float& entry) {
    const float tx0 = (lo.x - o.x) * inv.x, tx1 = (hi.x - o.x) * inv.x;
    const float ty0 = (lo.y - o.y) * inv.y, ty1 = (hi.y - o.y) * inv.y;
    const float tz0 = (lo.z - o.z) * inv.z, tz1 = (hi.z - o.z) * inv.z;
    const float en = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), tmin));
    const float ex = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
    entry = en;
    // widened by 1e-6 relative so that rounding never drops a triangle the exact box holds
    return en <= ex + 1e-6f * fmaxf(1.f, fabsf(ex));
}

// nearest triangle in (tmin, tmax): returns its position in leaf order (-1: none), t and id
// (ties in t go to the lower id); any_hit: stop at the first hit
template <bool ANY>
__device__ int mesh_trace(const MeshDev& M, const float o[3], const float d[3], float tmin, float tmax, float& t_best,
                          int& id_best, int& mat_best, int* err) {
    if (M.n_nodes == 0) return -1;
    const float3 of = make_float3(o[0], o[1], o[2]);
    const float3 inv = make_float3(1.f / (fabsf(d[0]) > 1e-30f ? d[0] : copysignf(1e-30f, d[0])),
                                   1.f / (fabsf(d[1]) > 1e-30f ? d[1] : copysignf(1e-30f, d[1])),
                                   1.f / (fabsf(d[2]) > 1e-30f ? d[2] : copysignf(1e-30f, d[2])));
    int stack[kMeshStack];
    int sp = 0, node = 0, best = -1;
    t_best = tmax;
    id_best = 0x7fffffff;
    mat_best = 0;
    int guard = 0;
    while (true) {
        if (++guard > 4 * M.n_nodes + 16) {
            atomicOr(err, kErrLoopGuard);
            break;
        }
        const float4 a = __ldg(M.nodes + 2 * node), b = __ldg(M.nodes + 2 * node + 1);
        float en;
        const bool hit = box_hit(a, b, of, inv, tmin, t_best, en);
        if (hit) {
            const int right = __float_as_int(b.w), left = __float_as_int(a.w);
            if (right < 0) {  // leaf: triangles [left, left - right)
                for (int k = max(left, 0); k < left - right && k < M.n_tri; ++k) {
                    float v0[3], v1[3], v2[3], t;
                    int id, mat;
                    load_tri(M, k, v0, v1, v2, id, mat);
                    // accept t < best, or t == best with a lower id (within the caller's tmax)
                    if (tri_hit(o, d, v0, v1, v2, tmin, tmax, t) && (t < t_best || (t == t_best && id < id_best))) {
                        t_best = t;
                        id_best = id;
                        mat_best = mat;
                        best = k;
                        if (ANY) return best;
                    }
                }
            } else if (left >= 0 && left < M.n_nodes && right < M.n_nodes) {
                if (sp < kMeshStack) stack[sp++] = right;
                else atomicOr(err, kErrStack);
                node = left;
                continue;
            } else {
                atomicOr(err, kErrIndex);
            }
        }
        if (sp == 0) break;
        node = stack[--sp];
    }
    return best;
}

__device__ __forceinline__ void reflect_ray(const float o[3], const float d[3], float t, const float v0[3],
                                            const float v1[3], const float v2[3], float P[3], float dr[3]) {
    const float e1[3] = {__fsub_rn(v1[0], v0[0]), __fsub_rn(v1[1], v0[1]), __fsub_rn(v1[2], v0[2])};
    const float e2[3] = {__fsub_rn(v2[0], v0[0]), __fsub_rn(v2[1], v0[1]), __fsub_rn(v2[2], v0[2])};
    float n[3];
    cross_rn(e1, e2, n);
    const float nl = __fsqrt_rn(dot3_rn(n, n));
    for (int k = 0; k < 3; ++k) n[k] = __fdiv_rn(n[k], nl);
    const float dn = dot3_rn(d, n);
    const float k2 = __fmul_rn(2.0f, dn);
    float r[3];
    for (int k = 0; k < 3; ++k) {
        P[k] = __fadd_rn(o[k], __fmul_rn(t, d[k]));
        r[k] = __fsub_rn(d[k], __fmul_rn(k2, n[k]));
    }
    const float rl = __fsqrt_rn(dot3_rn(r, r));
    for (int k = 0; k < 3; ++k) dr[k] = __fdiv_rn(r[k], rl);
}

__device__ __forceinline__ void hit_point(const float o[3], const float d[3], float t, float P[3]) {
    for (int k = 0; k < 3; ++k) P[k] = __fadd_rn(o[k], __fmul_rn(t, d[k]));
}

__device__ __forceinline__ void shadow_ray(const float P[3], const float3 L, float dir[3], float& dist) {
    const float w[3] = {__fsub_rn(L.x, P[0]), __fsub_rn(L.y, P[1]), __fsub_rn(L.z, P[2])};
    dist = __fsqrt_rn(dot3_rn(w, w));
    for (int k = 0; k < 3; ++k) dir[k] = __fdiv_rn(w[k], dist);
}

// ----------------------------------------------------------------------------------------
// Shadow rays, one per lane that has one (`want`), traced as a warp packet: the warp walks the
// union of the boxes its rays cross (depth first, one node fetch for all lanes) and each lane
// multiplies (1 - alpha) over the Gaussians with entry in [tmin, tmax) on its own ray, ids
// recorded for the adjoint.  The product only decreases, so the order of the factors cannot
// change the eps1 decision: a lane whose product falls below eps1 gets 0 (and no ids) and
// leaves the packet.
// ----------------------------------------------------------------------------------------
__device__ float shadow_transmittance_warp(const SceneArgs& S, const NodeSrc& nodes, int64_t pix, bool want,
                                           const float3 o, const float3 d, float tmin, float tmax, int& n_out) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const TraceParams& P = S.F.P;
    const float4* __restrict__ rec = S.F.rec;
    const float4* __restrict__ sph = S.F.sph;
    const float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    const float eps = fmaxf(P.eps1, 1e-30f);
    float Ts = 1.f;
    int n = 0;
    bool act = want;
    int st[kStackSize];  // the same on every lane
    int sp = 0, node = nodes.root, visits = 0;
    while (__any_sync(FULL, act)) {
        if (++visits > P.max_visits) {
            if (lane == 0) atomicOr(S.F.err, kErrLoopGuard);
            break;
        }
        float4 n0, n1, n2, n3;
        fetch_node(nodes, node, n0, n1, n2, n3);
        float en0, ex0, en1, ex1;
        slab2(n0, n1, n2, o, inv, en0, ex0, en1, ex1);
        const int r0 = __float_as_int(n3.x), r1 = __float_as_int(n3.y);
        const int c0 = __float_as_int(n3.z), c1 = __float_as_int(n3.w);
        const bool h0 = act && fmaxf(en0, tmin) <= fminf(ex0, tmax);
        const bool h1 = act && fmaxf(en1, tmin) <= fminf(ex1, tmax);
        int next = -1;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const bool hs = side ? h1 : h0;
            const int rr = side ? r1 : r0;
            if (!__any_sync(FULL, hs)) continue;
            if (rr < 0) {
                const int start = ~rr, num = leaf_count(nodes, ~rr, side ? c1 : c0);
                const uint32_t mask = leaf_sphere_mask(sph, start, num, hs, o, d);
                uint32_t todo = __reduce_or_sync(FULL, mask);
                while (todo) {
                    const int g = __ffs(todo) - 1;
                    todo &= todo - 1;
                    if (!act || !((mask >> g) & 1u)) continue;
                    const int q = start + g;
                    Hit h;
                    ray_ellipsoid<false>(o, d, __ldg(rec + 4 * q + 0), __ldg(rec + 4 * q + 1), __ldg(rec + 4 * q + 2),
                                         P.Q, tmin, h);
                    if (!h.hit || !(h.t1 < tmax)) continue;
                    Ts = __fmul_rn(Ts, __fsub_rn(1.f, response_alpha(__ldg(rec + 4 * q + 3).x, h.D2)));
                    if (Ts < eps) {
                        act = false;
                        Ts = 0.f;
                        n = 0;
                        continue;
                    }
                    if (n < S.shadow_cap) S.sids[pix * S.shadow_cap + n] = q;
                    else atomicOr(S.F.err, kErrListOverflow);
                    ++n;
                }
            } else if (next < 0) {
                next = rr;
            } else if (sp < kStackSize) {
                st[sp++] = rr;
            } else if (lane == 0) {
                atomicOr(S.F.err, kErrStack);
            }
        }
        if (next < 0) {
            if (sp == 0) break;
            next = st[--sp];
        }
        node = next;
    }
    n_out = n;
    return Ts;
}

// One warp per tile of 32 pixels.  Segment by segment (the segment index is the same on every
// lane): each lane that still has a segment finds its nearest triangle, then the warp
// composites the Gaussians before the triangles as one best-first packet, continuing each
// ray's colour, transmittance and count; a mirror reflects the lane's ray into the next
// segment, a diffuse triangle leaves a shadow ray, traced by the whole warp at the end.  The
// segments' pending hits sit in shared-memory rings (SmemKbuf, one K-slot block per warp), so
// top nodes are not staged.
__global__ void __launch_bounds__(128, 4) k_render_scene(SceneArgs S) {
    extern __shared__ float4 s_top[];  // the warps' k-buffer rings
    const FwdArgs& A = S.F;
    const NodeSrc ns{A.nodes, s_top, 0, A.wide, A.P.n_nodes, A.n_top, A.P.n_gauss, A.err};
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int64_t* kb_col = reinterpret_cast<int64_t*>(s_top) + (threadIdx.x >> 5) * (kSceneK * 32) + lane;
    const int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (tile >= A.total_tiles) return;  // the whole warp
    DevCam cam;
    int px, py;
    int64_t pix;
    const bool valid = tile_pixel(A, tile, lane, cam, px, py, pix);
    float3 o3, d3;
    camera_ray(cam, px, py, o3, d3);
    const float INF = __int_as_float(0x7f800000);
    const float eps = fmaxf(A.P.eps1, 1e-30f);
    float o[3] = {o3.x, o3.y, o3.z}, d[3] = {d3.x, d3.y, d3.z};
    float tmin = A.P.t_near;
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f, depth = 0.f;
    int count = 0, nsh = -1;
    float E[3] = {0.f, 0.f, 0.f};
    bool alive = valid;  // the lane has a segment to trace
    bool lit = false;    // the lane ended on a diffuse triangle: its shadow ray is pending
    float Pp[3] = {0.f, 0.f, 0.f}, dir[3] = {0.f, 0.f, 1.f}, dist = 0.f;
    float4 al = make_float4(0.f, 0.f, 0.f, 0.f);
    Counters cnt;
    int64_t last_key;
    for (int seg = 0; seg <= S.max_bounces && __any_sync(FULL, alive); ++seg) {
        float t_tri = INF;
        int tri = -1, id = 0, mat = 0;
        if (alive) {
            S.seg[(pix * 3 + seg) * 2] = make_float4(o[0], o[1], o[2], tmin);
            S.seg[(pix * 3 + seg) * 2 + 1] = make_float4(d[0], d[1], d[2], 0.f);
            tri = mesh_trace<false>(S.mesh, o, d, tmin, INF, t_tri, id, mat, A.err);
        }
        const SegRange R{tmin, (alive && tri >= 0) ? pack_key(t_tri, 0) : kEmptyKey, (int)((unsigned)seg << 30),
                         seg == 0};
        trace_forward_bf<kSceneK, false, 2, false, true, true>(A.rec, A.sph, ns, A.P, pix, alive,
                                                               make_float3(o[0], o[1], o[2]), make_float3(d[0], d[1], d[2]),
                                                               C0, C1, C2, T, depth, last_key, count, cnt, A.err, R, kb_col);
        if (!alive) continue;
        const bool cut = T < eps || count >= A.P.k_max;
        if (tri < 0) {
            E[0] = A.P.bg[0];
            E[1] = A.P.bg[1];
            E[2] = A.P.bg[2];
            alive = false;
            continue;
        }
        float v0[3], v1[3], v2[3];
        int id2, mat2;
        load_tri(S.mesh, tri, v0, v1, v2, id2, mat2);
        if (mat == 1) {
            hit_point(o, d, t_tri, Pp);
            shadow_ray(Pp, S.light, dir, dist);
            al = __ldg(S.mesh.albedo + id);
            lit = true;
            alive = false;
            continue;
        }
        if (cut || seg == S.max_bounces) {  // mirror: nothing beyond the last bounce
            alive = false;
            continue;
        }
        float Pn[3], dn[3];
        reflect_ray(o, d, t_tri, v0, v1, v2, Pn, dn);
        for (int k = 0; k < 3; ++k) {
            o[k] = Pn[k];
            d[k] = dn[k];
        }
        tmin = S.eps_off;
    }
    // shadow rays: the mesh blocks per lane (any hit), the Gaussians as one warp packet
    bool want = false;
    if (lit) {
        float t_occ;
        int oid, omat;
        want = mesh_trace<true>(S.mesh, Pp, dir, S.eps_off, dist, t_occ, oid, omat, A.err) < 0;
        nsh = 0;
    }
    int nw = 0;
    const float Tw = shadow_transmittance_warp(S, ns, pix, want, make_float3(Pp[0], Pp[1], Pp[2]),
                                               make_float3(dir[0], dir[1], dir[2]), S.eps_off, dist, nw);
    if (!valid) return;
    if (lit) {
        const float Ts = want ? Tw : 0.f;
        if (want) nsh = nw;
        E[0] = __fmul_rn(al.x, Ts);
        E[1] = __fmul_rn(al.y, Ts);
        E[2] = __fmul_rn(al.z, Ts);
        S.shadow[pix * 3] = make_float4(Pp[0], Pp[1], Pp[2], dist);
        S.shadow[pix * 3 + 1] = make_float4(dir[0], dir[1], dir[2], Ts);
        S.shadow[pix * 3 + 2] = al;
    }
    A.rgb[3 * pix + 0] = fmaf(T, E[0], C0);
    A.rgb[3 * pix + 1] = fmaf(T, E[1], C1);
    A.rgb[3 * pix + 2] = fmaf(T, E[2], C2);
    A.alpha[pix] = 1.f - T;
    if (A.depth) A.depth[pix] = depth;
    S.sT[pix] = T;
    S.sn[pix] = count;
    S.ssn[pix] = nsh;
    S.sE[pix] = make_float4(E[0], E[1], E[2], 0.f);
}

// dL/dalpha of Gaussian j on the ray (o, d) -> the 16-float accumulator (App. A.6 chain)
__device__ __forceinline__ void alpha_to_params(const float4* __restrict__ rec, int j, const float3 o, const float3 d,
                                                const TraceParams& P, float tmin, float dLda, float4* __restrict__ gtmp,
                                                BulkScatter& sc) {
    const float4 g0 = __ldg(rec + 4 * j + 0), g1 = __ldg(rec + 4 * j + 1), g2 = __ldg(rec + 4 * j + 2);
    const float4 sh = __ldg(rec + 4 * j + 3);
    Hit h;
    ray_ellipsoid<false>(o, d, g0, g1, g2, P.Q, tmin, h);
    closest_point_accurate(o, d, g0, g1, g2, h.tm, h.p, h.v);
    const float e = expf(__fmul_rn(-0.5f, h.D2));
    const float a = __fmul_rn(sh.x, e);
    const float gD2 = -0.5f * a * dLda;
    const float q0 = 2.f * gD2 * h.p[0], q1 = 2.f * gD2 * h.p[1], q2 = 2.f * gD2 * h.p[2];
    const float4 v[4] = {make_float4(q0 * h.v[0], q0 * h.v[1], q0 * h.v[2], -(g0.x * q0 + g1.x * q1 + g2.x * q2)),
                         make_float4(q1 * h.v[0], q1 * h.v[1], q1 * h.v[2], -(g0.y * q0 + g1.y * q1 + g2.y * q2)),
                         make_float4(q2 * h.v[0], q2 * h.v[1], q2 * h.v[2], -(g0.z * q0 + g1.z * q1 + g2.z * q2)),
                         make_float4(dLda * e, 0.f, 0.f, 0.f)};
    sc.add(gtmp + 4 * j, v);
}

// Dynamic shared memory: the threads' gradient staging slots (BulkScatter, as the list replay).
template <bool DEPTH>
__global__ void __launch_bounds__(128) k_scene_bwd(SceneArgs S, BwdArgs B) {
    extern __shared__ float4 s_stage[];
    BulkScatter sc(s_stage + BulkScatter::kFloat4 * threadIdx.x);
    const FwdArgs& A = S.F;
    const int lane = threadIdx.x & 31;
    const int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (tile >= A.total_tiles) return;
    DevCam cam;
    int px, py;
    int64_t pix;
    if (!tile_pixel(A, tile, lane, cam, px, py, pix)) return;
    Upstream g{{B.d_rgb[3 * pix], B.d_rgb[3 * pix + 1], B.d_rgb[3 * pix + 2]},
               B.d_alpha ? B.d_alpha[pix] : 0.f,
               DEPTH ? B.d_depth[pix] : 0.f,
               {0.f, 0.f, 0.f, -1.f}};
    const float Tf = S.sT[pix];
    const int n = min(S.sn[pix], S.list_cap);
    const float4 E = S.sE[pix];
    Adjoint s{Tf, E.x, E.y, E.z, 0.f, 0.f, 0.f, 0.f, 0.f, -1.f};
    for (int k = n - 1; k >= 0; --k) {
        const int e = S.ids[pix * S.list_cap + k];
        const int j = e & 0x3fffffff, seg = (int)((unsigned)e >> 30);
        if (j >= A.P.n_gauss || seg > 2) {
            atomicOr(A.err, kErrIndex);
            break;
        }
        const float4 so = S.seg[(pix * 3 + seg) * 2], sd = S.seg[(pix * 3 + seg) * 2 + 1];
        const float3 o = make_float3(so.x, so.y, so.z), d = make_float3(sd.x, sd.y, sd.z);
        float4 v[4];
        if (DEPTH && seg == 0) adjoint_hit<true>(A.rec, j, o, d, A.P, s, g, v);
        else adjoint_hit<false>(A.rec, j, o, d, A.P, s, g, v);
        sc.add(B.gtmp + 4 * j, v);
    }
    const int nsh = S.ssn[pix];
    if (nsh > 0) {
        const float4 Pp = S.shadow[pix * 3], dir = S.shadow[pix * 3 + 1], al = S.shadow[pix * 3 + 2];
        const float Ts = dir.w;
        const float ga = (g.c[0] * al.x + g.c[1] * al.y + g.c[2] * al.z) * Tf;
        const float3 o = make_float3(Pp.x, Pp.y, Pp.z), d = make_float3(dir.x, dir.y, dir.z);
        const int m = min(nsh, S.shadow_cap);
        for (int k = 0; k < m; ++k) {
            const int j = S.sids[pix * S.shadow_cap + k];
            if (j < 0 || j >= A.P.n_gauss) {
                atomicOr(A.err, kErrIndex);
                break;
            }
            Hit h;
            ray_ellipsoid<false>(o, d, __ldg(A.rec + 4 * j + 0), __ldg(A.rec + 4 * j + 1), __ldg(A.rec + 4 * j + 2),
                                 A.P.Q, S.eps_off, h);
            const float a = response_alpha(__ldg(A.rec + 4 * j + 3).x, h.D2);
            // d(T_f a T_s)/dalpha_j = -T_f a T_s / (1 - alpha_j)  (1 - alpha_j >= 1e-4)
            alpha_to_params(A.rec, j, o, d, A.P, S.eps_off, -ga * Ts / (1.f - a), B.gtmp, sc);
        }
    }
    sc.drain();
}

}  // namespace
}  // namespace rs

using namespace rs;

// ------------------------------------------------------------------------------------------
// host: mesh BVH (built once; median split on the longest centroid axis, leaves of <= 4)
// ------------------------------------------------------------------------------------------
struct rs_mesh {
    int device = 0;
    float4* nodes = nullptr;
    float4* tris = nullptr;
    float4* albedo = nullptr;
    int n_nodes = 0, n_tri = 0;
};

struct rs_scene_state {
    int device = 0;
    int64_t cap_pix = 0;
    int cap_cams = 0;
    DevCam* cams = nullptr;
    float* sT = nullptr;
    int* sn = nullptr;
    int* ssn = nullptr;
    float4* sE = nullptr;
    float4* seg = nullptr;
    float4* shadow = nullptr;
    int* ids = nullptr;
    int* sids = nullptr;
    float4* gtmp = nullptr;
    int64_t cap_gauss = 0;
    int list_cap = 0, shadow_cap = 0;
    // what the forward recorded
    SceneArgs args{};
    const rs_accel* accel = nullptr;
    const rs_mesh* mesh = nullptr;
    int64_t n_gauss = 0;
    bool valid = false;
    std::vector<DevCam> table;
};

namespace {

float bits_as_float(int v) {
    float f;
    memcpy(&f, &v, sizeof(f));
    return f;
}

struct BuildTri {
    float lo[3], hi[3], c[3];
    int id;
};

int build_node(std::vector<BuildTri>& T, int first, int count, std::vector<float4>& nodes) {
    const int me = (int)nodes.size() / 2;
    nodes.push_back(make_float4(0, 0, 0, 0));
    nodes.push_back(make_float4(0, 0, 0, 0));
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = first; i < first + count; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], T[i].lo[k]);
            hi[k] = std::max(hi[k], T[i].hi[k]);
            clo[k] = std::min(clo[k], T[i].c[k]);
            chi[k] = std::max(chi[k], T[i].c[k]);
        }
    int left, right;
    if (count <= 4) {
        left = first;
        right = -count;
    } else {
        int ax = 0;
        for (int k = 1; k < 3; ++k)
            if (chi[k] - clo[k] > chi[ax] - clo[ax]) ax = k;
        const int mid = first + count / 2;
        std::nth_element(T.begin() + first, T.begin() + mid, T.begin() + first + count,
                         [ax](const BuildTri& a, const BuildTri& b) { return a.c[ax] < b.c[ax] || (a.c[ax] == b.c[ax] && a.id < b.id); });
        left = build_node(T, first, mid - first, nodes);
        right = build_node(T, mid, first + count - mid, nodes);
    }
    nodes[2 * me] = make_float4(lo[0], lo[1], lo[2], bits_as_float(left));
    nodes[2 * me + 1] = make_float4(hi[0], hi[1], hi[2], bits_as_float(right));
    return me;
}

}  // namespace

extern "C" {

rs_status rs_build_mesh(const rs_mesh_desc* desc, rs_mesh** out) {
    if (!desc || !out) return set_error(RS_ERR_INVALID_ARG, "mesh: NULL argument");
    if (desc->n_tri < 0 || desc->n_tri > (1 << 26) || (desc->n_tri > 0 && (!desc->verts || !desc->material || !desc->albedo)))
        return set_error(RS_ERR_INVALID_ARG, "mesh: bad triangle arrays");
    const int n = (int)desc->n_tri;
    std::vector<BuildTri> T((size_t)n);
    for (int i = 0; i < n; ++i) {
        const float* v = desc->verts + 9 * i;
        for (int k = 0; k < 3; ++k) {
            if (!std::isfinite(v[k]) || !std::isfinite(v[3 + k]) || !std::isfinite(v[6 + k]))
                return set_error(RS_ERR_INVALID_ARG, "mesh: triangle %d is not finite", i);
            T[i].lo[k] = std::min(v[k], std::min(v[3 + k], v[6 + k]));
            T[i].hi[k] = std::max(v[k], std::max(v[3 + k], v[6 + k]));
            T[i].c[k] = (v[k] + v[3 + k] + v[6 + k]) / 3.f;
        }
        T[i].id = i;
        if (desc->material[i] != 0 && desc->material[i] != 1)
            return set_error(RS_ERR_INVALID_ARG, "mesh: material of triangle %d must be 0 or 1", i);
    }
    std::vector<float4> nodes;
    if (n > 0) build_node(T, 0, n, nodes);
    std::vector<float4> tris((size_t)3 * n), alb((size_t)std::max(n, 1));
    for (int k = 0; k < n; ++k) {
        const int id = T[k].id;
        const float* v = desc->verts + 9 * id;
        tris[3 * k] = make_float4(v[0], v[1], v[2], bits_as_float(id));
        tris[3 * k + 1] = make_float4(v[3], v[4], v[5], bits_as_float(desc->material[id]));
        tris[3 * k + 2] = make_float4(v[6], v[7], v[8], 0.f);
    }
    for (int i = 0; i < n; ++i)
        alb[i] = make_float4(desc->albedo[3 * i], desc->albedo[3 * i + 1], desc->albedo[3 * i + 2], 0.f);
    rs_mesh* M = new (std::nothrow) rs_mesh();
    if (!M) return set_error(RS_ERR_OOM, "host allocation failed");
    cudaGetDevice(&M->device);
    void *pn = nullptr, *pt = nullptr, *pa = nullptr;
    rs_status st;
    if ((st = device_realloc(&pn, sizeof(float4) * std::max<size_t>(nodes.size(), 2))) ||
        (st = device_realloc(&pt, sizeof(float4) * std::max<size_t>(tris.size(), 3))) ||
        (st = device_realloc(&pa, sizeof(float4) * alb.size()))) {
        if (pn) cudaFree(pn);
        if (pt) cudaFree(pt);
        if (pa) cudaFree(pa);
        delete M;
        return st;
    }
    M->nodes = static_cast<float4*>(pn);
    M->tris = static_cast<float4*>(pt);
    M->albedo = static_cast<float4*>(pa);
    M->n_nodes = (int)nodes.size() / 2;
    M->n_tri = n;
    if (n > 0) {
        cudaMemcpy(M->nodes, nodes.data(), sizeof(float4) * nodes.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(M->tris, tris.data(), sizeof(float4) * tris.size(), cudaMemcpyHostToDevice);
    }
    cudaMemcpy(M->albedo, alb.data(), sizeof(float4) * alb.size(), cudaMemcpyHostToDevice);
    *out = M;
    return cuda_check("rs_build_mesh");
}

rs_status rs_mesh_destroy(rs_mesh* M) {
    if (!M) return RS_OK;
    cudaDeviceSynchronize();
    cudaFree(M->nodes);
    cudaFree(M->tris);
    cudaFree(M->albedo);
    delete M;
    return cuda_check("rs_mesh_destroy");
}

rs_status rs_render_scene(const rs_gaussians* g, const rs_accel* accel, const rs_mesh* mesh,
                          const rs_scene_params* sp, const rs_camera* cams, int32_t n_cams,
                          const rs_render_params* p, const rs_tune_params* tune, rs_frame* out,
                          rs_scene_state** inout, void* cuda_stream) {
    if (!g || !accel || !mesh || !sp || !cams || n_cams < 1 || !p || !tune || !out || !out->rgb || !out->alpha || !inout)
        return set_error(RS_ERR_INVALID_ARG, "scene render: NULL or empty argument");
    if (accel->n != g->n || g->n < 1) return set_error(RS_ERR_INVALID_ARG, "scene render: accel built for another n");
    if (!(p->Q > 0.f) || !(p->Q <= accel->Q_box) || !(p->eps1 >= 0.f) || !(p->t_near >= 0.f) || p->k_max < 1)
        return set_error(RS_ERR_INVALID_ARG, "scene render: bad render parameters");
    if (p->sort_key != 0 || p->depth_mode != 0 || p->grad_mode != 0)
        return set_error(RS_ERR_UNSUPPORTED, "scene render: sort_key, depth_mode and grad_mode must be 0");
    if (sp->max_bounces < 0 || sp->max_bounces > 2 || !(sp->eps_off > 0.f) || !std::isfinite(sp->eps_off))
        return set_error(RS_ERR_INVALID_ARG, "scene render: max_bounces must be 0..2 and eps_off > 0");
    if (sp->list_cap < 1 || sp->list_cap > 4096 || sp->shadow_cap < 1 || sp->shadow_cap > 4096)
        return set_error(RS_ERR_INVALID_ARG, "scene render: list capacities must be 1..4096");
    if (tune->tile_w < 1 || tune->tile_w > 32 || (32 % tune->tile_w) != 0 || tune->tile_h != 32 / tune->tile_w)
        return set_error(RS_ERR_INVALID_ARG, "scene render: tile_w * tile_h must be 32");
    std::vector<DevCam> table((size_t)n_cams);
    int64_t tiles = 0, pix = 0;
    for (int c = 0; c < n_cams; ++c) {
        const rs_camera& C = cams[c];
        if (C.width < 1 || C.height < 1 || C.fx == 0.f || C.fy == 0.f)
            return set_error(RS_ERR_INVALID_ARG, "scene render: camera %d has a bad size or focal length", c);
        DevCam& D = table[(size_t)c];
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
    cudaStream_t s = (cudaStream_t)cuda_stream;
    rs_scene_state* S = *inout;
    if (!S) {
        S = new (std::nothrow) rs_scene_state();
        if (!S) return set_error(RS_ERR_OOM, "host allocation failed");
        cudaGetDevice(&S->device);
        *inout = S;
    }
    S->valid = false;
    rs_status st;
    auto grow = [&](auto*& ptr, int64_t count) -> rs_status {
        void* q = ptr;
        const rs_status r = device_realloc(&q, sizeof(*ptr) * (size_t)std::max<int64_t>(count, 1));
        ptr = static_cast<std::remove_reference_t<decltype(ptr)>>(q);
        return r;
    };
    if (pix > S->cap_pix || sp->list_cap != S->list_cap || sp->shadow_cap != S->shadow_cap) {
        S->cap_pix = 0;
        if ((st = grow(S->sT, pix)) || (st = grow(S->sn, pix)) || (st = grow(S->ssn, pix)) || (st = grow(S->sE, pix)) ||
            (st = grow(S->seg, pix * 6)) || (st = grow(S->shadow, pix * 3)) || (st = grow(S->ids, pix * sp->list_cap)) ||
            (st = grow(S->sids, pix * sp->shadow_cap)))
            return st;
        S->cap_pix = pix;
        S->list_cap = sp->list_cap;
        S->shadow_cap = sp->shadow_cap;
    }
    if (n_cams > S->cap_cams) {
        S->cap_cams = 0;
        if ((st = grow(S->cams, n_cams))) return st;
        S->cap_cams = n_cams;
    }
    if (cudaMemcpyAsync(S->cams, table.data(), sizeof(DevCam) * table.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return cuda_check("scene camera upload");
    S->table = table;
    SceneArgs& SA = S->args;
    SA = SceneArgs{};
    FwdArgs& A = SA.F;
    A.rec = accel->rec;
    A.sph = accel->sph;
    A.nodes = accel->nodes;
    A.top = accel->top;
    A.n_top = accel->n_top;
    A.wide = accel->wide;
    A.cams = S->cams;
    A.n_cams = n_cams;
    A.cam_single = -1;
    A.total_tiles = tiles;
    A.tile_w = tune->tile_w;
    TraceParams& P = A.P;
    P.Q = p->Q;
    P.eps1 = p->eps1;
    P.t_near = p->t_near;
    P.bg[0] = p->background[0];
    P.bg[1] = p->background[1];
    P.bg[2] = p->background[2];
    P.k_max = p->k_max;
    P.max_rounds = (int32_t)std::min<int64_t>(INT32_MAX, g->n / kSceneK + 3);
    P.max_visits = (int32_t)std::min<int64_t>(INT32_MAX, 2 * g->n + 16);
    P.n_gauss = (int32_t)g->n;
    P.n_nodes = (int32_t)std::max<int64_t>(1, g->n - 1);
    A.rgb = out->rgb;
    A.alpha = out->alpha;
    A.depth = out->depth;
    A.err = accel->err;
    SA.mesh = MeshDev{mesh->nodes, mesh->tris, mesh->albedo, mesh->n_nodes, mesh->n_tri};
    SA.light = make_float3(sp->light[0], sp->light[1], sp->light[2]);
    SA.max_bounces = sp->max_bounces;
    SA.eps_off = sp->eps_off;
    SA.list_cap = sp->list_cap;
    SA.shadow_cap = sp->shadow_cap;
    SA.sT = S->sT;
    SA.sn = S->sn;
    SA.ssn = S->ssn;
    SA.sE = S->sE;
    SA.seg = S->seg;
    SA.shadow = S->shadow;
    SA.ids = S->ids;
    SA.sids = S->sids;
    P.ids = S->ids;  // the segments' composited ids (segment << 30 | id)
    P.list_cap = sp->list_cap;
    const int block = 128;
    const int grid = (int)((tiles + 3) / 4);
    const size_t smem = (size_t)(block / 32) * kSceneK * 32 * sizeof(int64_t);
    k_render_scene<<<std::max(grid, 1), block, smem, s>>>(SA);
    st = cuda_check("scene render launch");
    if (st) return st;
    S->accel = accel;
    S->mesh = mesh;
    S->n_gauss = g->n;
    S->valid = true;
    return RS_OK;
}

rs_status rs_render_scene_backward(const rs_gaussians* g, const rs_accel* accel, const rs_scene_state* state,
                                   const rs_frame_grad* dl, rs_gaussian_grads* out, void* cuda_stream) {
    if (!g || !accel || !state || !dl || !dl->d_rgb || !out)
        return set_error(RS_ERR_INVALID_ARG, "scene backward: NULL argument");
    if (!state->valid || state->accel != accel || state->n_gauss != g->n || accel->n != g->n)
        return set_error(RS_ERR_INVALID_ARG, "scene backward: the state holds no render of this scene");
    rs_scene_state* S = const_cast<rs_scene_state*>(state);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (g->n > S->cap_gauss) {
        void* q = S->gtmp;
        const rs_status st = device_realloc(&q, sizeof(float4) * 4 * (size_t)g->n);
        S->gtmp = static_cast<float4*>(q);
        if (st) {
            S->cap_gauss = 0;
            return st;
        }
        S->cap_gauss = g->n;
    }
    if (cudaMemsetAsync(S->gtmp, 0, sizeof(float4) * 4 * (size_t)g->n, s) != cudaSuccess)
        return cuda_check("scene gradient scratch reset");
    BwdArgs B{dl->d_rgb, dl->d_alpha, dl->d_depth, S->gtmp, nullptr, 0};
    const int grid = (int)((S->args.F.total_tiles + 3) / 4);
    const size_t stage = (size_t)128 * BulkScatter::kFloat4 * sizeof(float4);
    if (dl->d_depth) k_scene_bwd<true><<<std::max(grid, 1), 128, stage, s>>>(S->args, B);
    else k_scene_bwd<false><<<std::max(grid, 1), 128, stage, s>>>(S->args, B);
    const cudaError_t e = launch_finalize(S->gtmp, accel->rec, accel->vals[0], g->quats, g->scales, g->n, *out, s);
    if (e != cudaSuccess) return set_error(RS_ERR_CUDA, "scene finalize launch: %s", cudaGetErrorString(e));
    return cuda_check("scene backward launch");
}

rs_status rs_scene_state_destroy(rs_scene_state* S) {
    if (!S) return RS_OK;
    cudaDeviceSynchronize();
    void* ptrs[] = {S->cams, S->sT, S->sn, S->ssn, S->sE, S->seg, S->shadow, S->ids, S->sids, S->gtmp};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete S;
    return cuda_check("rs_scene_state_destroy");
}

}  // extern "C"
