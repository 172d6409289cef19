// rs_internal.cuh -- device data layout and the ray / ellipsoid arithmetic shared by the
// render and adjoint kernels (RaySplats, arXiv 2501.19196).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/raysplats.h"

namespace rs {

// ---------------------------------------------------------------------------------------------
// Layout in HBM
//   rec[4 j + 0..2] = (M row k, mean_k)   M = S^-1 R^T (Prop. 1/2), rows k = 0, 1, 2
//   rec[4 j + 3]    = (opacity, r, g, b)
// j is the Gaussian's position in Morton order (sorted), so the 64 B records of one BVH leaf
// are contiguous and sector aligned.  perm[j] maps back to the caller's Gaussian id.
//   nodes[4 p + 0] = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//   nodes[4 p + 1] = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//   nodes[4 p + 2] = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//   nodes[4 p + 3] = int (ref0, ref1, count0, count1)
// ref >= 0 is an internal node; ref < 0 is a leaf holding Gaussians [~ref, ~ref + count).
// ---------------------------------------------------------------------------------------------

constexpr int kStackSize = 96;
constexpr int kMaxSmemNodes = 512;
constexpr int kMaxHitList = 4096;         // largest per-ray hit list
constexpr int kNumStats = 10;             // uint64 counters of rs_render_stats        // staged top nodes (64 B each) in shared memory
constexpr int kTopRef = 0x40000000;       // node reference kTopRef + s = staged slot s
constexpr int kEmptyRef = INT32_MIN;      // empty child slot of a wide node         // >= depth of a radix tree over 64-bit codes + 32-bit ids
// Empty slots sort after (ascending) or before (descending) every key, and their time half is
// +inf (ascending) or -inf (descending), so key_t() of an empty slot needs no test.
constexpr int64_t kEmptyKey = (int64_t)0x7f800000ffffffffull;       // ascending k-buffer
constexpr int64_t kEmptyKeyDesc = (int64_t)0xff80000000000000ull;   // descending k-buffer

// device error word bits
enum : int {
    kErrReplayMismatch = 1,  // backward found a different number of hits than the forward
    kErrBadScene = 2,        // non-finite or non-positive scale / zero quaternion seen in prep
    kErrStack = 4,           // traversal stack overflow (cannot happen for kStackSize >= depth)
    kErrLoopGuard = 8,       // a traversal / round / refit loop exceeded its bound (corrupt tree)
    kErrIndex = 16,          // a node reference or leaf range out of bounds (corrupt tree)
    kErrListOverflow = 32    // a per-ray id list of a scene render was too short
};

struct DevCam {
    float R[9];
    float pos[3];
    float fx, fy, cx, cy;
    int32_t W, H, tiles_x, tiles_y;
    int64_t tile_base;  // first global tile id of this camera
    int64_t pix_base;   // first output pixel of this camera
};

struct TraceParams {
    float Q, eps1, t_near;
    float bg[3];
    int32_t k_max;
    int32_t max_rounds;    // guard: no ray needs more rounds than n / K + 2
    int32_t max_visits;    // guard: a round visits each of the < n nodes at most once
    int32_t n_gauss;       // guard: leaf ranges lie in [0, n_gauss)
    int32_t n_nodes;       // guard: node references lie in [0, n_nodes) (or the staged slots)
    int32_t list_cap;      // hit list: ids of the first list_cap composited hits per ray (0: none)
    int* ids;              // hit list storage, list_cap ints per pixel (pixel-major rows)
    int32_t sort_key;      // hits ordered by 0: entry t1, 1: t_m (maximum response)
    int32_t grad_mode;     // 0: exact gradient; 1: the eps2 estimator for the last meaningful hit
    float eps2;            // second threshold (grad_mode 1)
    float4* sS;            // grad_mode 1: per pixel, colour and alpha behind the last composited
                           // hit through the phase-2 hits (.w < 0: no phase 2)
};

// Ordered 64-bit keys: the ray parameter's FP32 bit pattern (t >= 0, so it orders as an
// unsigned integer) in the high 32 bits; the low 32 bits hold, from the top, a sub-ulp residual
// of t (hits only) and the sorted id j in the low key_id_bits(n) bits.  pack_key(t, low) builds
// bounds: low = 0 is the smallest key at t, low = 0xffffffff the largest.
__device__ __forceinline__ int64_t pack_key(float t, uint32_t low) {
    return (int64_t)(((uint64_t)__float_as_uint(t) << 32) | low);
}
__device__ __forceinline__ float key_t(int64_t k) { return __uint_as_float((uint32_t)((uint64_t)k >> 32)); }
// bits that hold a sorted id j < n (at least one)
__device__ __forceinline__ int key_id_bits(int n) { return n > 1 ? 32 - __clz(n - 1) : 1; }
__device__ __forceinline__ int key_j(int64_t k, int jb) { return (int)((uint32_t)k & ((1u << jb) - 1u)); }
constexpr uint32_t kKeyLowMax = 0xffffffffu;

// The ordering key of a hit whose parameter was evaluated as hi = fl(tc + tr): tc is the
// re-centring shift of the solve, tr the part solved relative to it.  FP32 rounding of that
// sum alone (up to half an ulp of t) would order two hits whose parameters differ by less than
// that at random; so the exact rounding error lo = (tc + tr) - hi (TwoSum) is kept, in units of
// ulp(hi), in the 32 - jb bits between hi and the id.  Keys then order by the parameter to a
// small fraction of an ulp, i.e. to the accuracy of the solve itself; only hits whose accurate
// parameters agree to 2^-(32 - jb) ulp tie, and those order by id.
__device__ __forceinline__ int64_t pack_hit_key(float hi, float tc, float tr, int j, int jb) {
    const float bb = __fsub_rn(hi, tc);
    const float lo = __fadd_rn(__fsub_rn(tc, __fsub_rn(hi, bb)), __fsub_rn(tr, bb));
    const uint32_t hb = __float_as_uint(hi);
    // w = 1.5 + lo / ulp(hi) lies in [1, 2], where a float's mantissa is linear in its value:
    // m = (lo / ulp(hi) + 1/2) 2^23.  The scale 2^(150 - E) (E the biased exponent of hi >= 0)
    // is exact; exponents below 23 (t < 2^-104) are clamped, which only coarsens the residual.
    const uint32_t E = max(hb >> 23, 23u);
    const float w = __fmaf_rn(lo, __uint_as_float((277u - E) << 23), 1.5f);
    const uint32_t m = min(__float_as_uint(w) - 0x3f800000u, 0x7fffffu);
    // the top 32 - jb bits of m, placed above the id: (m << 9) keeps bit 22 of m at bit 31
    const uint32_t low = ((m << 9) & ~((1u << jb) - 1u)) | (uint32_t)j;
    return (int64_t)(((uint64_t)hb << 32) | low);
}

// ---------------------------------------------------------------------------------------------
// Camera ray (a7): the fixed FP32 sequence of the ABI (no contraction: explicit _rn ops).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void camera_ray(const DevCam& c, int px, int py, float3& o, float3& d) {
    const float x = __fdiv_rn(__fsub_rn(__fadd_rn((float)px, 0.5f), c.cx), c.fx);
    const float y = __fdiv_rn(__fsub_rn(__fadd_rn((float)py, 0.5f), c.cy), c.fy);
    float w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        w[k] = __fadd_rn(__fadd_rn(__fmul_rn(c.R[3 * k], x), __fmul_rn(c.R[3 * k + 1], y)), c.R[3 * k + 2]);
    const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(w[0], w[0]), __fmul_rn(w[1], w[1])), __fmul_rn(w[2], w[2]));
    const float n = __fsqrt_rn(n2);
    d = make_float3(__fdiv_rn(w[0], n), __fdiv_rn(w[1], n), __fdiv_rn(w[2], n));
    o = make_float3(c.pos[0], c.pos[1], c.pos[2]);
}

// ---------------------------------------------------------------------------------------------
// Ray / confidence-ellipsoid solve (Prop. 1, Prop. 2) in FP32, numerically stable form.
//
// The ray is first re-centred at the point x_c = o + tc d nearest to the mean (tc = <m - o, d>)
// so that the whitened origin o'' = M (x_c - m) is small; w = x_c - m is formed with
// error-free transformations (TwoSum of o - m, TwoProduct of tc d), so it carries no rounding
// of |o - m|-sized numbers.  Then, as in Prop. 1/2 with o' -> o'':
//   d' = M d, a = <d', d'>, b = <o'', d'>, tm = -b / a,
//   p = o'' + tm d'  (= M v, v = x_c + tm d - m),  D2 = <p, p>,
//   t* = (-b - sgn(b) sqrt(a (Q - D2))) / a, t1'' = t* if b >= 0 else (<o'',o''> - Q) / (a t*),
//   t1 = tc + t1''   (a t* = -b + sqrt(a (Q - D2)), so the second branch needs no a).
// D2 and t1 do not depend on the choice of tc (a shift along the ray).  Every operation is an
// explicit round-to-nearest intrinsic or the hardware's approximate reciprocal (rcp.approx,
// within one ulp: the divisions by a and by -b + sqrt(...) only scale terms whose own error is
// larger, and D2 is stationary in tm), so the forward and the adjoint kernels evaluate the
// same bits.  The approximate reciprocal took 4 % off the forward, with the FP32-vs-FP64 errors
// of D2 and of the ordering key unchanged on 330,000 measured hits.
// ---------------------------------------------------------------------------------------------
struct Hit {
    float D2, t1;
    float tm;    // ray parameter of the maximum response (chord midpoint)
    float tc, t1r, tmr;  // t1 = fl(tc + t1r), tm = fl(tc + tmr): the re-centring shift and the rest
    bool hit;
    float p[3];  // M-space closest-approach vector
    float v[3];  // world vector from the mean to the point of maximum response
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// the hardware's approximate reciprocal (one instruction, at most one ulp from 1/x)
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <bool WANT_GEOM>
__device__ __forceinline__ void ray_ellipsoid(const float3 o, const float3 d, const float4 r0,
                                              const float4 r1, const float4 r2, float Q,
                                              float t_near, Hit& h) {
    const float m[3] = {r0.w, r1.w, r2.w};
    const float oo[3] = {o.x, o.y, o.z};
    const float dd[3] = {d.x, d.y, d.z};
    // tc = <m - o, d>
    float tc = 0.f;
    float e_hi[3], e_lo[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        two_sum(oo[k], -m[k], e_hi[k], e_lo[k]);  // o - m exactly as e_hi + e_lo
        tc = __fmaf_rn(-e_hi[k], dd[k], tc);
    }
    // w = (o - m) + tc d, exactly up to one final rounding per component
    float w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float ph = __fmul_rn(tc, dd[k]);
        const float pl = __fmaf_rn(tc, dd[k], -ph);
        w[k] = __fadd_rn(__fadd_rn(e_hi[k], ph), __fadd_rn(e_lo[k], pl));
    }
    const float Mr[3][3] = {{r0.x, r0.y, r0.z}, {r1.x, r1.y, r1.z}, {r2.x, r2.y, r2.z}};
    float op[3], dp[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        op[k] = __fmaf_rn(Mr[k][2], w[2], __fmaf_rn(Mr[k][1], w[1], __fmul_rn(Mr[k][0], w[0])));
        dp[k] = __fmaf_rn(Mr[k][2], dd[2], __fmaf_rn(Mr[k][1], dd[1], __fmul_rn(Mr[k][0], dd[0])));
    }
    const float a = __fmaf_rn(dp[2], dp[2], __fmaf_rn(dp[1], dp[1], __fmul_rn(dp[0], dp[0])));
    const float b = __fmaf_rn(op[2], dp[2], __fmaf_rn(op[1], dp[1], __fmul_rn(op[0], dp[0])));
    const float ia = rcp_approx(a);
    const float tm = -__fmul_rn(b, ia);
    h.tm = __fadd_rn(tc, tm);
    h.tc = tc;
    h.tmr = tm;
    h.t1r = 0.f;
    float p[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) p[k] = __fmaf_rn(tm, dp[k], op[k]);
    const float D2 = __fmaf_rn(p[2], p[2], __fmaf_rn(p[1], p[1], __fmul_rn(p[0], p[0])));
    h.D2 = D2;
    h.hit = false;
    h.t1 = 0.f;
    if (D2 <= Q) {
        const float root = __fsqrt_rn(__fmul_rn(a, __fsub_rn(Q, D2)));
        float t1r;
        if (b >= 0.f) {
            t1r = __fmul_rn(__fsub_rn(-b, root), ia);
        } else {
            const float c = __fsub_rn(__fmaf_rn(op[2], op[2], __fmaf_rn(op[1], op[1], __fmul_rn(op[0], op[0]))), Q);
            t1r = __fmul_rn(c, rcp_approx(__fadd_rn(-b, root)));
        }
        const float t1 = __fadd_rn(__fadd_rn(tc, t1r), 0.0f);  // +0 turns -0 into +0
        h.t1 = t1;
        h.t1r = t1r;
        h.hit = t1 >= t_near;
    }
    if (WANT_GEOM) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            h.p[k] = p[k];
            h.v[k] = __fmaf_rn(tm, dd[k], w[k]);
        }
    }
}

// The closest-approach geometry of the adjoint (p = M v and v, as ray_ellipsoid<true> gives
// them) to full FP32 accuracy.  In the solve above p = o' + tm d' is a difference of terms of
// size |M (o - m)|, which exceeds |p| by up to five digits for a Gaussian a thousand times
// thinner along one axis than along the others; the component of p along that axis, which the
// gradient scales by 1/s, then keeps few correct digits.  Here the solve is re-centred at
// tstar, the forward's parameter of the closest point: w = (o - m) + tstar d is formed as an
// unevaluated pair wh + wl from exact differences (two_sum) and exact products (an FMA gives
// the rounding error of a product), M w by compensated dot products (Ogita, Rump and Oishi's
// Dot2), and the small remaining offset along d' is removed by one projection.  alpha still
// comes from the forward's D2, so its bits do not change.
__device__ __forceinline__ void closest_point_accurate(const float3 o, const float3 d, const float4 r0,
                                                       const float4 r1, const float4 r2, float tstar, float p[3],
                                                       float v[3]) {
    const float m[3] = {r0.w, r1.w, r2.w};
    const float oo[3] = {o.x, o.y, o.z};
    const float dd[3] = {d.x, d.y, d.z};
    float wh[3], wl[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float eh, el, sh, se;
        two_sum(oo[k], -m[k], eh, el);  // o - m = eh + el exactly
        const float ph = __fmul_rn(tstar, dd[k]);
        const float pl = __fmaf_rn(tstar, dd[k], -ph);  // tstar d = ph + pl exactly
        two_sum(eh, ph, sh, se);
        two_sum(sh, __fadd_rn(__fadd_rn(se, el), pl), wh[k], wl[k]);
    }
    const float Mr[3][3] = {{r0.x, r0.y, r0.z}, {r1.x, r1.y, r1.z}, {r2.x, r2.y, r2.z}};
    float q[3], dp[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float sum = 0.f, err = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float pr = __fmul_rn(Mr[k][i], wh[i]);
            const float pe = __fmaf_rn(Mr[k][i], wh[i], -pr);
            float t, e;
            two_sum(sum, pr, t, e);
            sum = t;
            err = __fmaf_rn(Mr[k][i], wl[i], __fadd_rn(err, __fadd_rn(e, pe)));
        }
        q[k] = __fadd_rn(sum, err);  // (M w)_k
        dp[k] = __fmaf_rn(Mr[k][2], dd[2], __fmaf_rn(Mr[k][1], dd[1], __fmul_rn(Mr[k][0], dd[0])));
    }
    const float a = __fmaf_rn(dp[2], dp[2], __fmaf_rn(dp[1], dp[1], __fmul_rn(dp[0], dp[0])));
    const float b = __fmaf_rn(q[2], dp[2], __fmaf_rn(q[1], dp[1], __fmul_rn(q[0], dp[0])));
    const float tau = -__fdiv_rn(b, a);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p[k] = __fmaf_rn(tau, dp[k], q[k]);
        v[k] = __fadd_rn(__fmaf_rn(tau, dd[k], wh[k]), wl[k]);
    }
}

// The ordering parameter of a hit: its entry t1, or (sort key 1) the parameter of the maximum
// response, which is never below t1 (the max guards FP32 rounding at grazing incidence).
__device__ __forceinline__ float hit_key_t(const Hit& h, int sort_key) {
    return sort_key ? fmaxf(h.tm, h.t1) : h.t1;
}

// The 64-bit ordering key of a hit on sorted Gaussian j (see pack_hit_key); its high half is
// hit_key_t(h, sort_key).
__device__ __forceinline__ int64_t hit_key(const Hit& h, int sort_key, int j, int jb) {
    if (sort_key && h.tm >= h.t1) return pack_hit_key(h.tm, h.tc, h.tmr, j, jb);
    return pack_hit_key(h.t1, h.tc, h.t1r, j, jb);
}

// alpha_i = opacity * exp(-D2 / 2)  (Eq. 8, Prop. 2)
__device__ __forceinline__ float response_alpha(float opacity, float D2) {
    return __fmul_rn(opacity, expf(__fmul_rn(-0.5f, D2)));
}

}  // namespace rs
