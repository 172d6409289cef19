/*
 * raysplats_oracle.c -- plain, slow CPU reference of the RaySplats rendering path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py may load this library.  The product path (the CUDA library in
 * paper_2501_19196_gb300/) never links, imports or calls it, and it shares no code with it.
 *
 * What it computes, with the paper passage each part follows (RaySplats, arXiv 2501.19196):
 *   - rotation from an unnormalised quaternion, s = 2/|q|^2 ........ App. A.6
 *   - Sigma = R S S^T R^T, whitening M = S^-1 R^T ................... Eq. 2, Prop. 2
 *   - ray / confidence-ellipsoid entry t1 (stable root + Viete) ..... Prop. 1, App. A.1
 *   - miss rule: no real root, or nearer root t1 below t_near ....... Sec. 3 "Intersection"
 *   - maximum response alpha = opacity * exp(-D^2/2) ................ Eq. 8, Prop. 2, App. A.2
 *   - front-to-back compositing with the eps1 cut and K_max ......... Eq. 3, Sec. 3 (Alg. 1 prose)
 *   - exact gradient of the rendered pixel w.r.t. every parameter .. App. A.3-A.6
 *   - Morton codes / stable order / binary radix tree ............... (acceleration structure;
 *     no paper counterpart -- the plain definitions of the Karras 2012 hierarchy)
 * Every floating-point step runs in FP64, except ray generation (raygen_f32) and Morton
 * quantisation, which are defined as fixed FP32 operation sequences so that both
 * implementations take the same discrete decisions.  Build with -ffp-contract=off.
 *
 * Every test is brute force: each ray is tested against every Gaussian (no acceleration).
 *
 * Readings of the paper that this file fixes (where the text is silent or garbled):
 *   - the norm in Prop. 2 is the SQUARED Mahalanobis distance D^2 (Gaussian definition);
 *   - Prop. 1's root uses sqrt(a (Q - D^2)) / a (the appendix form);
 *   - <o',d'> >= 0 takes the first branch; a ray is a hit at D^2 == Q (inclusive);
 *   - hits are ordered by (t_key, index) ascending, where t_key is the entry t1 (sort key 0)
 *     or the parameter t_m of the maximum response (sort key 1, the chord midpoint); the hit
 *     that brings T below eps1 is composited, then the ray stops; at most k_max hits are
 *     composited;
 *   - RGB = C + T_final * background, alpha = 1 - T_final, depth = sum w_i t_key_i;
 *   - the gradient is the exact derivative of those outputs (depth included) with the hit
 *     set, order and cut point held fixed (grad_mode 0);
 *   - grad_mode 1 is the paper's eps2 estimator (Sec. 3, Sec. 5): when T falls below eps1 at
 *     hit i, the hits behind it are collected in order, without compositing, until the
 *     product of their (1 - alpha) falls below eps2; dL/dalpha_i then uses the colour S and
 *     alpha S_A seen behind i through those hits (plus the background through what they let
 *     pass) instead of the background alone.  Every other gradient term is unchanged.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------ */
/* Plain data types (declared here independently; only the memory layout matches the      */
/* Python side of the oracle).                                                            */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    float R_wc[9]; /* camera -> world rotation, row major; camera axes x right, y down, z fwd */
    float pos[3];  /* camera centre in world space */
    float fx, fy, cx, cy;
    int32_t width, height;
} or_camera;

typedef struct {
    double Q;        /* squared Mahalanobis radius of the confidence ellipsoid */
    double eps1;     /* transmittance cut */
    double t_near;   /* rays start at t_near (>= 0) */
    double bg[3];    /* background colour */
    int32_t k_max;   /* at most k_max composited hits per ray */
    int32_t sort_key; /* 0: order hits by entry t1; 1: by t_m, the maximum-response parameter */
    double eps2;      /* second threshold of the last "meaningful" Gaussian's gradient (Sec. 3) */
    int32_t grad_mode; /* 0: exact gradient of the rendered image; 1: the eps2 estimator */
    int32_t pad;
} or_params;

/* Ambiguity flags (per ray).  FP32 and FP64 may legitimately take a different discrete
 * decision on such a ray:
 *   BOUNDARY  a Gaussian whose |Q - D^2| lies within the FP32 uncertainty of D^2 (see below), at
 *             or before the stop point,
 *   TIE       two consecutive hits whose t lie closer than their combined FP32 uncertainty
 *             (see OR_T_ERR_C below; up to the hit after the stop),
 *   EPS1      the transmittance after some composited hit within 1e-4 relative of eps1,
 *   TNEAR     a hit candidate with t1 within OR_TIE_REL max(1, t) of t_near.
 * IMPACT is set when one of those alternative decisions (toggle the boundary Gaussian, swap
 * the tied pair, flip the eps1 stop) changes the ray's RGB or alpha by more than
 * OR_IMPACT_TOL; only such pixels have no unique correct value at the parity tolerance. */
enum {
    OR_AMB_BOUNDARY = 1,
    OR_AMB_TIE = 2,
    OR_AMB_EPS1 = 4,
    OR_AMB_TNEAR = 8,
    OR_AMB_IMPACT = 16,
    OR_AMB_EPS2 = 256, /* a phase-2 product within 1e-4 relative of eps2 (the eps2 stop) */
    /* which alternative produced the impact (diagnostics) */
    OR_IMP_BOUNDARY = 32,
    OR_IMP_TIE = 64,
    OR_IMP_EPS1 = 128
};
/* The bands follow the FP32 error of the renderer's ray/ellipsoid solve.  BOUNDARY uses a band
 * per Gaussian (d2tol, a first-order model of that error, see ray_gauss); TIE uses a band per
 * pair of hits: the sum of their t-uncertainties (ttol) plus OR_T_QUANTUM units of the FP32
 * spacing at t (the renderer orders by keys resolved to a fraction of that spacing).  TNEAR
 * keeps a relative band: the renderer's t >= t_near test uses the FP32-rounded t.  The renderer
 * rounds each entry of the whitening once from FP64; on 330,000 hits of three scenes its
 * measured errors then stay below 1.9 (t1), 2.5 (t_m) and 2.7 (D2) times the unscaled models, so
 * the scales below leave a margin of two.  The D2 model is capped at OR_BOUNDARY_REL Q: its
 * flat-Gaussian term assumes a worst-case rounding of the whitening, while the largest measured
 * D2 error is 3.8e-6 Q. */
#define OR_IMPACT_TOL 1e-4
#define OR_BOUNDARY_REL 1e-5
#define OR_TIE_REL 5e-7
#define OR_T_ERR_C 4.0
#define OR_TM_ERR_C 5.0
#define OR_D2_ERR_C 6.0
#define OR_T_QUANTUM (1.0 / 256.0)

/* ------------------------------------------------------------------------------------ */
/* App. A.6: rotation matrix from a (possibly unnormalised) quaternion q = (a, b, c, d),  */
/* a the real part; s = 2 / |q|^2.  R = I + s K(q) with K quadratic in q.                  */
/* ------------------------------------------------------------------------------------ */
static void quat_to_K(const double q[4], double K[9]) {
    const double a = q[0], b = q[1], c = q[2], d = q[3];
    K[0] = -(c * c + d * d); K[1] = b * c - a * d;       K[2] = b * d + a * c;
    K[3] = b * c + a * d;    K[4] = -(b * b + d * d);    K[5] = c * d - a * b;
    K[6] = b * d - a * c;    K[7] = c * d + a * b;       K[8] = -(b * b + c * c);
}

void or_quat_to_rot(const double q[4], double R[9]) {
    double K[9];
    const double s = 2.0 / (q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    quat_to_K(q, K);
    for (int i = 0; i < 9; ++i) R[i] = ((i % 4) == 0 ? 1.0 : 0.0) + s * K[i];
}

/* dR/dq_x for x = 0..3 (a, b, c, d): d(sK)/dq_x = (ds/dq_x) K + s dK/dq_x, ds/dq_x = -s^2 q_x.
 * Derived directly from the App. A.6 formula for R (the printed dR^T/dq matrices are not used). */
static void quat_drot(const double q[4], double dR[4][9]) {
    const double a = q[0], b = q[1], c = q[2], d = q[3];
    const double s = 2.0 / (a * a + b * b + c * c + d * d);
    double K[9];
    quat_to_K(q, K);
    const double dK[4][9] = {
        {0, -d, c, d, 0, -b, -c, b, 0},
        {0, c, d, c, -2 * b, -a, d, a, -2 * b},
        {-2 * c, b, a, b, 0, d, -a, d, -2 * c},
        {-2 * d, -a, b, a, -2 * d, c, b, c, 0},
    };
    for (int x = 0; x < 4; ++x) {
        const double ds = -s * s * q[x];
        for (int i = 0; i < 9; ++i) dR[x][i] = ds * K[i] + s * dK[x][i];
    }
}

/* Whitening M = S^-1 R^T (Prop. 1/2): M[k][l] = R[l][k] / s_k. */
static void whitening(const double q[4], const double s[3], double M[9]) {
    double R[9];
    or_quat_to_rot(q, R);
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) M[3 * k + l] = R[3 * l + k] / s[k];
}

/* ------------------------------------------------------------------------------------ */
/* Ray generation.  A pinhole ray through the pixel centre, origin at the camera centre,  */
/* unit direction.  Defined as a fixed FP32 operation sequence (each +,-,*,/ and sqrt     */
/* rounded to nearest, no fused multiply-add) so the CUDA path reproduces it bit-exactly. */
/* ------------------------------------------------------------------------------------ */
static void ray_f32(const or_camera* c, int32_t px, int32_t py, float o[3], float d[3]) {
    const float x = (((float)px + 0.5f) - c->cx) / c->fx;
    const float y = (((float)py + 0.5f) - c->cy) / c->fy;
    float w[3];
    for (int k = 0; k < 3; ++k) {
        const float t0 = c->R_wc[3 * k + 0] * x;
        const float t1 = c->R_wc[3 * k + 1] * y;
        w[k] = (t0 + t1) + c->R_wc[3 * k + 2];
    }
    const float n2 = ((w[0] * w[0]) + (w[1] * w[1])) + (w[2] * w[2]);
    const float n = sqrtf(n2);
    for (int k = 0; k < 3; ++k) {
        d[k] = w[k] / n;
        o[k] = c->pos[k];
    }
}

void or_raygen_f32(const or_camera* cams, int64_t n_rays, const int32_t* ray_cam,
                   const int32_t* px, const int32_t* py, float* o, float* d) {
    for (int64_t r = 0; r < n_rays; ++r) ray_f32(&cams[ray_cam[r]], px[r], py[r], o + 3 * r, d + 3 * r);
}

/* The same ray in FP64 (for closed-form pins that need more than FP32 resolution). */
void or_raygen_f64(const double* cam /* R_wc[9], pos[3], fx, fy, cx, cy */, int64_t n_rays,
                   const int32_t* px, const int32_t* py, double* o, double* d) {
    for (int64_t r = 0; r < n_rays; ++r) {
        const double x = ((double)px[r] + 0.5 - cam[14]) / cam[12];
        const double y = ((double)py[r] + 0.5 - cam[15]) / cam[13];
        double w[3];
        for (int k = 0; k < 3; ++k) w[k] = cam[3 * k] * x + cam[3 * k + 1] * y + cam[3 * k + 2];
        const double n = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        for (int k = 0; k < 3; ++k) {
            d[3 * r + k] = w[k] / n;
            o[3 * r + k] = cam[9 + k];
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* One ray against one Gaussian: Prop. 1 (entry t1) and Prop. 2 (D^2).                    */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    double op[3], dp[3]; /* o' = M (o - m), d' = M d */
    double a, b;         /* a = <d',d'>, b = <o',d'> */
    double tau;          /* b / a */
    double p[3];         /* o' - tau d'  (the M-space closest-approach vector) */
    double D2;           /* <p, p> = squared Mahalanobis distance of the ray (Prop. 2) */
    double t1;           /* ellipsoid entry (valid when D2 <= Q) */
    double ttol;         /* uncertainty of an FP32 evaluation of t1 (hits) */
    double mtol;         /* the same for the maximum-response parameter -tau */
    double d2tol;        /* the same for D2 (hits and near misses) */
} or_geom;

/* FP32 spacing (ulp) at |t| */
static double ulp32(double t) {
    int e = 0;
    frexp(fabs(t), &e);
    return ldexp(1.0, e - 24);
}

static void ray_gauss(const double o[3], const double d[3], const double m[3], const double M[9],
                      double Q, or_geom* g) {
    double om[3] = {o[0] - m[0], o[1] - m[1], o[2] - m[2]};
    for (int k = 0; k < 3; ++k) {
        g->op[k] = M[3 * k] * om[0] + M[3 * k + 1] * om[1] + M[3 * k + 2] * om[2];
        g->dp[k] = M[3 * k] * d[0] + M[3 * k + 1] * d[1] + M[3 * k + 2] * d[2];
    }
    g->a = g->dp[0] * g->dp[0] + g->dp[1] * g->dp[1] + g->dp[2] * g->dp[2];
    g->b = g->op[0] * g->dp[0] + g->op[1] * g->dp[1] + g->op[2] * g->dp[2];
    g->tau = g->b / g->a;
    for (int k = 0; k < 3; ++k) g->p[k] = g->op[k] - g->tau * g->dp[k];
    g->D2 = g->p[0] * g->p[0] + g->p[1] * g->p[1] + g->p[2] * g->p[2];
    /* Prop. 1 (App. A.1): t* = (-b - sgn(b) sqrt(a (Q - D2))) / a;  t1 = t* if b >= 0,
     * else (<o',o'> - Q) / (a t*) (Viete).  For D2 > Q (no root) t1 is evaluated at the
     * clamped discriminant so that near misses still get a position for the ambiguity test. */
    const double disc = g->a * (Q - g->D2 > 0.0 ? Q - g->D2 : 0.0);
    const double root = sqrt(disc);
    if (g->b >= 0.0) {
        g->t1 = (-g->b - root) / g->a;
    } else {
        const double tstar = (-g->b + root) / g->a;
        const double c = (g->op[0] * g->op[0] + g->op[1] * g->op[1] + g->op[2] * g->op[2]) - Q;
        g->t1 = c / (g->a * tstar);
    }
    /* Uncertainty model of an FP32 evaluation of the solve (relative rounding u = 2^-24), in
     * world units.  A solve re-centred at the ray point nearest the mean works with the offset
     * w = (o - m) - <o - m, d> d, the step tm_r from there to the maximum response, and the half
     * chord r = sqrt((Q - D2) / a).  Rounding of these gives errors of size |w| + r.  A rounded
     * whitening M (rows of size 1 / s_k) perturbs M w and M d by about u |w| / s_min and
     * u / s_min, which moves t by (|w| + |tm_r| + r) k with k = 1 / (s_min |M d|) (1 for an
     * isotropic Gaussian, up to s_max / s_min for a flat one seen edge-on), and moves D2 by
     * about 2 D |v| / s_min (v = w + tm_r d, the closest-approach offset); an error of D2 enters
     * t1 amplified by 1 / (2 a r), i.e. by D / sqrt(Q - D2) relative to the terms above.  These
     * are models, not bounds: OR_T_ERR_C, OR_TM_ERR_C and OR_D2_ERR_C scale them to cover the
     * FP32 errors measured on the renderer's solve with a margin of two. */
    g->ttol = g->mtol = g->d2tol = 0.0;
    if (g->D2 > 1.01 * Q) return; /* far from a hit: no decision to flag */
    const double od = om[0] * d[0] + om[1] * d[1] + om[2] * d[2];
    double w[3], v[3], rowmax = 0.0;
    const double tmr = -g->tau + od; /* maximum response relative to the re-centred point */
    for (int k = 0; k < 3; ++k) {
        w[k] = om[k] - od * d[k];
        v[k] = w[k] + tmr * d[k];
        const double rn = M[3 * k] * M[3 * k] + M[3 * k + 1] * M[3 * k + 1] + M[3 * k + 2] * M[3 * k + 2];
        rowmax = fmax(rowmax, rn);
    }
    const double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    const double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const double inv_smin = sqrt(rowmax); /* rows of M = S^-1 R^T have norms 1 / s_k */
    const double kk = inv_smin / sqrt(g->a);
    const double D = sqrt(g->D2);
    const double u = ldexp(1.0, -24);
    g->d2tol = fmin(OR_D2_ERR_C * u * (g->D2 + 2.0 * D * vn * inv_smin), OR_BOUNDARY_REL * Q);
    if (g->D2 > Q) return;
    const double gap = Q - g->D2;
    const double r = sqrt(gap / g->a);
    const double amp = gap > 0.0 ? D / sqrt(gap) : INFINITY;
    g->ttol = OR_T_ERR_C * u * (kk * (wn + fabs(tmr) + r) * (1.0 + amp) + wn + r);
    g->mtol = OR_TM_ERR_C * u * (kk + 1.0) * (wn + fabs(tmr));
}

/* Exported for unit pins: one ray (double) against one Gaussian given by (mean, quat, scale).
 * out[0] = D2, out[1] = t1, out[2] = hit flag (1/0), out[3] = tau = <o',d'>/<d',d'>,
 * out[4] = the t1 uncertainty model (ttol), out[5] = the D2 uncertainty model (d2tol),
 * out[6] = the t_m uncertainty model (mtol). */
void or_ray_gaussian(const double o[3], const double d[3], const double m[3], const double q[4],
                     const double s[3], double Q, double t_near, double out[7]) {
    double M[9];
    or_geom g;
    whitening(q, s, M);
    ray_gauss(o, d, m, M, Q, &g);
    out[0] = g.D2;
    out[1] = g.t1;
    out[2] = (g.D2 <= Q && g.t1 >= t_near) ? 1.0 : 0.0;
    out[3] = g.tau;
    out[4] = g.ttol;
    out[5] = g.d2tol;
    out[6] = g.mtol;
}

/* ------------------------------------------------------------------------------------ */
/* Per-ray render (+ optional gradient), brute force over all Gaussians.                  */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    double t;
    int64_t idx;
    double D2;
    double tol; /* uncertainty of an FP32 evaluation of t (TIE band) */
} or_hit;

static int hit_cmp(const void* x, const void* y) {
    const or_hit* a = (const or_hit*)x;
    const or_hit* b = (const or_hit*)y;
    if (a->t < b->t) return -1;
    if (a->t > b->t) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx ? 1 : 0);
}

typedef struct {
    int64_t idx;
    double v[14]; /* d means[3], d quats[4], d scales[3], d opacity, d rgb[3] */
} or_contrib;

typedef struct {
    /* scene */
    int64_t n;
    const double *means, *quats, *scales, *opac, *rgb;
    const double* M; /* 9 per Gaussian, precomputed whitening */
    /* rays */
    int64_t n_rays;
    const double *ray_o, *ray_d;
    const or_params* prm;
    /* outputs */
    double *out_rgb, *out_alpha, *out_depth, *out_T;
    int32_t *out_nhits, *out_mask;
    /* gradient inputs */
    const double *dl_rgb, *dl_alpha, *dl_depth;
    /* work split */
    int64_t r0, r1;
    /* per-thread gradient contributions */
    or_contrib* contrib;
    int64_t n_contrib, cap_contrib;
    int failed;
} or_job;

static void push_contrib(or_job* J, int64_t idx, const double v[14]) {
    if (J->n_contrib == J->cap_contrib) {
        int64_t cap = J->cap_contrib ? 2 * J->cap_contrib : 1024;
        or_contrib* p = (or_contrib*)realloc(J->contrib, (size_t)cap * sizeof(or_contrib));
        if (!p) {
            J->failed = 1;
            return;
        }
        J->contrib = p;
        J->cap_contrib = cap;
    }
    J->contrib[J->n_contrib].idx = idx;
    memcpy(J->contrib[J->n_contrib].v, v, sizeof(double) * 14);
    J->n_contrib++;
}

/* App. A.6 chain from dL/dalpha (and dL/dt_key for the depth output) of hit Gaussian i on the
 * ray (o, d) to its mean, quaternion, scales and opacity: fills v[0..10]. */
static void param_chain(const or_job* J, const double o[3], const double d[3], int64_t i, double a,
                        double dLda, double dLdt, double v[14]) {
    const double Q = J->prm->Q;
    const double* m = J->means + 3 * i;
    const double* q = J->quats + 4 * i;
    const double* s = J->scales + 3 * i;
    const double* M = J->M + 9 * i;
    or_geom g;
    ray_gauss(o, d, m, M, J->prm->Q, &g);
    const double e = exp(-0.5 * g.D2);
    v[10] = dLda * e;                         /* d opacity */
    const double dLdD2 = -0.5 * a * dLda;     /* alpha = opacity exp(-D2/2) */
    /* t_key as a function of (o', d'): t_m = -tau = -b/a and t1 = t_m - r with
     * r = sqrt((Q - D2)/a), so
     *   dt_m = -db/a + tau da/a,  dt1 = dt_m + dD2/(2 r a) + (Q - D2) da/(2 r a^2),
     * with da = 2<d', dd'>, db = <do', d'> + <o', dd'> and dD2 as below. */
    const int use_tm = J->prm->sort_key == 1;
    const double rr = sqrt(fmax(Q - g.D2, 0.0) / g.a);
    /* dD2/dbox = 2<p, do'> - 2 tau <p, dd'> */
    double om[3] = {o[0] - m[0], o[1] - m[1], o[2] - m[2]};
    /* means: do'/dm_x = -M e_x, dd'/dm_x = 0 */
    for (int x = 0; x < 3; ++x) {
        double dop[3] = {-M[x], -M[3 + x], -M[6 + x]};
        double dD2 = 2.0 * (g.p[0] * dop[0] + g.p[1] * dop[1] + g.p[2] * dop[2]);
        v[x] = dLdD2 * dD2;
        if (dLdt != 0.0) {
            const double db = dop[0] * g.dp[0] + dop[1] * g.dp[1] + dop[2] * g.dp[2];
            const double dtm = -db / g.a; /* da = 0 */
            v[x] += dLdt * (use_tm ? dtm : dtm + dD2 / (2.0 * rr * g.a));
        }
    }
    /* scales: do'/ds_k = -(1/s_k) o'_k e_k, dd'/ds_k = -(1/s_k) d'_k e_k */
    for (int k = 0; k < 3; ++k) {
        double dD2 = 2.0 * g.p[k] * (-g.op[k] / s[k]) - 2.0 * g.tau * g.p[k] * (-g.dp[k] / s[k]);
        v[7 + k] = dLdD2 * dD2;
        if (dLdt != 0.0) {
            const double dop_k = -g.op[k] / s[k], ddp_k = -g.dp[k] / s[k];
            const double da = 2.0 * g.dp[k] * ddp_k;
            const double db = dop_k * g.dp[k] + g.op[k] * ddp_k;
            const double dtm = -db / g.a + g.tau * da / g.a;
            const double dt1 = dtm + dD2 / (2.0 * rr * g.a) + (Q - g.D2) * da / (2.0 * rr * g.a * g.a);
            v[7 + k] += dLdt * (use_tm ? dtm : dt1);
        }
    }
    /* quaternion: do'/dq_x = S^-1 (dR/dq_x)^T (o - m), dd'/dq_x = S^-1 (dR/dq_x)^T d */
    double dR[4][9];
    quat_drot(q, dR);
    for (int x = 0; x < 4; ++x) {
        double dop[3], ddp[3];
        for (int k = 0; k < 3; ++k) {
            /* row k of (dR)^T is column k of dR */
            double ro = dR[x][k] * om[0] + dR[x][3 + k] * om[1] + dR[x][6 + k] * om[2];
            double rd = dR[x][k] * d[0] + dR[x][3 + k] * d[1] + dR[x][6 + k] * d[2];
            dop[k] = ro / s[k];
            ddp[k] = rd / s[k];
        }
        double dD2 = 2.0 * (g.p[0] * dop[0] + g.p[1] * dop[1] + g.p[2] * dop[2]) -
                     2.0 * g.tau * (g.p[0] * ddp[0] + g.p[1] * ddp[1] + g.p[2] * ddp[2]);
        v[3 + x] = dLdD2 * dD2;
        if (dLdt != 0.0) {
            const double da = 2.0 * (g.dp[0] * ddp[0] + g.dp[1] * ddp[1] + g.dp[2] * ddp[2]);
            const double db = (dop[0] * g.dp[0] + dop[1] * g.dp[1] + dop[2] * g.dp[2]) +
                              (g.op[0] * ddp[0] + g.op[1] * ddp[1] + g.op[2] * ddp[2]);
            const double dtm = -db / g.a + g.tau * da / g.a;
            const double dt1 = dtm + dD2 / (2.0 * rr * g.a) + (Q - g.D2) * da / (2.0 * rr * g.a * g.a);
            v[3 + x] += dLdt * (use_tm ? dtm : dt1);
        }
    }
}

/* Gradient of one ray's outputs (rgb, alpha) w.r.t. the parameters of its composited hits.
 * App. A.3: dI/dc_i = alpha_i T_i, dI/d(box) = dI/dalpha_i dalpha_i/d(box).
 * dI/dalpha_i is evaluated division-free, back to front: with U_n = background and
 * U_{i-1} = alpha_i c_i + (1 - alpha_i) U_i (the colour seen behind hit i),
 * dI/dalpha_i = T_i (c_i - U_i); this equals App. A.4/A.5's recurrence (checked by the tests).
 * For the alpha output use c = 1 and background 0.  Then App. A.6:
 * dalpha/dopacity = exp(-D2/2), dalpha/dD2 = -alpha/2,
 * dD2/d(box) = 2 <p, do'/d(box)> - 2 tau <p, dd'/d(box)>. */
static void ray_gradient(or_job* J, const double o[3], const double d[3], const or_hit* hits,
                         int nh, const double* alpha, const double* T, const double* gc,
                         double ga, double gd, const double* S_over) {
    const double* bg = J->prm->bg;
    const double Q = J->prm->Q;
    double U[3] = {bg[0], bg[1], bg[2]};
    double UA = 0.0, UD = 0.0; /* alpha and depth seen behind hit i (background depth 0) */
    for (int h = nh - 1; h >= 0; --h) {
        const int64_t i = hits[h].idx;
        const double* c = J->rgb + 3 * i;
        const double a = alpha[h], Ti = T[h];
        double v[14];
        memset(v, 0, sizeof(v));
        /* colour */
        for (int ch = 0; ch < 3; ++ch) v[11 + ch] = gc[ch] * Ti * a;
        /* dL/dalpha; depth is composited like a colour channel with value t_key */
        const double tk = hits[h].t;
        /* eps2 estimator: the last composited hit sees the phase-2 colour / alpha behind it */
        const int over = S_over && h == nh - 1;
        const double* Ub = over ? S_over : U;
        const double UAb = over ? S_over[3] : UA;
        double dLda = ga * Ti * (1.0 - UAb) + gd * Ti * (tk - UD);
        for (int ch = 0; ch < 3; ++ch) dLda += gc[ch] * Ti * (c[ch] - Ub[ch]);
        for (int ch = 0; ch < 3; ++ch) U[ch] = a * c[ch] + (1.0 - a) * U[ch];
        UA = a + (1.0 - a) * UA;
        UD = a * tk + (1.0 - a) * UD;
        const double dLdt = gd * Ti * a; /* depth = sum w_i t_key_i, w_i = T_i alpha_i */
        param_chain(J, o, d, i, a, dLda, dLdt, v);
        push_contrib(J, i, v);
    }
}

/* Front-to-back compositing of a sorted hit list (Eq. 3) with the eps1 cut applied after
 * the colour update and at most k_max hits (Sec. 3).  `flip_eps1_at` >= 0 inverts the eps1
 * decision at that composited position (used only to evaluate ambiguity alternatives). */
typedef struct {
    double C[3], depth, T;
    int64_t count;
    int stopped;
} or_comp;

static void composite(const or_job* J, const or_hit* hits, int64_t nh, int64_t flip_eps1_at,
                      double* alpha, double* T, or_comp* out) {
    const or_params* P = J->prm;
    double C[3] = {0, 0, 0}, depth = 0.0, Tr = 1.0;
    int64_t count = 0;
    int stopped = 0;
    for (int64_t h = 0; h < nh; ++h) {
        if (count >= P->k_max) {
            stopped = 1;
            break;
        }
        const int64_t i = hits[h].idx;
        const double al = J->opac[i] * exp(-0.5 * hits[h].D2); /* Prop. 2 */
        const double w = Tr * al;
        for (int ch = 0; ch < 3; ++ch) C[ch] += w * J->rgb[3 * i + ch];
        depth += w * hits[h].t;
        if (alpha) alpha[count] = al;
        if (T) T[count] = Tr;
        Tr *= (1.0 - al);
        count++;
        int stop = Tr < P->eps1;
        if (h == flip_eps1_at) stop = !stop;
        if (stop) {
            stopped = 1;
            break;
        }
    }
    for (int ch = 0; ch < 3; ++ch) out->C[ch] = C[ch] + Tr * P->bg[ch];
    out->depth = depth;
    out->T = Tr;
    out->count = count;
    out->stopped = stopped;
}

static double comp_diff(const or_comp* a, const or_comp* b) {
    double m = fabs(a->T - b->T); /* alpha = 1 - T */
    for (int ch = 0; ch < 3; ++ch) m = fmax(m, fabs(a->C[ch] - b->C[ch]));
    return m;
}

static void* render_worker(void* arg) {
    or_job* J = (or_job*)arg;
    const or_params* P = J->prm;
    const double Q = P->Q;
    const size_t cap = (size_t)(J->n > 0 ? J->n : 1) + 1;
    or_hit* hits = (or_hit*)malloc(sizeof(or_hit) * cap);
    or_hit* alt = (or_hit*)malloc(sizeof(or_hit) * cap);
    double* alpha = (double*)malloc(sizeof(double) * cap);
    double* T = (double*)malloc(sizeof(double) * cap);
    or_hit* cand = (or_hit*)malloc(sizeof(or_hit) * cap);
    int* cand_kind = (int*)malloc(sizeof(int) * cap);
    if (!hits || !alt || !alpha || !T || !cand || !cand_kind) {
        J->failed = 1;
        free(hits); free(alt); free(alpha); free(T); free(cand); free(cand_kind);
        return NULL;
    }
    for (int64_t r = J->r0; r < J->r1; ++r) {
        const double* o = J->ray_o + 3 * r;
        const double* d = J->ray_d + 3 * r;
        int64_t nh = 0, nc = 0;
        int32_t mask = 0;
        /* 1. every Gaussian: hit test (Prop. 1); candidates for ambiguous decisions */
        for (int64_t i = 0; i < J->n; ++i) {
            or_geom g;
            ray_gauss(o, d, J->means + 3 * i, J->M + 9 * i, Q, &g);
            const int inside = g.D2 <= Q;
            const int is_hit = inside && g.t1 >= P->t_near;
            if (is_hit) {
                hits[nh].t = P->sort_key == 1 ? -g.tau : g.t1;
                hits[nh].idx = i;
                hits[nh].D2 = g.D2;
                hits[nh].tol = P->sort_key == 1 ? g.mtol : g.ttol;
                nh++;
            }
            const int near_bd = fabs(Q - g.D2) < g.d2tol && g.t1 >= P->t_near;
            const int near_tn = inside && fabs(g.t1 - P->t_near) < OR_TIE_REL * fmax(1.0, fabs(g.t1));
            if (near_bd || near_tn) {
                cand[nc].t = P->sort_key == 1 ? -g.tau : (g.t1 > P->t_near ? g.t1 : P->t_near);
                cand[nc].idx = i;
                cand[nc].D2 = g.D2;
                cand[nc].tol = P->sort_key == 1 ? g.mtol : g.ttol;
                cand_kind[nc] = (near_bd ? OR_AMB_BOUNDARY : 0) | (near_tn ? OR_AMB_TNEAR : 0);
                nc++;
            }
        }
        /* 2. order hits by (t1, index) */
        qsort(hits, (size_t)nh, sizeof(or_hit), hit_cmp);
        /* 3. composite */
        or_comp prim;
        composite(J, hits, nh, -1, alpha, T, &prim);
        const int64_t count = prim.count;
        /* 4. ambiguity: flags, and the effect of each alternative decision */
        const double t_stop = (prim.stopped && count > 0) ? hits[count - 1].t : INFINITY;
        double impact = 0.0;
        for (int64_t c = 0; c < nc; ++c) {
            if (!(cand[c].t <= t_stop + OR_TIE_REL * fmax(1.0, fabs(t_stop)))) continue;
            mask |= cand_kind[c];
            /* alternative: toggle this Gaussian's membership in the hit list */
            int64_t na = 0, found = 0;
            for (int64_t h = 0; h < nh; ++h) {
                if (hits[h].idx == cand[c].idx) {
                    found = 1;
                    continue;
                }
                alt[na++] = hits[h];
            }
            if (!found) {
                alt[na] = cand[c];
                alt[na].D2 = fmin(cand[c].D2, Q);
                na++;
                qsort(alt, (size_t)na, sizeof(or_hit), hit_cmp);
            }
            or_comp ac;
            composite(J, alt, na, -1, NULL, NULL, &ac);
            const double df = comp_diff(&prim, &ac);
            if (df > OR_IMPACT_TOL) mask |= OR_IMP_BOUNDARY;
            impact = fmax(impact, df);
        }
        {
            const int64_t last = (count < nh) ? count : nh - 1; /* include the pair across the stop */
            for (int64_t h = 0; h + 1 <= last && h + 1 < nh; ++h) {
                const double tt = hits[h + 1].t;
                if (fabs(tt - hits[h].t) < hits[h].tol + hits[h + 1].tol + OR_T_QUANTUM * ulp32(tt)) {
                    mask |= OR_AMB_TIE;
                    memcpy(alt, hits, sizeof(or_hit) * (size_t)nh);
                    alt[h] = hits[h + 1];
                    alt[h + 1] = hits[h];
                    or_comp ac;
                    composite(J, alt, nh, -1, NULL, NULL, &ac);
                    const double df = comp_diff(&prim, &ac);
                    if (df > OR_IMPACT_TOL) mask |= OR_IMP_TIE;
                    impact = fmax(impact, df);
                }
            }
        }
        for (int64_t h = 0; h < count; ++h) {
            const double Tafter = T[h] * (1.0 - alpha[h]);
            if (fabs(Tafter - P->eps1) < 1e-4 * P->eps1) {
                mask |= OR_AMB_EPS1;
                or_comp ac;
                composite(J, hits, nh, h, NULL, NULL, &ac);
                const double df = comp_diff(&prim, &ac);
                if (df > OR_IMPACT_TOL) mask |= OR_IMP_EPS1;
                impact = fmax(impact, df);
            }
        }
        if (impact > OR_IMPACT_TOL) mask |= OR_AMB_IMPACT;
        /* 4b. eps2 estimator: phase 2 after an eps1 stop (Sec. 3) */
        double S[4];
        int use_S = 0;
        if (P->grad_mode == 1 && count > 0 && prim.T < P->eps1) {
            double T2 = 1.0;
            S[0] = S[1] = S[2] = 0.0;
            for (int64_t h = count; h < nh; ++h) {
                const int64_t i = hits[h].idx;
                const double al = J->opac[i] * exp(-0.5 * hits[h].D2);
                for (int ch = 0; ch < 3; ++ch) S[ch] += T2 * al * J->rgb[3 * i + ch];
                T2 *= (1.0 - al);
                if (fabs(T2 - P->eps2) < 1e-4 * P->eps2) mask |= OR_AMB_EPS2;
                if (T2 < P->eps2) break;
            }
            for (int ch = 0; ch < 3; ++ch) S[ch] += T2 * P->bg[ch];
            S[3] = 1.0 - T2;
            use_S = 1;
        }
        for (int ch = 0; ch < 3; ++ch) J->out_rgb[3 * r + ch] = prim.C[ch];
        J->out_alpha[r] = 1.0 - prim.T;
        J->out_depth[r] = prim.depth;
        J->out_T[r] = prim.T;
        J->out_nhits[r] = (int32_t)count;
        J->out_mask[r] = mask;
        /* 5. optional gradient */
        if (J->dl_rgb) {
            const double* gc = J->dl_rgb + 3 * r;
            const double ga = J->dl_alpha ? J->dl_alpha[r] : 0.0;
            const double gd = J->dl_depth ? J->dl_depth[r] : 0.0;
            ray_gradient(J, o, d, hits, (int)count, alpha, T, gc, ga, gd, use_S ? S : NULL);
        }
    }
    free(hits);
    free(alt);
    free(alpha);
    free(T);
    free(cand);
    free(cand_kind);
    return NULL;
}

/*
 * Render n_rays rays (ray_o/ray_d, 3 doubles each) against n Gaussians (FP64 parameters;
 * quats (w,x,y,z) unnormalised, scales physical > 0, opacities in (0,1)).
 * Outputs per ray: rgb[3], alpha, depth, T_final, n_hits, ambiguity mask.
 * If dl_rgb != NULL, the gradients of
 *   sum_r <dl_rgb[r], rgb[r]> + dl_alpha[r] alpha[r] + dl_depth[r] depth[r]
 * (dl_alpha, dl_depth may be NULL) are ADDED into g_means[3n], g_quats[4n], g_scales[3n],
 * g_opac[n], g_rgb[3n].
 * Returns 0 on success, -1 on allocation failure.
 */
int or_render(int64_t n, const double* means, const double* quats, const double* scales,
              const double* opac, const double* rgb, int64_t n_rays, const double* ray_o,
              const double* ray_d, const or_params* prm, double* out_rgb, double* out_alpha,
              double* out_depth, double* out_T, int32_t* out_nhits, int32_t* out_mask,
              const double* dl_rgb, const double* dl_alpha, const double* dl_depth, double* g_means,
              double* g_quats,
              double* g_scales, double* g_opac, double* g_rgb, int32_t nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (n_rays < nthreads) nthreads = (int32_t)(n_rays > 0 ? n_rays : 1);
    double* M = (double*)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
    or_job* jobs = (or_job*)calloc((size_t)nthreads, sizeof(or_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!M || !jobs || !th) {
        free(M); free(jobs); free(th);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) whitening(quats + 4 * i, scales + 3 * i, M + 9 * i);
    int rc = 0;
    for (int t = 0; t < nthreads; ++t) {
        or_job* J = &jobs[t];
        J->n = n; J->means = means; J->quats = quats; J->scales = scales; J->opac = opac;
        J->rgb = rgb; J->M = M; J->n_rays = n_rays; J->ray_o = ray_o; J->ray_d = ray_d;
        J->prm = prm; J->out_rgb = out_rgb; J->out_alpha = out_alpha; J->out_depth = out_depth;
        J->out_T = out_T; J->out_nhits = out_nhits; J->out_mask = out_mask;
        J->dl_rgb = dl_rgb; J->dl_alpha = dl_alpha; J->dl_depth = dl_depth;
        J->r0 = n_rays * t / nthreads;
        J->r1 = n_rays * (t + 1) / nthreads;
    }
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, render_worker, &jobs[t]) != 0) jobs[t].failed = 2;
    render_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t)
        if (jobs[t].failed != 2) pthread_join(th[t], NULL);
    /* merge gradient contributions in ray order (deterministic) */
    for (int t = 0; t < nthreads; ++t) {
        or_job* J = &jobs[t];
        if (J->failed) rc = -1;
        for (int64_t c = 0; c < J->n_contrib; ++c) {
            const int64_t i = J->contrib[c].idx;
            const double* v = J->contrib[c].v;
            for (int k = 0; k < 3; ++k) g_means[3 * i + k] += v[k];
            for (int k = 0; k < 4; ++k) g_quats[4 * i + k] += v[3 + k];
            for (int k = 0; k < 3; ++k) g_scales[3 * i + k] += v[7 + k];
            g_opac[i] += v[10];
            for (int k = 0; k < 3; ++k) g_rgb[3 * i + k] += v[11 + k];
        }
        free(J->contrib);
    }
    free(M);
    free(jobs);
    free(th);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Acceleration-structure references (no paper counterpart: the plain definitions the    */
/* device LBVH must reproduce bit-exactly).                                               */
/* ------------------------------------------------------------------------------------ */

/* Morton codes: lo/hi = min/max of the means per axis; ext = hi - lo (0 -> 1);
 * u = (m - lo) / ext in FP32 (one rounded subtraction, one rounded division);
 * cell = clamp(floor(u * 2^b), 0, 2^b - 1); the code interleaves x (high) y z (low) from the
 * most significant cell bit down.
 *   bits = 10: 30-bit code;  bits = 21: 63-bit code;
 *   bits = 20: extended 63-bit code with a 3-bit size class spliced in below the top four
 *   levels: [x y z interleave of cell bits 19..16][class][interleave of bits 15..0], where
 *   class = clamp(E(max_k s_k) - E(max_k ext_k) + 11, 0, 7) and E(x) is the biased binary
 *   exponent of the FP32 value x (its bits 30..23).  `scales` is needed only for bits = 20. */
static uint32_t f32_exponent(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    return (u >> 23) & 0xffu;
}

void or_morton(int64_t n, const float* means, const float* scales, int32_t bits, uint64_t* codes,
               float* lohi) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            const float v = means[3 * i + k];
            if (v < lo[k]) lo[k] = v;
            if (v > hi[k]) hi[k] = v;
        }
    float ext[3];
    for (int k = 0; k < 3; ++k) {
        ext[k] = hi[k] - lo[k];
        if (!(ext[k] > 0.0f)) ext[k] = 1.0f;
        if (lohi) {
            lohi[k] = lo[k];
            lohi[3 + k] = hi[k];
        }
    }
    const float ext_max = fmaxf(fmaxf(ext[0], ext[1]), ext[2]);
    const float scale = (float)(1u << bits);
    const uint32_t cmax = (1u << bits) - 1u;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t cell[3];
        for (int k = 0; k < 3; ++k) {
            const float u = (means[3 * i + k] - lo[k]) / ext[k];
            const float f = floorf(u * scale);
            cell[k] = f <= 0.0f ? 0u : (f >= (float)cmax ? cmax : (uint32_t)f);
        }
        uint64_t code = 0;
        if (bits == 20) {
            for (int b = 19; b >= 16; --b)
                for (int k = 0; k < 3; ++k) code = (code << 1) | ((cell[k] >> b) & 1u);
            const float smax = fmaxf(fmaxf(scales[3 * i], scales[3 * i + 1]), scales[3 * i + 2]);
            int c = (int)f32_exponent(smax) - (int)f32_exponent(ext_max) + 11;
            c = c < 0 ? 0 : (c > 7 ? 7 : c);
            code = (code << 3) | (uint64_t)c;
            for (int b = 15; b >= 0; --b)
                for (int k = 0; k < 3; ++k) code = (code << 1) | ((cell[k] >> b) & 1u);
        } else {
            for (int b = bits - 1; b >= 0; --b)
                for (int k = 0; k < 3; ++k) code = (code << 1) | ((cell[k] >> b) & 1u);
        }
        codes[i] = code;
    }
}

typedef struct {
    uint64_t code;
    uint32_t idx;
} or_key;

static int key_cmp(const void* x, const void* y) {
    const or_key* a = (const or_key*)x;
    const or_key* b = (const or_key*)y;
    if (a->code != b->code) return a->code < b->code ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

/* Stable order of the codes: perm[j] = index of the j-th smallest (code, index). */
int or_sort_perm(int64_t n, const uint64_t* codes, uint32_t* perm, uint64_t* sorted_codes) {
    or_key* k = (or_key*)malloc(sizeof(or_key) * (size_t)(n > 0 ? n : 1));
    if (!k) return -1;
    for (int64_t i = 0; i < n; ++i) {
        k[i].code = codes[i];
        k[i].idx = (uint32_t)i;
    }
    qsort(k, (size_t)n, sizeof(or_key), key_cmp);
    for (int64_t i = 0; i < n; ++i) {
        perm[i] = k[i].idx;
        if (sorted_codes) sorted_codes[i] = k[i].code;
    }
    free(k);
    return 0;
}

/* Binary radix tree over the sorted keys made unique as (code, position), built top down by
 * its definition: a node covers a range [first, last] of sorted positions; it splits after
 * the last position whose key has a 0 at the highest bit where key[first] and key[last]
 * differ.  Internal nodes are numbered as in Karras 2012: the root is 0, a left child
 * range [first, split] is internal node `split`, a right child range [split+1, last] is
 * internal node `split + 1`; single positions are leaves.  Outputs, for internal node
 * i in [0, n-2]: first[i], last[i], split[i].  Iterative (explicit stack), O(n log n). */
static int highest_diff_bit(uint64_t ca, uint32_t ia, uint64_t cb, uint32_t ib) {
    /* bit index in the 96-bit key (code:64 | position:32); larger = more significant */
    if (ca != cb) return 32 + 63 - __builtin_clzll(ca ^ cb);
    return 31 - __builtin_clz(ia ^ ib);
}

static int key_bit(uint64_t c, uint32_t i, int bit) {
    return bit >= 32 ? (int)((c >> (bit - 32)) & 1u) : (int)((i >> bit) & 1u);
}

int or_radix_tree(int64_t n, const uint64_t* sorted_codes, int32_t* first, int32_t* last,
                  int32_t* split) {
    if (n < 2) return 0;
    int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)n);
    if (!stack) return -1;
    int64_t sp = 0;
    stack[sp++] = 0; /* node */
    stack[sp++] = 0; /* first */
    stack[sp++] = n - 1;
    while (sp > 0) {
        const int64_t l = stack[--sp], f = stack[--sp], node = stack[--sp];
        const int bit = highest_diff_bit(sorted_codes[f], (uint32_t)f, sorted_codes[l], (uint32_t)l);
        int64_t s = f;
        while (s + 1 <= l && key_bit(sorted_codes[s + 1], (uint32_t)(s + 1), bit) == 0) ++s;
        first[node] = (int32_t)f;
        last[node] = (int32_t)l;
        split[node] = (int32_t)s;
        if (s > f) {
            stack[sp++] = s;
            stack[sp++] = f;
            stack[sp++] = s;
        }
        if (s + 1 < l) {
            stack[sp++] = s + 1;
            stack[sp++] = s + 1;
            stack[sp++] = l;
        }
    }
    free(stack);
    return 0;
}

/* Q = F^-1_{chi^2(3)}(p) by bisection on the closed-form CDF
 * F(x) = erf(sqrt(x/2)) - sqrt(2x/pi) exp(-x/2)  (chi-square, three degrees of freedom). */
double or_chi2_3_quantile(double p) {
    double lo = 0.0, hi = 200.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        const double F = erf(sqrt(0.5 * mid)) - sqrt(2.0 * mid / M_PI) * exp(-0.5 * mid);
        if (F < p) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------------------ */
/* Scenes with triangles: a mirror mesh, diffuse surfaces, one point light (the paper's    */
/* mesh / mirror / shadow demonstrations, Sec. 1 and Fig. 1; the paper gives no algorithm, */
/* so the rules below are this renderer's own and stated in full).                        */
/*                                                                                        */
/*   A ray runs in segments.  In each, Gaussians whose entry t1 lies in [t_min, t_tri)    */
/*   are composited in (t1, index) order with the eps1 cut and k_max (counted over the    */
/*   whole ray), t_tri being the nearest triangle.  Then, unless the ray was cut:         */
/*     - no triangle: the environment term is the background;                              */
/*     - diffuse triangle (albedo a): the term is a * T_s, T_s the transmittance of a     */
/*       shadow ray from the hit point to the light: the product of (1 - alpha) over the   */
/*       Gaussians it hits (entry in [eps_off, distance)); 0 if a triangle blocks it or    */
/*       the product falls below eps1 (the shadow ray's own cut, as for camera rays);     */
/*     - mirror triangle: the ray reflects and continues (at most max_bounces times; past  */
/*       that the term is 0).                                                              */
/*   A ray cut by eps1 or k_max takes the term of the segment it stopped in (a mirror      */
/*   gives 0).  RGB = sum of composited colours + T_final * term, alpha = 1 - T_final,     */
/*   depth = sum of w_i t1_i over the first segment.                                       */
/*   Triangle hits, reflected rays and shadow rays follow fixed FP32 operation sequences   */
/*   (as camera rays do) so that both implementations take the same surface decisions;     */
/*   the Gaussian arithmetic along those rays is FP64.  The gradient is the exact          */
/*   derivative w.r.t. the Gaussian parameters (the mesh and the light are fixed).         */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int64_t n_tri;
    const float* verts;    /* 9 per triangle: v0, v1, v2 */
    const int32_t* mat;    /* 0: mirror, 1: diffuse */
    const float* albedo;   /* 3 per triangle (diffuse) */
    float light[3];
    int32_t max_bounces;
    float eps_off;         /* start of reflected and shadow rays along their direction */
} or_scene;

#define OR_AMB_SURFACE 512 /* a triangle decision within FP32 rounding (edge, tie, t_min) */

/* Moller-Trumbore in a fixed FP32 sequence; returns 1 and (t, u, v) when tmin < t < tmax. */
static int tri_hit_f32(const float o[3], const float d[3], const float* v, float tmin, float tmax, float* t_out,
                       float* u_out, float* v_out) {
    const float e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
    const float e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
    const float p[3] = {d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2], d[0] * e2[1] - d[1] * e2[0]};
    const float det = (e1[0] * p[0] + e1[1] * p[1]) + e1[2] * p[2];
    if (fabsf(det) < 1e-12f) return 0;
    const float inv = 1.0f / det;
    const float s[3] = {o[0] - v[0], o[1] - v[1], o[2] - v[2]};
    const float u = ((s[0] * p[0] + s[1] * p[1]) + s[2] * p[2]) * inv;
    if (u < 0.0f || u > 1.0f) return 0;
    const float q[3] = {s[1] * e1[2] - s[2] * e1[1], s[2] * e1[0] - s[0] * e1[2], s[0] * e1[1] - s[1] * e1[0]};
    const float w = ((d[0] * q[0] + d[1] * q[1]) + d[2] * q[2]) * inv;
    if (w < 0.0f || u + w > 1.0f) return 0;
    const float t = ((e2[0] * q[0] + e2[1] * q[1]) + e2[2] * q[2]) * inv;
    if (!(t > tmin && t < tmax)) return 0;
    *t_out = t;
    *u_out = u;
    *v_out = w;
    return 1;
}

/* nearest triangle (smallest t, then smallest index) in (tmin, tmax); -1 if none */
static int64_t nearest_tri(const or_scene* S, const float o[3], const float d[3], float tmin, float tmax, float* t,
                           int32_t* mask) {
    int64_t best = -1;
    float bt = tmax, bu = 0.f, bv = 0.f;
    for (int64_t k = 0; k < S->n_tri; ++k) {
        float tt, uu, vv;
        if (tri_hit_f32(o, d, S->verts + 9 * k, tmin, bt, &tt, &uu, &vv) && (tt < bt || best < 0)) {
            best = k;
            bt = tt;
            bu = uu;
            bv = vv;
        }
    }
    if (best >= 0) {
        const float band = 1e-5f;
        if (bu < band || bv < band || 1.0f - bu - bv < band || bt < tmin * 1.001f + 1e-6f) *mask |= OR_AMB_SURFACE;
        /* a second triangle at nearly the same t */
        for (int64_t k = 0; k < S->n_tri; ++k) {
            float tt, uu, vv;
            if (k != best && tri_hit_f32(o, d, S->verts + 9 * k, tmin, tmax, &tt, &uu, &vv) &&
                fabsf(tt - bt) < 1e-5f * fmaxf(1.0f, bt))
                *mask |= OR_AMB_SURFACE;
        }
    }
    *t = bt;
    return best;
}

/* fixed FP32 sequences: hit point, unit normal, reflected direction, shadow ray */
static void reflect_f32(const float o[3], const float d[3], float t, const float* v, float P[3], float dr[3]) {
    const float e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
    const float e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
    float n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const float nl = sqrtf((n[0] * n[0] + n[1] * n[1]) + n[2] * n[2]);
    for (int k = 0; k < 3; ++k) n[k] = n[k] / nl;
    const float dn = (d[0] * n[0] + d[1] * n[1]) + d[2] * n[2];
    const float k2 = 2.0f * dn;
    float r[3];
    for (int k = 0; k < 3; ++k) {
        P[k] = o[k] + t * d[k];
        r[k] = d[k] - k2 * n[k];
    }
    const float rl = sqrtf((r[0] * r[0] + r[1] * r[1]) + r[2] * r[2]);
    for (int k = 0; k < 3; ++k) dr[k] = r[k] / rl;
}

static void shadow_ray_f32(const float P[3], const float L[3], float dir[3], float* dist) {
    const float w[3] = {L[0] - P[0], L[1] - P[1], L[2] - P[2]};
    const float dl = sqrtf((w[0] * w[0] + w[1] * w[1]) + w[2] * w[2]);
    for (int k = 0; k < 3; ++k) dir[k] = w[k] / dl;
    *dist = dl;
}

typedef struct {
    int64_t idx;
    int32_t seg;
    double t, D2;
    double tol; /* uncertainty of an FP32 evaluation of t (TIE band) */
} or_shit;

static int shit_cmp(const void* x, const void* y) {
    const or_shit* a = (const or_shit*)x;
    const or_shit* b = (const or_shit*)y;
    if (a->t < b->t) return -1;
    if (a->t > b->t) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx ? 1 : 0);
}

/* Gaussians hit by the ray (o, d) with entry in [tmin, tmax), appended to `out`; flags the
 * boundary / t_min / t_max decisions that FP32 may take differently */
static int64_t gather_hits(const or_job* J, const float of[3], const float df[3], double tmin, double tmax, int32_t seg,
                           or_shit* out, int32_t* mask) {
    const double o[3] = {of[0], of[1], of[2]}, d[3] = {df[0], df[1], df[2]};
    const double Q = J->prm->Q;
    int64_t nh = 0;
    for (int64_t i = 0; i < J->n; ++i) {
        or_geom g;
        ray_gauss(o, d, J->means + 3 * i, J->M + 9 * i, Q, &g);
        const double band = OR_TIE_REL * fmax(1.0, fabs(g.t1));
        if (fabs(Q - g.D2) < g.d2tol && g.t1 >= tmin - band && g.t1 < tmax + band) *mask |= OR_AMB_BOUNDARY;
        if (g.D2 > Q) continue;
        if (fabs(g.t1 - tmin) < band || (tmax < INFINITY && fabs(g.t1 - tmax) < band)) *mask |= OR_AMB_TNEAR;
        if (g.t1 >= tmin && g.t1 < tmax) {
            out[nh].idx = i;
            out[nh].seg = seg;
            out[nh].t = g.t1;
            out[nh].D2 = g.D2;
            out[nh].tol = g.ttol;
            nh++;
        }
    }
    qsort(out, (size_t)nh, sizeof(or_shit), shit_cmp);
    return nh;
}

int or_render_scene(int64_t n, const double* means, const double* quats, const double* scales, const double* opac,
                    const double* rgb, const or_scene* S, int64_t n_rays, const float* ray_o, const float* ray_d,
                    const or_params* prm, double* out_rgb, double* out_alpha, double* out_depth,
                    int32_t* out_nhits, int32_t* out_mask, const double* dl_rgb, const double* dl_alpha,
                    const double* dl_depth, double* g_means, double* g_quats, double* g_scales, double* g_opac,
                    double* g_rgb) {
    double* M = (double*)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
    const size_t cap = (size_t)(n > 0 ? n : 1) + 1;
    or_shit* seg_hits = (or_shit*)malloc(sizeof(or_shit) * cap);
    or_shit* comp = (or_shit*)malloc(sizeof(or_shit) * cap * 4);
    or_shit* sh = (or_shit*)malloc(sizeof(or_shit) * cap);
    double* alpha = (double*)malloc(sizeof(double) * cap * 4);
    double* Tb = (double*)malloc(sizeof(double) * cap * 4);
    if (!M || !seg_hits || !comp || !sh || !alpha || !Tb) {
        free(M); free(seg_hits); free(comp); free(sh); free(alpha); free(Tb);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) whitening(quats + 4 * i, scales + 3 * i, M + 9 * i);
    or_job J;
    memset(&J, 0, sizeof(J));
    J.n = n; J.means = means; J.quats = quats; J.scales = scales; J.opac = opac; J.rgb = rgb; J.M = M;
    J.prm = prm;
    const or_params* P = prm;
    int rc = 0;
    for (int64_t r = 0; r < n_rays; ++r) {
        float so[4][3], sd[4][3], stmin[4];
        int32_t mask = 0;
        for (int k = 0; k < 3; ++k) {
            so[0][k] = ray_o[3 * r + k];
            sd[0][k] = ray_d[3 * r + k];
        }
        stmin[0] = (float)P->t_near;
        double C[3] = {0, 0, 0}, depth = 0.0, Tr = 1.0, E[3] = {0, 0, 0};
        int64_t count = 0, nsh = 0;
        int cut = 0, shadow_used = 0;
        float sdir[3] = {0, 0, 0}, sP[3] = {0, 0, 0}, sdist = 0.f, alb[3] = {0, 0, 0};
        for (int seg = 0; seg <= S->max_bounces; ++seg) {
            float t_tri = INFINITY;
            const int64_t tri = nearest_tri(S, so[seg], sd[seg], stmin[seg], INFINITY, &t_tri, &mask);
            const int64_t nh = gather_hits(&J, so[seg], sd[seg], stmin[seg], tri >= 0 ? (double)t_tri : INFINITY, seg,
                                           seg_hits, &mask);
            for (int64_t h = 0; h < nh && !cut; ++h) {
                if (count >= P->k_max) {
                    cut = 1;
                    break;
                }
                const int64_t i = seg_hits[h].idx;
                const double al = opac[i] * exp(-0.5 * seg_hits[h].D2);
                const double w = Tr * al;
                for (int ch = 0; ch < 3; ++ch) C[ch] += w * rgb[3 * i + ch];
                if (seg == 0) depth += w * seg_hits[h].t;
                comp[count] = seg_hits[h];
                alpha[count] = al;
                Tb[count] = Tr;
                Tr *= (1.0 - al);
                if (h + 1 < nh && fabs(seg_hits[h + 1].t - seg_hits[h].t) <
                                      seg_hits[h].tol + seg_hits[h + 1].tol + OR_T_QUANTUM * ulp32(seg_hits[h].t))
                    mask |= OR_AMB_TIE;
                if (fabs(Tr - P->eps1) < 1e-4 * P->eps1) mask |= OR_AMB_EPS1;
                count++;
                if (Tr < P->eps1) cut = 1;
            }
            /* the environment term of this segment */
            if (tri < 0) {
                for (int ch = 0; ch < 3; ++ch) E[ch] = P->bg[ch];
                break;
            }
            if (S->mat[tri] == 1) {
                float dummy[3];
                reflect_f32(so[seg], sd[seg], t_tri, S->verts + 9 * tri, sP, dummy);
                shadow_ray_f32(sP, S->light, sdir, &sdist);
                float t_occ = 0.f;
                const int64_t occ = nearest_tri(S, sP, sdir, S->eps_off, sdist, &t_occ, &mask);
                double Ts = 0.0;
                if (occ < 0) {
                    nsh = gather_hits(&J, sP, sdir, S->eps_off, sdist, -1, sh, &mask);
                    Ts = 1.0;
                    for (int64_t h = 0; h < nsh; ++h) Ts *= 1.0 - opac[sh[h].idx] * exp(-0.5 * sh[h].D2);
                    if (fabs(Ts - P->eps1) < 1e-4 * P->eps1) mask |= OR_AMB_EPS1;
                    if (Ts < P->eps1) Ts = 0.0;  /* opaque: the shadow ray's eps1 cut */
                    shadow_used = Ts > 0.0;
                }
                for (int ch = 0; ch < 3; ++ch) {
                    alb[ch] = S->albedo[3 * tri + ch];
                    E[ch] = alb[ch] * Ts;
                }
                break;
            }
            /* mirror */
            if (cut || seg == S->max_bounces) break;
            reflect_f32(so[seg], sd[seg], t_tri, S->verts + 9 * tri, so[seg + 1], sd[seg + 1]);
            stmin[seg + 1] = S->eps_off;
        }
        for (int ch = 0; ch < 3; ++ch) out_rgb[3 * r + ch] = C[ch] + Tr * E[ch];
        out_alpha[r] = 1.0 - Tr;
        out_depth[r] = depth;
        out_nhits[r] = (int32_t)count;
        out_mask[r] = mask;
        if (!dl_rgb) continue;
        const double* gc = dl_rgb + 3 * r;
        const double ga = dl_alpha ? dl_alpha[r] : 0.0;
        const double gd = dl_depth ? dl_depth[r] : 0.0;
        /* composited hits, back to front over the segments: U starts at the environment term */
        double U[3] = {E[0], E[1], E[2]}, UA = 0.0, UD = 0.0;
        for (int64_t h = count - 1; h >= 0; --h) {
            const int64_t i = comp[h].idx;
            const int s = comp[h].seg;
            const double* c = rgb + 3 * i;
            const double a = alpha[h], Ti = Tb[h];
            const double tk = s == 0 ? comp[h].t : 0.0;  /* depth counts the first segment */
            double dLda = ga * Ti * (1.0 - UA) + gd * Ti * (tk - UD);
            for (int ch = 0; ch < 3; ++ch) dLda += gc[ch] * Ti * (c[ch] - U[ch]);
            for (int ch = 0; ch < 3; ++ch) U[ch] = a * c[ch] + (1.0 - a) * U[ch];
            UA = a + (1.0 - a) * UA;
            UD = a * tk + (1.0 - a) * UD;
            double v[14];
            memset(v, 0, sizeof(v));
            for (int ch = 0; ch < 3; ++ch) v[11 + ch] = gc[ch] * Ti * a;
            const double od[3] = {so[s][0], so[s][1], so[s][2]}, dd[3] = {sd[s][0], sd[s][1], sd[s][2]};
            param_chain(&J, od, dd, i, a, dLda, s == 0 ? gd * Ti * a : 0.0, v);
            push_contrib(&J, i, v);
        }
        /* shadow hits: d(T_final a T_s)/dalpha_j = -T_final a prod_{k != j} (1 - alpha_k) */
        if (shadow_used && nsh > 0) {
            const double ga_s = (gc[0] * alb[0] + gc[1] * alb[1] + gc[2] * alb[2]) * Tr;
            for (int64_t h = 0; h < nsh; ++h) {
                double others = 1.0;
                for (int64_t k = 0; k < nsh; ++k)
                    if (k != h) others *= 1.0 - opac[sh[k].idx] * exp(-0.5 * sh[k].D2);
                const int64_t i = sh[h].idx;
                const double a = opac[i] * exp(-0.5 * sh[h].D2);
                double v[14];
                memset(v, 0, sizeof(v));
                const double od[3] = {sP[0], sP[1], sP[2]}, dd[3] = {sdir[0], sdir[1], sdir[2]};
                param_chain(&J, od, dd, i, a, -ga_s * others, 0.0, v);
                push_contrib(&J, i, v);
            }
        }
    }
    if (J.failed) rc = -1;
    for (int64_t c = 0; c < J.n_contrib; ++c) {
        const int64_t i = J.contrib[c].idx;
        const double* v = J.contrib[c].v;
        for (int k = 0; k < 3; ++k) g_means[3 * i + k] += v[k];
        for (int k = 0; k < 4; ++k) g_quats[4 * i + k] += v[3 + k];
        for (int k = 0; k < 3; ++k) g_scales[3 * i + k] += v[7 + k];
        g_opac[i] += v[10];
        for (int k = 0; k < 3; ++k) g_rgb[3 * i + k] += v[11 + k];
    }
    free(J.contrib);
    free(M); free(seg_hits); free(comp); free(sh); free(alpha); free(Tb);
    return rc;
}
