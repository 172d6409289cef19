/*
 * raysplats.h -- C ABI of the GB300 (sm_103a) RaySplats rendering path.
 *
 * The library renders images by tracing camera rays through a scene of 3D Gaussians held as
 * confidence ellipsoids with an opacity and an RGB colour, and computes the adjoint of that
 * render.  Paper: RaySplats (arXiv 2501.19196).  What each call computes:
 *   - the scene: G = {(N(m_i, Sigma_i), opacity_i, c_i)}, Sigma = R S S^T R^T    (Eq. 1, Eq. 2)
 *   - a ray hits Gaussian i when it meets the confidence ellipsoid
 *     (x - m)^T Sigma^-1 (x - m) = Q at an entry parameter t1 >= t_near          (Sec. 3, Prop. 1)
 *   - each hit contributes alpha_i = opacity_i * exp(-D_i^2 / 2), D_i^2 the squared
 *     Mahalanobis distance of the ray from m_i (the maximum response)           (Eq. 8, Prop. 2)
 *   - hits are composited front to back in (t1, id) order, C = sum c_i alpha_i T_i, T_i =
 *     prod_{j<i}(1 - alpha_j); the hit that brings T below eps1 is the last, and at most
 *     k_max hits are composited                                                 (Eq. 3, Sec. 3)
 *   - the backward pass is the exact derivative of that render                  (App. A.3-A.6)
 *
 * Conventions for every call:
 *   - All pointers marked "device" are CUDA device pointers on the current device; all sizes
 *     are element counts.  The caller owns every parameter, output and gradient buffer.
 *   - The library owns rs_accel and rs_fwd_state (opaque handles).  Passing a pointer to a
 *     NULL handle creates one; passing an existing handle reuses (and if needed grows) its
 *     device memory, so repeated calls with the same sizes allocate nothing (required for
 *     CUDA-graph capture).
 *   - Every call is stream ordered on `cuda_stream` (a cudaStream_t; NULL = legacy default
 *     stream) and asynchronous; nothing is synchronised except where stated.  Nothing throws
 *     across the ABI: each call returns an rs_status and records a message for
 *     rs_last_error() (per host thread).
 *   - Arguments are validated on the host before any launch (RS_ERR_INVALID_ARG).  Device-side
 *     consistency checks set an error word that rs_check_device() reports.
 */
#ifndef RAYSPLATS_H
#define RAYSPLATS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RS_ABI_VERSION 1

typedef int32_t rs_status;
enum {
    RS_OK = 0,
    RS_ERR_INVALID_ARG = -1, /* a NULL pointer, a bad size or an out-of-range parameter */
    RS_ERR_OOM = -2,         /* device or pinned-host allocation failed */
    RS_ERR_CUDA = -3,        /* a CUDA runtime call failed (message has the CUDA error) */
    RS_ERR_UNSUPPORTED = -4, /* valid request this build does not implement */
    RS_ERR_INTERNAL = -5,    /* a device-side consistency check failed */
    RS_ERR_TIMEOUT = -6      /* reserved: a bounded device wait gave up (no kernel waits today) */
};

/* Scene (Eq. 1, Eq. 2).  Structure of arrays, FP32, all device pointers, n >= 1:
 *   means[3n]      m_i
 *   quats[4n]      (w, x, y, z) rotation quaternion, need not be normalised (R uses
 *                  s = 2/|q|^2, App. A.6); must be non-zero
 *   scales[3n]     physical scales s_i > 0 (S = diag(s)); activations such as exp/sigmoid are
 *                  the caller's
 *   opacities[n]   physical opacity in [0, 1); the backward pass needs 1 - alpha > 0
 *   rgb[3n]        colour c_i */
typedef struct {
    int64_t n;
    const float* means;
    const float* quats;
    const float* scales;
    const float* opacities;
    const float* rgb;
} rs_gaussians;

/* Pinhole camera (host struct).  world = R_wc * cam + pos; camera axes x right, y down,
 * z forward.  Ray of pixel (u, v): direction normalise(R_wc * ((u + 0.5 - cx) / fx,
 * (v + 0.5 - cy) / fy, 1)) evaluated as a fixed FP32 operation sequence (no fused
 * multiply-add), origin pos.  width, height >= 1 and width * height < 2^31. */
typedef struct {
    float R_wc[9]; /* row major */
    float pos[3];
    float fx, fy, cx, cy;
    int32_t width, height;
} rs_camera;

/* Render parameters (Sec. 3).
 *   Q           squared Mahalanobis radius of the confidence ellipsoid, 0 < Q <= the accel's
 *               Q_box (Q = F^-1_chi2(3)(confidence); 11.3449 for 0.99)
 *   eps1        transmittance cut, >= 0
 *   t_near      smallest accepted entry parameter t1, >= 0 (units of the unit-length ray)
 *   background  added as T_final * background
 *   k_max       at most k_max composited hits per ray, >= 1 (INT32_MAX = unbounded)
 *   depth_mode  0: depth = sum_i w_i t_i (unnormalised), t_i the hit's sort key; other
 *               values unsupported
 *   sort_key    0: order hits by (t1, id), t1 the ellipsoid entry (Prop. 1); 1: by (t_m, id),
 *               t_m the ray parameter of the Gaussian's maximum response (Prop. 2, the chord
 *               midpoint); the hit test (D^2 <= Q, t1 >= t_near) is the same for both
 *   grad_mode   0: the adjoint is the exact derivative of the rendered outputs; 1: the paper's
 *               eps2 estimator (Sec. 3, Sec. 5): a ray cut by eps1 after hit i goes on
 *               collecting the hits behind i, without compositing them, until the product of
 *               their (1 - alpha) falls below eps2, and dL/dalpha_i uses the colour and alpha
 *               seen through them (plus the background) instead of the background alone; the
 *               image is the same in both modes (16 B more state per ray)
 *   eps2        the second threshold, > 0 (read when grad_mode is 1) */
typedef struct {
    float Q;
    float eps1;
    float t_near;
    float background[3];
    int32_t k_max;
    int32_t depth_mode;
    int32_t sort_key;
    int32_t grad_mode;
    float eps2;
} rs_render_params;

/* Frame outputs, device, cameras concatenated in order, each camera row major (y, x):
 *   rgb[3 * sum W*H], alpha[sum W*H], depth[sum W*H] (depth may be NULL). */
typedef struct {
    float* rgb;
    float* alpha;
    float* depth;
} rs_frame;

/* Upstream gradient (device, same layout as rs_frame): d_rgb required, d_alpha and d_depth
 * may be NULL.  The depth gradient moves opacities (through alpha) and the hits' sort keys
 * (through the geometry): the exact derivative of sum_i w_i t_i. */
typedef struct {
    const float* d_rgb;
    const float* d_alpha;
    const float* d_depth;
} rs_frame_grad;

/* Parameter gradients (device, same layout as rs_gaussians).  ACCUMULATED into (+=); the
 * caller zeroes them.  Any pointer may be NULL to skip that gradient. */
typedef struct {
    float* d_means;
    float* d_quats;
    float* d_scales;
    float* d_opacities;
    float* d_rgb;
} rs_gaussian_grads;

/* Tunables.  None changes a result of rs_render (tests check this), only speed.  In scenes with
 * triangles a shadow ray multiplies its (1 - alpha) factors in traversal order, so tunables can
 * change the last bits of lit colours there.
 *   tile_w, tile_h  ray tile handled by one warp; tile_w * tile_h == 32
 *   kbuf            per-ray k-buffer depth: 8, 16 or 32 (with traversal 2 and 32, the
 *                   forward keeps it in shared memory instead of registers)
 *   leaf_size       BVH leaf size 1..32 (used by rs_build_accel); a warp pre-tests a leaf
 *                   with one bounding sphere per lane
 *   morton_bits     10 (30-bit codes) or 21 (63-bit codes) bits per axis, or 20: extended
 *                   63-bit codes, 20 bits per axis plus a 3-bit size class (from the exponent
 *                   of the largest scale) below the top four levels
 *   persistent      0: one launch per camera; 1: one persistent launch over all cameras'
 *                   ray tiles through a device work queue
 *   block_warps     warps per CTA: 1..4
 *   traversal       0: each lane traverses its own ray (depth first); 1: the 32 rays of a
 *                   tile traverse as a warp packet (shared node sequence, per-ray state, depth
 *                   first); 2: warp packet in best-first order of box entry (a priority queue
 *                   distributed over the warp's registers); 3: as 2 over 4-wide nodes (each
 *                   binary node's grandchildren; rs_build_accel builds them when given 3)
 *   smem_nodes      0..512: the top BVH nodes (breadth first) that rs_build_accel stages for
 *                   the render kernels' shared memory (64 B each); 0 disables staging.  The
 *                   forward with its k-buffer in shared memory does not use them
 *   hit_list        0..4096: rs_render records the sorted ids of each ray's first hit_list
 *                   composited hits (4 B each, hit_list * 4 B per ray in the state), and the
 *                   adjoint replays every ray with at most hit_list hits from that list instead
 *                   of re-traversing the BVH (the paper's index buffer, Sec. 3 and 5); rays
 *                   with more hits re-traverse (none when k_max <= hit_list, the paper's
 *                   setting).  0: every ray re-traverses.  The adjoint follows the setting of
 *                   the rs_render it differentiates. */
typedef struct {
    int32_t tile_w, tile_h;
    int32_t kbuf;
    int32_t leaf_size;
    int32_t morton_bits;
    int32_t persistent;
    int32_t block_warps;
    int32_t traversal;
    int32_t smem_nodes;
    int32_t hit_list;
} rs_tune_params;

typedef struct rs_accel rs_accel;
typedef struct rs_fwd_state rs_fwd_state;

/* Counters of the instrumented render (rs_render_counted): per-call sums over all rays. */
typedef struct {
    uint64_t rays;             /* rays traced */
    uint64_t nodes_visited;    /* BVH nodes fetched (64 B each) */
    uint64_t gaussians_tested; /* ray / ellipsoid tests (48 B record each) */
    uint64_t hits_composited;  /* composited hits (16 B shade record each) */
    uint64_t rounds;           /* k-buffer traversal rounds */
    uint64_t hits_inserted;    /* candidates inserted into a k-buffer */
    uint64_t rays_retraced;    /* adjoint only: rays replayed by re-traversal (not from the list) */
    uint64_t hits_listed;      /* adjoint only: hits replayed from the hit list */
    uint64_t warp_node_fetches;    /* packet traversals: nodes fetched by whole warps; lane
                                      efficiency = nodes_visited / (32 * warp_node_fetches) */
    uint64_t warp_leaf_iterations; /* packet traversals: full-test iterations of whole warps
                                      (one per leaf Gaussian whose bounding sphere some lane's
                                      ray meets); lane efficiency = gaussians_tested / (32 * this) */
} rs_render_stats;

/* ABI version (RS_ABI_VERSION of the build). */
int32_t rs_abi_version(void);

/* Message of the last failed call on this host thread ("" if none). */
const char* rs_last_error(void);

/* Fill *out with the default tunables (8x4 tiles, kbuf 32, leaf 32, 63-bit codes,
 * persistent launch, 4 warps per CTA, best-first warp-packet traversal, 256 staged nodes,
 * hit lists of 256 ids per ray). */
rs_status rs_default_tune(rs_tune_params* out);

/* Build the acceleration structure of a scene (LBVH): per-Gaussian render records
 * (M = S^-1 R^T and the mean, opacity and colour) and conservative boxes of the confidence
 * ellipsoids |M (x - m)|^2 <= Q_box in Morton order, a 63- or 30-bit Morton sort, a Karras
 * binary radix tree with leaves of at most leaf_size Gaussians, and a bottom-up box refit.
 * Q_box > 0 bounds the Q of every rs_render that uses this accel.  *inout: NULL to create,
 * else reused.  The accel reads the scene at build time only; rebuild after the parameters
 * change.  On failure a newly created handle is freed (*inout stays NULL); a reused handle
 * stays valid but holds no build until a later call succeeds. */
rs_status rs_build_accel(const rs_gaussians* g, float Q_box, const rs_tune_params* tune,
                         rs_accel** inout, void* cuda_stream);

/* Render n_cams cameras (host array) of the scene `g` through `accel` (built from the same
 * scene).  Writes out->rgb / alpha / depth and, in *inout_state (NULL to create, else reused),
 * what the backward pass needs: per ray the final transmittance, the (t1, id) key of the
 * last composited hit and the hit count (16 B per ray), plus the cameras and parameters.
 * On failure a reused state holds no render (rs_render_backward rejects it). */
rs_status rs_render(const rs_gaussians* g, const rs_accel* accel, const rs_camera* cams,
                    int32_t n_cams, const rs_render_params* params, const rs_tune_params* tune,
                    rs_frame* out, rs_fwd_state** inout_state, void* cuda_stream);

/* rs_render plus per-call counters: *stats_device (device memory, 10 uint64, zeroed by the
 * caller) is incremented with the rs_render_stats fields.  Slower; for measurement only. */
rs_status rs_render_counted(const rs_gaussians* g, const rs_accel* accel, const rs_camera* cams,
                            int32_t n_cams, const rs_render_params* params,
                            const rs_tune_params* tune, rs_frame* out,
                            rs_fwd_state** inout_state, uint64_t* stats_device,
                            void* cuda_stream);

/* Adjoint of the last rs_render recorded in `state` (App. A.3-A.6): replays every ray back
 * to front (from its hit list, or by re-traversing `accel`; see hit_list), recovers the
 * transmittance from the stored final value, and ACCUMULATES dL/d(means, quats, scales,
 * opacities, rgb) into `out`.  `g` and `accel` must be the ones the forward pass used.  The
 * sums over rays are formed by atomic FP32 additions in device memory (float4 atomics, or one
 * 64 B bulk reduction per replayed hit), so their rounding, and the gradients' last bits,
 * change from call to call; the forward's outputs do not. */
rs_status rs_render_backward(const rs_gaussians* g, const rs_accel* accel,
                             const rs_fwd_state* state, const rs_frame_grad* dl,
                             const rs_tune_params* tune, rs_gaussian_grads* out,
                             void* cuda_stream);

/* rs_render_backward plus per-call counters of the replay (same layout as rs_render_counted:
 * rays, nodes visited, tests, replayed hits, rounds, inserted, rays re-traversed, hits
 * replayed from the list). */
rs_status rs_render_backward_counted(const rs_gaussians* g, const rs_accel* accel,
                                     const rs_fwd_state* state, const rs_frame_grad* dl,
                                     const rs_tune_params* tune, rs_gaussian_grads* out,
                                     uint64_t* stats_device, void* cuda_stream);

/* Autotuner (a11).  Times one training step (rs_build_accel + rs_render + optionally
 * rs_render_backward) of the caller's scene and cameras for each of n_candidates tunables
 * (1 untimed warm-up + `reps` steps timed with CUDA events on `cuda_stream`), writes the mean
 * milliseconds per step of candidate k to ms_out[k] (host array, may be NULL) and the fastest
 * candidate to *best.  scratch / scratch_grads / dl: caller's device buffers of the rs_render /
 * rs_render_backward layouts, used as outputs of the timed steps (their contents are
 * overwritten / accumulated into); dl == NULL times the forward only.  Allocates its own
 * temporary accel and state and synchronises the stream.  A candidate that fails validation is
 * skipped (ms_out = -1); RS_ERR_INVALID_ARG if none is valid. */
rs_status rs_tune(const rs_gaussians* g, float Q_box, const rs_camera* cams, int32_t n_cams,
                  const rs_render_params* params, const rs_tune_params* candidates,
                  int32_t n_candidates, int32_t reps, rs_frame* scratch,
                  const rs_frame_grad* dl, rs_gaussian_grads* scratch_grads,
                  rs_tune_params* best, float* ms_out, void* cuda_stream);

/* ---- Fixed-scratch render (no counterpart in the paper) ----------------------------------
 * For callers that cannot allocate device memory -- plug-ins whose host application owns every
 * device allocation (they are handed buffers, not an allocator), and tools that run under a
 * fixed device-memory budget and must not grow the process's footprint -- this entry point
 * builds the acceleration structure and renders the cameras (the work of rs_build_accel +
 * rs_render) without any cudaMalloc, cudaFree or other allocating call.  Every intermediate
 * lives in one file-scope device array of fixed size (about 12 MB, held by every GPU that
 * loads the library until the process exits).  The caller still passes the scene, the cameras
 * and the output buffers; there is no per-ray state for a backward pass.
 *   - Limits: g->n <= RS_FIXED_MAX_GAUSSIANS, n_cams <= RS_FIXED_MAX_CAMERAS, sum of W*H <=
 *     RS_FIXED_MAX_PIXELS (each camera is checked on its own first); larger requests, and
 *     non-finite camera or render parameters, return RS_ERR_INVALID_ARG before any launch.
 *   - The first call on a device resolves the array's device address (set-up, once per
 *     device, with that device current) and caches it; make no call on a device after a
 *     cudaDeviceReset of it.
 *   - All calls share the array and it keeps the previous call's contents (the call clears
 *     what must start at zero): calls that overlap on the GPU race with each other.
 *   - The camera table is passed to the device as a kernel argument: no host buffer is read
 *     after the call returns.
 *   - Q plays the role of rs_build_accel's Q_box.  Device consistency checks are not reported
 *     (there is no handle to query). */
#define RS_FIXED_MAX_GAUSSIANS 32768
#define RS_FIXED_MAX_PIXELS 262144
#define RS_FIXED_MAX_CAMERAS 16
rs_status rs_render_fixed_scratch(const rs_gaussians* g, const rs_camera* cams, int32_t n_cams,
                                  const rs_render_params* params, const rs_tune_params* tune,
                                  rs_frame* out, void* cuda_stream);

/* Free a handle (NULL is accepted).  Synchronises the device before freeing. */
rs_status rs_accel_destroy(rs_accel* accel);
rs_status rs_state_destroy(rs_fwd_state* state);

/* Synchronise `cuda_stream` and report the device error words of accel/state (either may be
 * NULL): RS_ERR_INTERNAL with a message if a device consistency check failed, else RS_OK.
 * Clears the words. */
rs_status rs_check_device(const rs_accel* accel, const rs_fwd_state* state, void* cuda_stream);

/* ---- Introspection (tests and tooling) -------------------------------------------------- */

/* Copy the LBVH of `accel` to host arrays (synchronises).  Each pointer may be NULL.
 *   codes[n]   sorted Morton codes          perm[n]   sorted position -> Gaussian id
 *   first[n-1], last[n-1], split[n-1]   Karras internal node ranges and split positions
 *   boxes[6 * (n-1)]  internal node boxes (lo xyz, hi xyz)   prim_boxes[6n] per sorted
 *   Gaussian, lo_hi[6] scene bounds of the means.  *n_out receives n. */
rs_status rs_accel_export(const rs_accel* accel, int64_t* n_out, uint64_t* codes, uint32_t* perm,
                          int32_t* first, int32_t* last, int32_t* split, float* boxes,
                          float* prim_boxes, float* lo_hi);

/* Generate the camera rays of n_rays listed pixels on the device (the exact FP32 operation
 * sequence the renderer uses).  cam_idx/px/py: device int32[n_rays]; o, d: device float[3 n]. */
rs_status rs_debug_rays(const rs_camera* cams, int32_t n_cams, int64_t n_rays,
                        const int32_t* cam_idx, const int32_t* px, const int32_t* py, float* o,
                        float* d, void* cuda_stream);

/* The renderer's ray/Gaussian test for n_pairs (ray r, sorted Gaussian j) pairs of `accel`:
 * out[8 * k .. 8 * k + 7] = D^2, t1, hit (1/0), alpha, r, b, tm, rm (device floats), where r is
 * the sub-ulp residual that the hit's ordering key carries below t1, decoded to units of
 * ulp(t1) (the centre of its bin, in [-1/2, 1/2]; 0 for a miss), and b the number of residual
 * bits, so that t1 + r ulp(t1) is the parameter the renderer orders hits by; tm and rm are the
 * same pair for the t_m ordering (sort_key 1: the key's high half max(t_m, t1) and its residual
 * in units of ulp(tm)).  ray_o/ray_d device float[3 n_pairs], sorted_j device int32[n_pairs];
 * out device float[8 n_pairs].  A sorted_j outside [0, n) gives NaN in all eight outputs. */
rs_status rs_debug_hits(const rs_accel* accel, int64_t n_pairs, const float* ray_o,
                        const float* ray_d, const int32_t* sorted_j, float Q, float t_near,
                        float* out, void* cuda_stream);

/* ---- Training-step pieces around the path (Sec. 3 "Loss Function", App. A.7, Sec. 5) ------ */

typedef struct rs_loss_state rs_loss_state;

/* Loss of a batch of rendered images against their targets and its gradient.  For each image
 * and colour channel, L_ch = (1 - lambda) mean((I - I^)^2) + lambda (1 - SSIM) / 2, with SSIM
 * the mean over pixels of App. A.7's per-pixel index: an 11 x 11 Gaussian window (sigma 1.5,
 * normalised), c1 = 0.01^2, c2 = 0.03^2, pixels outside the image taken as 0.  The image loss
 * is the mean over its three channels (App. A.7) and the batch loss the mean over images.
 *   rgb, target  device float[P * 3] in the rs_render layout (images concatenated camera by
 *                camera, pixel-major); only cams[c].width / height are read
 *   lambda       in [0, 1]
 *   loss_device  device float: the batch loss (written)
 *   d_rgb        device float[P * 3]: dL/drgb (written, not accumulated), App. A.7's
 *                ((E*w) + I^ (F*w) - I (G*w)) form; feed it to rs_render_backward
 *   *inout       scratch handle (NULL to create, else reused; 36 B per pixel)
 * Deterministic: the partial sums are reduced in a fixed order. */
rs_status rs_loss_l2_dssim(const float* rgb, const float* target, const rs_camera* cams,
                           int32_t n_cams, float lambda, float* loss_device, float* d_rgb,
                           rs_loss_state** inout, void* cuda_stream);
rs_status rs_loss_state_destroy(rs_loss_state* state);

/* One Adam update (Sec. 5; the paper uses beta1 0.9, beta2 0.999, eps 1e-8) of `count`
 * parameters, in place: m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2;
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).  params, m, v: device
 * float[count] (read and written); grads: device float[count]; step >= 1. */
rs_status rs_adam_step(float* params, const float* grads, float* m, float* v, int64_t count,
                       float lr, float beta1, float beta2, float eps, int32_t step,
                       void* cuda_stream);

/* The sigmoid activation of the opacities and scales (Sec. 5) and its adjoint: y = 1/(1 + e^-x);
 * dx = dy y (1 - y) (written).  Device float[count] each. */
rs_status rs_sigmoid(const float* x, float* y, int64_t count, void* cuda_stream);
rs_status rs_sigmoid_backward(const float* y, const float* dy, float* dx, int64_t count,
                              void* cuda_stream);

/* ---- Scenes with triangles: mirrors and shadows (Sec. 1, Fig. 1) -------------------------
 * The paper renders Gaussians together with meshes (mirrors, shadows) but gives no algorithm;
 * these are the rules implemented (and written out in the oracle):
 *   - a ray runs in segments; in each, the Gaussians whose entry t1 lies in [t_min, t_tri) are
 *     composited in (t1, id) order with the eps1 cut and k_max (counted over the whole ray),
 *     t_tri the nearest triangle (Moller-Trumbore; ties to the lower triangle id);
 *   - no triangle: the environment term is the background; a diffuse triangle (albedo a):
 *     a * T_s, T_s the transmittance of a shadow ray from the hit point to the light (product
 *     of (1 - alpha) over the Gaussians with entry in [eps_off, distance); 0 if a triangle
 *     blocks it or if the product falls below eps1, the shadow ray's own cut); a mirror
 *     triangle: the ray reflects (at most max_bounces times; beyond that the term is 0) and
 *     the next segment starts at t_min = eps_off;
 *   - a ray cut by eps1 or k_max keeps the term of the segment it stopped in (a mirror: 0);
 *   - RGB = composited colour + T_final * term, alpha = 1 - T_final, depth = sum w_i t1_i over
 *     the first segment; triangle hits, reflections and shadow rays follow fixed FP32
 *     sequences (the same as the camera rays', round-to-nearest, no contraction);
 *   - the adjoint is the exact gradient w.r.t. the Gaussian parameters (the mesh and the
 *     light are fixed).
 * Only sort_key 0, depth_mode 0 and grad_mode 0 are supported here. */
typedef struct rs_mesh rs_mesh;
typedef struct rs_scene_state rs_scene_state;

typedef struct {
    int64_t n_tri;
    const float* verts;       /* host float[9 n_tri]: v0, v1, v2 */
    const int32_t* material;  /* host int32[n_tri]: 0 mirror, 1 diffuse */
    const float* albedo;      /* host float[3 n_tri] (diffuse) */
} rs_mesh_desc;

typedef struct {
    float light[3];           /* point light position */
    int32_t max_bounces;      /* 0..2 mirror reflections */
    float eps_off;            /* > 0: t_min of reflected and shadow rays */
    int32_t list_cap;         /* 1..4096 composited ids kept per ray for the adjoint */
    int32_t shadow_cap;       /* 1..4096 shadow-ray ids kept per ray */
} rs_scene_params;

/* Build the mesh's BVH (host, once: median splits, leaves of <= 4 triangles) and upload it. */
rs_status rs_build_mesh(const rs_mesh_desc* desc, rs_mesh** out);
rs_status rs_mesh_destroy(rs_mesh* mesh);

/* Render n_cams cameras of the Gaussians `g` (LBVH `accel`) together with `mesh`; outputs as
 * rs_render.  *inout: the per-ray state the adjoint needs (NULL to create; about
 * 150 B + 4 B (list_cap + shadow_cap) per ray).  A ray whose ids overflow a list sets a device
 * error bit that rs_check_device(accel, ...) reports (its gradient is then incomplete). */
rs_status rs_render_scene(const rs_gaussians* g, const rs_accel* accel, const rs_mesh* mesh,
                          const rs_scene_params* sp, const rs_camera* cams, int32_t n_cams,
                          const rs_render_params* params, const rs_tune_params* tune,
                          rs_frame* out, rs_scene_state** inout, void* cuda_stream);

/* ACCUMULATE the gradient of the last rs_render_scene recorded in `state` w.r.t. the Gaussian
 * parameters (d_alpha and d_depth may be NULL). */
rs_status rs_render_scene_backward(const rs_gaussians* g, const rs_accel* accel,
                                   const rs_scene_state* state, const rs_frame_grad* dl,
                                   rs_gaussian_grads* out, void* cuda_stream);
rs_status rs_scene_state_destroy(rs_scene_state* state);

/* Allocation-failure injection, for tests of the out-of-memory paths (the paper has no
 * counterpart).  With n > 0 the n-th device allocation the library makes from now on fails
 * with RS_ERR_OOM (no cudaMalloc is attempted) and the hook disarms itself; n = 0 disarms it.
 * Process-wide and not thread-safe; n < 0 returns RS_ERR_INVALID_ARG.  A call that fails this
 * way leaves its handle unusable but valid: rs_render / rs_render_backward reject it with
 * RS_ERR_INVALID_ARG until a later rs_build_accel / rs_render succeeds on it, and the
 * *_destroy functions free it. */
rs_status rs_test_fail_alloc(int64_t n);

#ifdef __cplusplus
}
#endif
#endif /* RAYSPLATS_H */
