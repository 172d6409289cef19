// render_bwd.cu -- the adjoint's entry points (a10): hit-list replay, re-traversal of the
// overflow tiles, and the finalize map to (quaternion, scale).  The kernels and their templated
// launchers are in render_bwd.cuh; this unit instantiates them without the depth gradient and
// render_bwd_depth.cu with it.
#include "render_bwd.cuh"

namespace rs {

// dL/dM, dL/dm, dL/dopacity, dL/drgb (Morton order) -> caller's gradients (Gaussian ids).
// M = S^-1 R^T:  dL/ds_k = -(1/s_k) sum_l G[k][l] M[k][l];  dL/dR[l][k] = G[k][l] / s_k;
// R = I + s_q K(q), s_q = 2/|q|^2 (App. A.6):  dR/dq_x = -s_q^2 q_x K + s_q dK/dq_x.
__global__ void k_finalize(const float4* __restrict__ gtmp, const float4* __restrict__ rec,
                           const uint32_t* __restrict__ perm, const float* __restrict__ quats,
                           const float* __restrict__ scales, int64_t n, rs_gaussian_grads out) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t i = perm[j];
    const float4 G0 = gtmp[4 * j], G1 = gtmp[4 * j + 1], G2 = gtmp[4 * j + 2], G3 = gtmp[4 * j + 3];
    if (out.d_means) {
        out.d_means[3 * i] += G0.w;
        out.d_means[3 * i + 1] += G1.w;
        out.d_means[3 * i + 2] += G2.w;
    }
    if (out.d_opacities) out.d_opacities[i] += G3.x;
    if (out.d_rgb) {
        out.d_rgb[3 * i] += G3.y;
        out.d_rgb[3 * i + 1] += G3.z;
        out.d_rgb[3 * i + 2] += G3.w;
    }
    if (!out.d_scales && !out.d_quats) return;
    const float GM[3][3] = {{G0.x, G0.y, G0.z}, {G1.x, G1.y, G1.z}, {G2.x, G2.y, G2.z}};
    const float4 m0 = rec[4 * j], m1 = rec[4 * j + 1], m2 = rec[4 * j + 2];
    const float M[3][3] = {{m0.x, m0.y, m0.z}, {m1.x, m1.y, m1.z}, {m2.x, m2.y, m2.z}};
    const float s[3] = {scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]};
    if (out.d_scales) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
            out.d_scales[3 * i + k] += -(GM[k][0] * M[k][0] + GM[k][1] * M[k][1] + GM[k][2] * M[k][2]) / s[k];
    }
    if (out.d_quats) {
        const float qa = quats[4 * i], qb = quats[4 * i + 1], qc = quats[4 * i + 2], qd = quats[4 * i + 3];
        const float sq = 2.f / (qa * qa + qb * qb + qc * qc + qd * qd);
        float GR[3][3];  // dL/dR[l][k]
#pragma unroll
        for (int l = 0; l < 3; ++l)
#pragma unroll
            for (int k = 0; k < 3; ++k) GR[l][k] = GM[k][l] / s[k];
        const float Kq[3][3] = {{-(qc * qc + qd * qd), qb * qc - qa * qd, qb * qd + qa * qc},
                                {qb * qc + qa * qd, -(qb * qb + qd * qd), qc * qd - qa * qb},
                                {qb * qd - qa * qc, qc * qd + qa * qb, -(qb * qb + qc * qc)}};
        float GK = 0.f;
#pragma unroll
        for (int l = 0; l < 3; ++l)
#pragma unroll
            for (int k = 0; k < 3; ++k) GK += GR[l][k] * Kq[l][k];
        // sum over entries of GR (.) dK/dq_x
        const float da = GR[0][1] * (-qd) + GR[0][2] * qc + GR[1][0] * qd + GR[1][2] * (-qb) + GR[2][0] * (-qc) +
                         GR[2][1] * qb;
        const float db = GR[0][1] * qc + GR[0][2] * qd + GR[1][0] * qc + GR[1][1] * (-2.f * qb) + GR[1][2] * (-qa) +
                         GR[2][0] * qd + GR[2][1] * qa + GR[2][2] * (-2.f * qb);
        const float dc = GR[0][0] * (-2.f * qc) + GR[0][1] * qb + GR[0][2] * qa + GR[1][0] * qb + GR[1][2] * qd +
                         GR[2][0] * (-qa) + GR[2][1] * qd + GR[2][2] * (-2.f * qc);
        const float dd = GR[0][0] * (-2.f * qd) + GR[0][1] * (-qa) + GR[0][2] * qb + GR[1][0] * qa +
                         GR[1][1] * (-2.f * qd) + GR[1][2] * qc + GR[2][0] * qb + GR[2][1] * qc;
        const float ns = -sq * sq * GK;
        out.d_quats[4 * i] += ns * qa + sq * da;
        out.d_quats[4 * i + 1] += ns * qb + sq * db;
        out.d_quats[4 * i + 2] += ns * qc + sq * dc;
        out.d_quats[4 * i + 3] += ns * qd + sq * dd;
    }
}


// ---------------------------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------------------------
int persistent_grid_bwd(int K, int block, bool count, int mode, int n_top, int sms, bool depth) {
    return depth ? persistent_grid_bwd_depth(K, block, count, mode, n_top, sms)
                 : persistent_grid_bwd_d<false>(K, block, count, mode, n_top, sms);
}

cudaError_t launch_backward(const FwdArgs& A, const BwdArgs& B, int K, bool persistent, bool count, int mode,
                            int grid, int block, cudaStream_t st) {
    return B.d_depth ? launch_backward_depth(A, B, K, persistent, count, mode, grid, block, st)
                     : launch_bwd_d<false>(A, B, K, persistent, count, mode, grid, block, st);
}

int list_replay_grid(bool count, int block, int sms, bool depth) {
    return depth ? list_replay_grid_depth(count, block, sms) : list_replay_grid_d<false>(count, block, sms);
}

cudaError_t launch_list_replay(const FwdArgs& A, const BwdArgs& B, bool persistent, bool count, int grid, int block,
                               cudaStream_t st) {
    if (B.d_depth) launch_list_replay_depth(A, B, persistent, count, grid, block, st);
    else launch_list_d<false>(A, B, persistent, count, grid, block, st);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const float4* gtmp, const float4* rec, const uint32_t* perm, const float* quats,
                            const float* scales, int64_t n, const rs_gaussian_grads& out, cudaStream_t st) {
    k_finalize<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(gtmp, rec, perm, quats, scales, n, out);
    return cudaGetLastError();
}

}  // namespace rs
