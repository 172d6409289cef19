// render_bwd_depth.cu -- the adjoint's kernels and launchers with the depth gradient
// (DEPTH = true), compiled apart from render_bwd.cu so that the two halves of the kernel
// instantiations build in parallel.
#include "render_bwd.cuh"

namespace rs {

int persistent_grid_bwd_depth(int K, int block, bool count, int mode, int n_top, int sms) {
    return persistent_grid_bwd_d<true>(K, block, count, mode, n_top, sms);
}

cudaError_t launch_backward_depth(const FwdArgs& A, const BwdArgs& B, int K, bool persistent, bool count, int mode,
                                  int grid, int block, cudaStream_t st) {
    return launch_bwd_d<true>(A, B, K, persistent, count, mode, grid, block, st);
}

int list_replay_grid_depth(bool count, int block, int sms) { return list_replay_grid_d<true>(count, block, sms); }

void launch_list_replay_depth(const FwdArgs& A, const BwdArgs& B, bool persistent, bool count, int grid, int block,
                              cudaStream_t st) {
    launch_list_d<true>(A, B, persistent, count, grid, block, st);
}

}  // namespace rs
