// Host entry points of the 1D stage kernels: shared-memory sizes and launches, dispatched on
// the state precision to the instantiations in kern1d_f32.cu / kern1d_f64.cu.
#include "kern1d_fused.cuh"

namespace frsg {

cudaError_t k1d_stage_f32(const frsg_config& cfg, const StageArgs& A, cudaStream_t st);
cudaError_t k1d_stage_f64(const frsg_config& cfg, const StageArgs& A, cudaStream_t st);
cudaError_t k1d_step_f32(const frsg_config& cfg, const StageArgs* A3, unsigned* bar, int* grid, cudaStream_t st);
cudaError_t k1d_step_f64(const frsg_config& cfg, const StageArgs* A3, unsigned* bar, int* grid, cudaStream_t st);
cudaError_t k1d_fused_f32(const frsg_config& cfg, const StageArgs* A3, unsigned long long* tok, cudaStream_t st,
                          bool check_only);
cudaError_t k1d_fused_f64(const frsg_config& cfg, const StageArgs* A3, unsigned long long* tok, cudaStream_t st,
                          bool check_only);
cudaError_t k1d_batched_f32(int equation, const StageArgs* args, const int4* tiles, int ntiles, size_t smem, int grid,
                            cudaStream_t st);
cudaError_t k1d_batched_f64(int equation, const StageArgs* args, const int4* tiles, int ntiles, size_t smem, int grid,
                            cudaStream_t st);
cudaError_t k1d_batched_rec_f64(int equation, const StageArgs* args, const int4* tiles, int ntiles, size_t smem,
                                int grid, int seg_j, int log_n, cudaStream_t st);
int k1d_batched_occ_f32(int equation, size_t smem);
int k1d_batched_occ_f64(int equation, size_t smem);

size_t stage1d_smem_bytes(bool fp64, int TE, int NP, int M, int Q, int S) {
    return fp64 ? smem1d_bytes<double>(TE, NP, M, Q, S) : smem1d_bytes<float>(TE, NP, M, Q, S);
}

size_t stage1d_wide_smem_bytes(bool fp64, int TE, int NP, int M, int Q, int S) {
    return fp64 ? smem1d_wide_bytes<double>(TE, NP, M, Q, S) : smem1d_wide_bytes<float>(TE, NP, M, Q, S);
}

size_t stage1d_fused_smem_bytes(bool fp64, int TE, int NP, int M, int Q, int S) {
    return fp64 ? smem1d_fused_bytes<double>(TE, NP, M, Q, S) : smem1d_fused_bytes<float>(TE, NP, M, Q, S);
}

cudaError_t launch_stage1d(const frsg_config& cfg, bool fp64, const StageArgs& A, cudaStream_t st) {
    StageArgs B = A;
    prepare_float_scalars(B);
    return fp64 ? k1d_stage_f64(cfg, B, st) : k1d_stage_f32(cfg, B, st);
}

cudaError_t launch_stage1d_batched(bool fp64, int equation, const StageArgs* args, const int4* tiles, int ntiles,
                                   size_t smem, int grid, cudaStream_t st) {
    return fp64 ? k1d_batched_f64(equation, args, tiles, ntiles, smem, grid, st)
                : k1d_batched_f32(equation, args, tiles, ntiles, smem, grid, st);
}

cudaError_t launch_stage1d_batched_rec(int equation, const StageArgs* args, const int4* tiles, int ntiles,
                                       size_t smem, int grid, int seg_j, int log_n, cudaStream_t st) {
    return k1d_batched_rec_f64(equation, args, tiles, ntiles, smem, grid, seg_j, log_n, st);
}

cudaError_t launch_step1d(const frsg_config& cfg, bool fp64, const StageArgs* A3, unsigned* bar, int* grid,
                          cudaStream_t st) {
    StageArgs B3[3] = {A3[0], A3[1], A3[2]};
    for (int s = 0; s < 3; ++s) prepare_float_scalars(B3[s]);
    return fp64 ? k1d_step_f64(cfg, B3, bar, grid, st) : k1d_step_f32(cfg, B3, bar, grid, st);
}

cudaError_t launch_fused1d(const frsg_config& cfg, bool fp64, const StageArgs* A3, unsigned long long* tok,
                           cudaStream_t st, bool check_only) {
    StageArgs B3[3] = {A3[0], A3[1], A3[2]};
    for (int s = 0; s < 3; ++s) prepare_float_scalars(B3[s]);
    return fp64 ? k1d_fused_f64(cfg, B3, tok, st, check_only) : k1d_fused_f32(cfg, B3, tok, st, check_only);
}

int stage1d_batched_blocks_per_sm(bool fp64, int equation, size_t smem) {
    return fp64 ? k1d_batched_occ_f64(equation, smem) : k1d_batched_occ_f32(equation, smem);
}

}  // namespace frsg
