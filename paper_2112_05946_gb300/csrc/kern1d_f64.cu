// Instantiations of the 1D stage kernels for double states (the kernel templates are in
// kern1d.cuh; one translation unit per precision keeps the build parallel).
#include "kern1d_fused.cuh"

namespace frsg {

cudaError_t k1d_stage_f64(const frsg_config& cfg, const StageArgs& A, cudaStream_t st) {
    return launch_np<double>(cfg, A, st);
}

cudaError_t k1d_step_f64(const frsg_config& cfg, const StageArgs* A3, unsigned* bar, int* grid, cudaStream_t st) {
    return step_np<double>(cfg, A3, bar, grid, st);
}

cudaError_t k1d_fused_f64(const frsg_config& cfg, const StageArgs* A3, unsigned long long* tok, cudaStream_t st,
                          bool check_only) {
    return fused_np<double>(cfg, A3, tok, st, check_only);
}

cudaError_t k1d_batched_f64(int equation, const StageArgs* args, const int4* tiles, int ntiles, size_t smem, int grid,
                          cudaStream_t st) {
    if (equation == FRSG_EQ_ADVECTION) return batched_typed<double, FRSG_EQ_ADVECTION>(args, tiles, ntiles, smem, grid, st);
    if (equation == FRSG_EQ_BURGERS) return batched_typed<double, FRSG_EQ_BURGERS>(args, tiles, ntiles, smem, grid, st);
    return cudaErrorInvalidValue;
}

cudaError_t k1d_batched_rec_f64(int equation, const StageArgs* args, const int4* tiles, int ntiles, size_t smem,
                                int grid, int seg_j, int log_n, cudaStream_t st) {
    if (equation == FRSG_EQ_ADVECTION)
        return batched_rec_typed<double, FRSG_EQ_ADVECTION>(args, tiles, ntiles, smem, grid, seg_j, log_n, st);
    if (equation == FRSG_EQ_BURGERS)
        return batched_rec_typed<double, FRSG_EQ_BURGERS>(args, tiles, ntiles, smem, grid, seg_j, log_n, st);
    return cudaErrorInvalidValue;
}

int k1d_batched_occ_f64(int equation, size_t smem) {
    if (equation == FRSG_EQ_ADVECTION) return batched_occ<double, FRSG_EQ_ADVECTION>(smem);
    return batched_occ<double, FRSG_EQ_BURGERS>(smem);
}

}  // namespace frsg
