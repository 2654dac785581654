// The FP64 variant of the stage and limiter kernels (its own translation unit,
// compiled in parallel with the others).
#include "adg_device.cuh"

namespace adg {

cudaError_t launch_stage_fp64(const Mech &M, const StageArgs &A, int Q, int n_tiles,
                              cudaStream_t st) {
  return launch_stage_variant<ADG_FP64, false>(M, A, Q, n_tiles, st);
}

cudaError_t launch_limiter_fp64(const Mech &M, const LimArgs &A, int Q, int nv, int n_blocks,
                                cudaStream_t st) {
  return launch_limiter_variant<false>(M, A, Q, nv, n_blocks, st);
}

cudaError_t prepare_fp64() {
  cudaError_t e = prepare_stage_variant<ADG_FP64, false>();
  return e != cudaSuccess ? e : prepare_limiter_variant<false>();
}

cudaError_t upload_tables_fp64(const Basis *tables) { return upload_unit_tables(tables); }

}  // namespace adg
