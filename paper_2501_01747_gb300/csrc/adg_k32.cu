// The ADG_MIXED variant of the stage kernel (FP32 flux and DG operator, FP64
// chemistry) and the FP32 limiter of both mixed variants (its own translation
// unit, compiled in parallel with the others).
#include "adg_device.cuh"

namespace adg {

cudaError_t launch_stage_mixed(const Mech &M, const StageArgs &A, int Q, int n_tiles,
                              cudaStream_t st) {
  return launch_stage_variant<ADG_MIXED, false>(M, A, Q, n_tiles, st);
}

cudaError_t launch_limiter_mixed(const Mech &M, const LimArgs &A, int Q, int nv, int n_blocks,
                                cudaStream_t st) {
  return launch_limiter_variant<true>(M, A, Q, nv, n_blocks, st);
}

cudaError_t prepare_mixed() {
  cudaError_t e = prepare_stage_variant<ADG_MIXED, false>();
  return e != cudaSuccess ? e : prepare_limiter_variant<true>();
}

cudaError_t upload_tables_mixed(const Basis *tables) { return upload_unit_tables(tables); }

}  // namespace adg
