// The mixed-precision (MIX) variant of the stage and limiter kernels (its own translation unit,
// compiled in parallel with the others).
#include "adg_device.cuh"

namespace adg {

cudaError_t launch_stage_mixed(const Mech &M, const StageArgs &A, int Q, int n_tiles,
                              cudaStream_t st) {
  return launch_stage_variant<true, false>(M, A, Q, n_tiles, st);
}

cudaError_t launch_limiter_mixed(const Mech &M, const LimArgs &A, int Q, int nv, int n_blocks,
                                cudaStream_t st) {
  return launch_limiter_variant<true>(M, A, Q, nv, n_blocks, st);
}

cudaError_t prepare_mixed() { return prepare_variant<true>(); }

cudaError_t upload_tables_mixed(const Basis *tables) { return upload_unit_tables(tables); }

}  // namespace adg
