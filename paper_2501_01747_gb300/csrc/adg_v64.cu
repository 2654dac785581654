// The stage kernel with the viscous terms (LDG), FP64 variant, in its own
// translation unit so that the Euler kernels keep their register budget and the
// units compile in parallel.
#include "adg_device.cuh"

namespace adg {

cudaError_t launch_stage_visc_fp64(const Mech &M, const StageArgs &A, int Q, int n_tiles,
                                   cudaStream_t st) {
  return launch_stage_variant<ADG_FP64, true>(M, A, Q, n_tiles, st);
}

cudaError_t prepare_visc_fp64() { return prepare_stage_variant<ADG_FP64, true>(); }

cudaError_t upload_tables_visc_fp64(const Basis *tables) { return upload_unit_tables(tables); }

}  // namespace adg
