// The ADG_MIXED_F32CHEM variant of the stage kernel (FP32 flux and DG operator;
// chemistry exponents as float pairs, its exponentials, products and sums in
// FP32), in its own translation unit, compiled in parallel with the others. Its
// limiter is the FP32 one of adg_k32.cu.
#include "adg_device.cuh"

namespace adg {

cudaError_t launch_stage_f32chem(const Mech &M, const StageArgs &A, int Q, int n_tiles,
                                 cudaStream_t st) {
  return launch_stage_variant<ADG_MIXED_F32CHEM, false>(M, A, Q, n_tiles, st);
}

cudaError_t prepare_f32chem() { return prepare_stage_variant<ADG_MIXED_F32CHEM, false>(); }

cudaError_t upload_tables_f32chem(const Basis *tables) { return upload_unit_tables(tables); }

}  // namespace adg
