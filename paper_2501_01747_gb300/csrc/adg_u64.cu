// The unsynchronised mode, FP64 variant (the limiter's CTAs hold 16 or 32
// elements, as in the group's synchronous limiter).
#include "adg_unsync.cuh"

namespace adg {

cudaError_t launch_unsync_fp64(const Mech &M, const UnsyncArgs &U, int Q, int nv,
                               cudaStream_t st) {
  if (U.EPB == 16) return unsync_launch_variant<false, 16>(M, U, Q, nv, st);
  if (U.EPB != LIM_EPB_MAX) return cudaErrorInvalidValue;
  return unsync_launch_variant<false, LIM_EPB_MAX>(M, U, Q, nv, st);
}

cudaError_t prepare_unsync_fp64() {
  cudaError_t e = unsync_prepare_variant<false, 16>();
  return e != cudaSuccess ? e : unsync_prepare_variant<false, LIM_EPB_MAX>();
}

cudaError_t upload_tables_unsync_fp64(const Basis *tables) { return upload_unit_tables(tables); }

}  // namespace adg
