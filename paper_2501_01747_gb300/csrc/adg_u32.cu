// The unsynchronised mode, mixed-precision variant (the limiter's CTAs hold 8,
// 16 or 32 elements, as the synchronous launches of the same group).
#include "adg_unsync.cuh"

namespace adg {

cudaError_t launch_unsync_mixed(const Mech &M, const UnsyncArgs &U, int Q, int nv,
                                cudaStream_t st) {
  if (U.EPB == 8) return unsync_launch_variant<true, 8>(M, U, Q, nv, st);
  if (U.EPB == 16) return unsync_launch_variant<true, 16>(M, U, Q, nv, st);
  if (U.EPB == LIM_EPB_MAX) return unsync_launch_variant<true, LIM_EPB_MAX>(M, U, Q, nv, st);
  return cudaErrorInvalidValue;
}

cudaError_t prepare_unsync_mixed() {
  cudaError_t e = unsync_prepare_variant<true, 8>();
  if (e == cudaSuccess) e = unsync_prepare_variant<true, 16>();
  if (e == cudaSuccess) e = unsync_prepare_variant<true, LIM_EPB_MAX>();
  return e;
}

cudaError_t upload_tables_unsync_mixed(const Basis *tables) { return upload_unit_tables(tables); }

}  // namespace adg
