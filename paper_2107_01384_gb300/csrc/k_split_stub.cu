// Placeholder for the split-precision tensor-core contractions until they are built.
#include "atc_internal.cuh"

namespace atc {
int launch_gram_split(const void*, int, int64_t, int64_t, int64_t, int, double*, cudaStream_t) {
  return fail(ATC_EUNSUP, "split-precision Gram not available in this build");
}
int launch_ttm_split(const void*, int, int64_t, int64_t, int64_t, const double*, int64_t, int, int, void*, int,
                     cudaStream_t) {
  return fail(ATC_EUNSUP, "split-precision TTM not available in this build");
}
}  // namespace atc
