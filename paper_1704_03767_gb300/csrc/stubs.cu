#include "ktau_impl.cuh"
extern "C" {
ktau_status ktau_query(const ktau_ranked*, const ktau_ranked*, double*, void*, void*, int32_t, int32_t,
                       int32_t*, double*, const ktau_options*, void*) {
  return ktau_fail(KTAU_EINVAL, "query form not available");
}
ktau_status ktau_query_scratch_bytes(const ktau_ranked*, int64_t, int32_t, size_t*) {
  return ktau_fail(KTAU_EINVAL, "query form not available");
}
}
