#include "ktau_impl.cuh"
extern "C" {
ktau_status ktau_batch_create(const ktau_batch_desc*, int32_t, const ktau_options*, ktau_batch** out) {
  if (out) *out = nullptr;
  return ktau_fail(KTAU_EINVAL, "batched form not available");
}
ktau_status ktau_batch_run(ktau_batch*, void*) { return ktau_fail(KTAU_EINVAL, "n/a"); }
ktau_status ktau_batch_graph_launch(ktau_batch*, void*) { return ktau_fail(KTAU_EINVAL, "n/a"); }
ktau_status ktau_batch_check(ktau_batch*, void*) { return ktau_fail(KTAU_EINVAL, "n/a"); }
ktau_status ktau_batch_paths(const ktau_batch*, int32_t*, int32_t*) { return ktau_fail(KTAU_EINVAL, "n/a"); }
ktau_status ktau_batch_pairs(const ktau_batch*, uint64_t*) { return ktau_fail(KTAU_EINVAL, "n/a"); }
ktau_status ktau_batch_free(ktau_batch*) { return KTAU_OK; }
ktau_status ktau_query(const ktau_ranked*, const ktau_ranked*, double*, void*, void*, int32_t, int32_t,
                       int32_t*, double*, const ktau_options*, void*) {
  return ktau_fail(KTAU_EINVAL, "query form not available");
}
ktau_status ktau_query_scratch_bytes(const ktau_ranked*, int64_t, int32_t, size_t*) {
  return ktau_fail(KTAU_EINVAL, "query form not available");
}
}
