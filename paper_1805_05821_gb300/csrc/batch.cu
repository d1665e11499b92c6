// Batched streams: placeholder entry points until the persistent multi-stream kernel lands.
#include "api_internal.cuh"

extern "C" int foa_dmd_batch_create(int32_t, const int64_t *, const int32_t *, int32_t, const foa_dmd_opts *,
                                    foa_dmd_batch_t **out) {
  if (out) *out = nullptr;
  return FOA_DMD_EINVAL;
}
extern "C" int foa_dmd_batch_push(foa_dmd_batch_t *, const void *const *, double *) { return FOA_DMD_EINVAL; }
extern "C" int foa_dmd_batch_get_state(foa_dmd_batch_t *, int32_t, int32_t *, int32_t *, double *, double *,
                                       int32_t) {
  return FOA_DMD_EINVAL;
}
extern "C" int foa_dmd_batch_get_basis(foa_dmd_batch_t *, int32_t, int32_t, int32_t, void *, int64_t) {
  return FOA_DMD_EINVAL;
}
extern "C" void foa_dmd_batch_destroy(foa_dmd_batch_t *) {}
