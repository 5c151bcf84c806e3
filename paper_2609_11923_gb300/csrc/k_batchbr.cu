// Batched best-response kernel instances (see batch.cuh).
#include "k_batch.cuh"
namespace cfr {
cudaError_t launch_batch_br(int maxa, int lanes, int threads, int n, cudaStream_t s, const InstDesc *table) {
#define BR_CASE(MA, L, TH)                                                   \
  if (maxa == MA && lanes == L && threads == TH) {                           \
    batch_br_kernel<MA, L, TH><<<n, TH, 0, s>>>(table, n);                   \
    return cudaGetLastError();                                               \
  }
  CFR_BATCH_ALL(BR_CASE)
#undef BR_CASE
  return cudaErrorInvalidValue;
}
}  // namespace cfr
