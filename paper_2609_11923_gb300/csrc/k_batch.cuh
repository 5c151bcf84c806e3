// k_batch.cuh — dispatch of the batched kernels over their instances.
#pragma once
#include "launch.h"

namespace cfr {

#define CFR_BATCH_LANES(X, MA, TH) X(MA, 2, TH) X(MA, 4, TH) X(MA, 8, TH) X(MA, 32, TH)
#define CFR_BATCH_ALL(X) \
  CFR_BATCH_LANES(X, 4, 256) CFR_BATCH_LANES(X, 4, 1024) CFR_BATCH_LANES(X, 8, 256) CFR_BATCH_LANES(X, 8, 1024)

template <typename T>
cudaError_t launch_batch_iterate(int maxa, int lanes, int threads, int n, cudaStream_t s, const InstDesc *table) {
#define IT_CASE(MA, L, TH)                                                   \
  if (maxa == MA && lanes == L && threads == TH) {                           \
    batch_iterate_kernel<T, MA, L, TH><<<n, TH, 0, s>>>(table, n);           \
    return cudaGetLastError();                                               \
  }
  CFR_BATCH_ALL(IT_CASE)
#undef IT_CASE
  return cudaErrorInvalidValue;
}

}  // namespace cfr
