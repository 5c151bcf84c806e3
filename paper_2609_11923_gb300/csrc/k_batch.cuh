// k_batch.cuh — dispatch of the batched kernels over their instances.
#pragma once
#include "launch.h"

namespace cfr {

#define CFR_BATCH_LANES(X, MA, TH) X(MA, 2, TH) X(MA, 4, TH) X(MA, 8, TH) X(MA, 32, TH)
#define CFR_BATCH_ALL(X) \
  CFR_BATCH_LANES(X, 4, 256) CFR_BATCH_LANES(X, 4, 1024) CFR_BATCH_LANES(X, 8, 256) CFR_BATCH_LANES(X, 8, 1024)

// cluster == 1: one CTA per instance; else a cluster of `cluster` CTAs per
// instance (the clustered instances, launched with a cluster dimension).
template <typename T, int MA, int L, int TH>
static cudaError_t launch_batch_one(int cluster, int n, cudaStream_t s, const InstDesc *table) {
  if (cluster == 1) {
    batch_iterate_kernel<T, MA, L, TH, false><<<n, TH, 0, s>>>(table, n);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n * cluster));
  cfg.blockDim = dim3(TH);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_iterate_kernel<T, MA, L, TH, true>, table, n);
}

template <typename T>
cudaError_t launch_batch_iterate(int maxa, int lanes, int threads, int cluster, int n, cudaStream_t s,
                                 const InstDesc *table) {
#define IT_CASE(MA, L, TH) \
  if (maxa == MA && lanes == L && threads == TH) return launch_batch_one<T, MA, L, TH>(cluster, n, s, table);
  CFR_BATCH_ALL(IT_CASE)
#undef IT_CASE
  return cudaErrorInvalidValue;
}

}  // namespace cfr
