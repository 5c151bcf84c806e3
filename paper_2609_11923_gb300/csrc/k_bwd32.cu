// Backward-level kernel instances, P32 (see kernels.cuh).
#include "launch_impl.cuh"
namespace cfr {
template cudaError_t launch_bwd_level<float>(int, int, int, cudaStream_t, GameView, StateView<float>, LevelWork, int, int, int, int, bool);
}

namespace cfr {
template <int MA>
static cudaError_t stream_one(int grid, cudaStream_t s, GameView g, StateView<float> st, const SetInfo *info,
                              const StreamChunk *chunks, int c0, int c1, int rule, int upd, int *err, bool pdl,
                              int early) {
  return launch_k(bwd_stream_kernel<MA>, grid, kStreamThreads, (size_t)kStreamDynSmem, s, pdl, g, st, info, chunks,
                  c0, c1, rule, upd, err, early);
}

cudaError_t prepare_bwd_stream() {
  const int dyn = kStreamDynSmem;
  cudaError_t e = cudaFuncSetAttribute(bwd_stream_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(bwd_stream_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  return e;
}

cudaError_t launch_bwd_stream(int maxa, int grid, cudaStream_t s, GameView g, StateView<float> st,
                              const SetInfo *info, const StreamChunk *chunks, int c0, int c1, int rule, int upd,
                              int *err, bool pdl, bool early) {
  const int e = early ? 1 : 0;
  if (maxa == 4) return stream_one<4>(grid, s, g, st, info, chunks, c0, c1, rule, upd, err, pdl, e);
  if (maxa == 8) return stream_one<8>(grid, s, g, st, info, chunks, c0, c1, rule, upd, err, pdl, e);
  return cudaErrorInvalidValue;
}
}  // namespace cfr
