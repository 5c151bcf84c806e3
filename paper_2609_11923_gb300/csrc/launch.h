// launch.h — host wrappers that pick the kernel instance (actions tier x
// lanes per information set). Each wrapper is defined in its own translation
// unit so the instances compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "bwd_stream.cuh"

namespace cfr {

// Launch of a per-level kernel; with pdl set, as a programmatic dependent
// launch (the kernel waits for its predecessor itself: pdl_enter).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, bool pdl,
                            Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// The streaming FP32 backward of one depth (bwd_stream_kernel); grid = the
// streaming CTAs over the depth's chunks [c0, c1) (set and chance chunks).
// early (with pdl only, and only when the launch before is the backward
// launch of the next depth): copy every input but the children's values
// before waiting for that launch.
cudaError_t launch_bwd_stream(int maxa, int grid, cudaStream_t s, GameView g, StateView<float> st,
                              const SetInfo *info, const StreamChunk *chunks, int c0, int c1, int rule, int upd,
                              int *err, bool pdl, bool early);
// Allows the streaming kernel its dynamic shared memory (call before the
// first launch, outside any stream capture; idempotent).
cudaError_t prepare_bwd_stream();

template <typename T>
cudaError_t launch_bwd_level(int maxa, int lanes, int grid, cudaStream_t s, GameView g, StateView<T> st,
                             LevelWork w, int nb_chance, int rule, int upd, int bump, bool pdl = false);

// query_occupancy != nullptr: only report resident blocks per SM of the
// chosen instance (nothing is launched).
template <typename T>
cudaError_t launch_persistent(int maxa, int lanes, int grid, cudaStream_t s, PersistArgs<T> a,
                              int *query_occupancy);

cudaError_t launch_br_level(int maxa, int lanes, int grid, cudaStream_t s, GameView g, const double2 *reach2,
                            const double *sbs, double2 *vb, double *vavg, LevelWork w, int nb_chance);

}  // namespace cfr

#include "batch.cuh"

namespace cfr {
template <typename T>
cudaError_t launch_batch_iterate(int maxa, int lanes, int threads, int cluster, int n, cudaStream_t s,
                                 const InstDesc *table);
cudaError_t launch_batch_br(int maxa, int lanes, int threads, int n, cudaStream_t s, const InstDesc *table);
}  // namespace cfr
