// launch_impl.cuh — definitions of the launch wrappers declared in launch.h.
#pragma once
#include "launch.h"

namespace cfr {

template <typename T>
cudaError_t launch_bwd_level(int maxa, int lanes, int grid, cudaStream_t s, GameView g, StateView<T> st,
                             LevelWork w, int nb_chance, int rule, int upd, int bump, bool pdl) {
#define BWD_CASE(MA, L)                                                                                     \
  if (maxa == MA && lanes == L)                                                                             \
    return launch_k(bwd_level_kernel<T, MA, L>, grid, kThreads, 0, s, pdl, g, st, w, nb_chance, rule, upd, bump);
  BWD_CASE(4, 1) BWD_CASE(4, 2) BWD_CASE(4, 4) BWD_CASE(4, 8) BWD_CASE(4, 16) BWD_CASE(4, 32) BWD_CASE(4, kThreads)
  BWD_CASE(8, 1) BWD_CASE(8, 2) BWD_CASE(8, 4) BWD_CASE(8, 8) BWD_CASE(8, 16) BWD_CASE(8, 32) BWD_CASE(8, kThreads)
  BWD_CASE(64, 4) BWD_CASE(64, 8) BWD_CASE(64, 16) BWD_CASE(64, 32)
#undef BWD_CASE
  return cudaErrorInvalidValue;
}

template <typename T, int MA, int L>
static cudaError_t persistent_one(int grid, cudaStream_t s, PersistArgs<T> a, int *occ) {
  auto kern = persistent_kernel<T, MA, L>;
  if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, kThreads, 0);
  if (grid == 1) {
    kern<<<1, kThreads, 0, s>>>(a);
    return cudaGetLastError();
  }
  void *args[] = {&a};
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(kThreads), args, 0, s);
}

template <typename T>
cudaError_t launch_persistent(int maxa, int lanes, int grid, cudaStream_t s, PersistArgs<T> a, int *occ) {
#define P_CASE(MA, L) \
  if (maxa == MA && lanes == L) return persistent_one<T, MA, L>(grid, s, a, occ);
  P_CASE(4, 1) P_CASE(4, 2) P_CASE(4, 4) P_CASE(4, 8) P_CASE(4, 16) P_CASE(4, 32)
  P_CASE(8, 1) P_CASE(8, 2) P_CASE(8, 4) P_CASE(8, 8) P_CASE(8, 16) P_CASE(8, 32)
  P_CASE(64, 4) P_CASE(64, 8) P_CASE(64, 16) P_CASE(64, 32)
#undef P_CASE
  return cudaErrorInvalidValue;
}

}  // namespace cfr
