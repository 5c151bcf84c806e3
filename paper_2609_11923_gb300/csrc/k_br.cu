// Exact best-response kernel instances (see kernels.cuh).
#include "launch_impl.cuh"
namespace cfr {
cudaError_t launch_br_level(int maxa, int lanes, int grid, cudaStream_t s, GameView g, const double2 *reach2,
                            const double *sbs, double2 *vb, double *vavg, LevelWork w, int nb_chance) {
#define BR_CASE(MA, L)                                                                        \
  if (maxa == MA && lanes == L) {                                                             \
    br_level_kernel<MA, L><<<grid, kThreads, 0, s>>>(g, reach2, sbs, vb, vavg, w, nb_chance); \
    return cudaGetLastError();                                                                \
  }
  BR_CASE(4, 1) BR_CASE(4, 2) BR_CASE(4, 4) BR_CASE(4, 8) BR_CASE(4, 16) BR_CASE(4, 32)
  BR_CASE(8, 1) BR_CASE(8, 2) BR_CASE(8, 4) BR_CASE(8, 8) BR_CASE(8, 16) BR_CASE(8, 32)
  BR_CASE(64, 4) BR_CASE(64, 8) BR_CASE(64, 16) BR_CASE(64, 32)
#undef BR_CASE
  return cudaErrorInvalidValue;
}
}  // namespace cfr
