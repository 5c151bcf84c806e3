// Backward-level kernel instances, P32 (see kernels.cuh).
#include "launch_impl.cuh"
namespace cfr {
template cudaError_t launch_bwd_level<float>(int, int, int, cudaStream_t, GameView, StateView<float>, LevelWork, int, int, int, int);
}
