// Backward-level kernel instances, P64 (see kernels.cuh).
#include "launch_impl.cuh"
namespace cfr {
template cudaError_t launch_bwd_level<double>(int, int, int, cudaStream_t, GameView, StateView<double>, LevelWork, int, int, int, int, bool);
}
