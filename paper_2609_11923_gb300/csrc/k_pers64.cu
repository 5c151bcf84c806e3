// Persistent-kernel instances, P64 (see kernels.cuh).
#include "launch_impl.cuh"
namespace cfr {
template cudaError_t launch_persistent<double>(int, int, int, cudaStream_t, PersistArgs<double>, int *);
}
