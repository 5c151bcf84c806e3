// Persistent-kernel instances, P32 (see kernels.cuh).
#include "launch_impl.cuh"
namespace cfr {
template cudaError_t launch_persistent<float>(int, int, int, cudaStream_t, PersistArgs<float>, int *);
}
