// Batched-iteration kernel instances, FP32 (see batch.cuh).
#include "k_batch.cuh"
namespace cfr {
template cudaError_t launch_batch_iterate<float>(int, int, int, int, int, cudaStream_t, const InstDesc *);
}
