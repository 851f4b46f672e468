// Persistent cooperative solve kernels: 2D, mixed-precision path.
#include "persist.cuh"

namespace mg {
template cudaError_t persist_launch_mixed<2>(const PSolve<float>*, int, int, size_t, cudaStream_t, int*);
}  // namespace mg
