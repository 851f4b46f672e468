// Persistent cooperative solve kernels: 3D, mixed-precision path.
#include "persist.cuh"

namespace mg {
template cudaError_t persist_launch_mixed<3>(const PSolve<float>*, int, int, size_t, cudaStream_t, int*);
}  // namespace mg
