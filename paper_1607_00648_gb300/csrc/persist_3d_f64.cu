// Persistent cooperative solve kernels: 3D, FP64 path.
#include "persist.cuh"

namespace mg {
template cudaError_t persist_launch_fp64<3>(const PSolve<double>*, int, int, size_t, cudaStream_t, int*);
}  // namespace mg
