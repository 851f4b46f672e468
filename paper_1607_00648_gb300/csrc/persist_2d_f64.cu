// Persistent cooperative solve kernels: 2D, FP64 path.
#include "persist.cuh"

namespace mg {
template cudaError_t persist_launch_fp64<2>(const PSolve<double>*, int, int, size_t, cudaStream_t, int*);
}  // namespace mg
