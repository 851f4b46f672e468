// Batched-solve kernel instantiations: 3D, float.
#include "batch_kernels.cuh"

#define MG_BSWEEP_27(DIM, T) bsweep_b<DIM, T, 9>(ba, g, op, amc, src, dst, s);
#define MG_BTRANSFER_27(DIM, T) btransfer_b<DIM, T, 9, 9>(ba, g, r, pm, s);
MG_BATCH_INSTANTIATE(3, float)
