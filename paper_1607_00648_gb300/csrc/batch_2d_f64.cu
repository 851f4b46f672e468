// Batched-solve kernel instantiations: 2D, double.
#include "batch_kernels.cuh"

#define MG_BSWEEP_27(DIM, T) bsweep_b<DIM, T, 27>(ba, g, op, amc, src, dst, s);
#define MG_BTRANSFER_27(DIM, T) if (g.BC == 9 && g.BF == 27) btransfer_b<DIM, T, 9, 27>(ba, g, r, pm, s); else btransfer_b<DIM, T, 27, 27>(ba, g, r, pm, s);
MG_BATCH_INSTANTIATE(2, double)
