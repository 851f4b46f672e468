// Hot-path kernel instantiations: 3D, double.
#include "launch_impl.cuh"

#define MG_SWEEP_27(DIM, T) sweep_b<DIM, T, 9>(a, op, amode, s);
#define MG_TRANSFER_27(DIM, T) transfer_b<DIM, T, 9, 9>(Lc, Lf, r, pmode, in, out, ph, ps, s, li, nl, zc);
MG_INSTANTIATE_LAUNCHERS(3, double)
