// Hot-path kernel instantiations: 2D, float.
#include "launch_impl.cuh"

#define MG_SWEEP_27(DIM, T) sweep_b<DIM, T, 27>(a, op, amode, s);
#define MG_TRANSFER_27(DIM, T) if (Lc.B == 9 && Lf.B == 27) transfer_b<DIM, T, 9, 27>(Lc, Lf, r, pmode, in, out, ph, ps, s, li, nl, zc); else transfer_b<DIM, T, 27, 27>(Lc, Lf, r, pmode, in, out, ph, ps, s, li, nl, zc);
MG_INSTANTIATE_LAUNCHERS(2, float)
