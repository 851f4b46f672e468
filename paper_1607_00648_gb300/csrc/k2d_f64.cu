// Hot-path kernel instantiations: 2D, double.
#include "launch_impl.cuh"
#include "sweep_pair.cuh"

#define MG_SWEEP_27(DIM, T) sweep_b<DIM, T, 27>(a, op, amode, s);
#define MG_TRANSFER_27(DIM, T) if (Lc.B == 9 && Lf.B == 27) transfer_b<DIM, T, 9, 27>(Lc, Lf, r, pmode, in, out, ph, ps, s, li, nl, zc); else transfer_b<DIM, T, 27, 27>(Lc, Lf, r, pmode, in, out, ph, ps, s, li, nl, zc);
MG_INSTANTIATE_LAUNCHERS(2, double)

namespace mg {
void launch_sweep_pair_2d_f64(SweepArgs<double> a, int amode, cudaStream_t s) {
  const int64_t nb = a.L.n_bricks;
  const int B = a.L.B;  // 27, or 9 (2D level 2)
  const int R = B == 9 ? (nb >= 152 ? 9 : 3) : (nb >= 152 ? 27 : (nb * 3 >= 152 ? 9 : 3));
  a.R = R;
  const dim3 grid(static_cast<unsigned>(nb), static_cast<unsigned>(B / R));
#define MG_SP(AM)                                                                      \
  do {                                                                                 \
    if (B == 9) {                                                                      \
      if (R == 9) launch_pdl(k_sweep_pair<double, AM, 9, 9>, grid, 256, 0, s, a);          \
      else launch_pdl(k_sweep_pair<double, AM, 3, 9>, grid, 256, 0, s, a);                 \
    } else if (R == 27) launch_pdl(k_sweep_pair<double, AM, 27>, grid, 256, 0, s, a);       \
    else if (R == 9) launch_pdl(k_sweep_pair<double, AM, 9>, grid, 256, 0, s, a);           \
    else launch_pdl(k_sweep_pair<double, AM, 3>, grid, 256, 0, s, a);                       \
  } while (0)
  if (amode == 1) MG_SP(1);
  else MG_SP(0);
#undef MG_SP
}
}  // namespace mg
