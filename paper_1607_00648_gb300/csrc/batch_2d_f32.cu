// Batched-solve kernel instantiations: 2D, float.
#include "batch_kernels.cuh"
#include "sweep_pair.cuh"

#define MG_BSWEEP_27(DIM, T) bsweep_b<DIM, T, 27>(ba, g, op, amc, src, dst, s);
#define MG_BTRANSFER_27(DIM, T) if (g.BC == 9 && g.BF == 27) btransfer_b<DIM, T, 9, 27>(ba, g, r, pm, s); else btransfer_b<DIM, T, 27, 27>(ba, g, r, pm, s);
MG_BATCH_INSTANTIATE(2, float)

namespace mg {
template <int AMC, int B>
__global__ void __launch_bounds__(256) k_bsweep_pair(BatchArgs<float> ba, const int4* items, int src, int dst) {
  const int4 it = items[blockIdx.x];
  const int p = it.x, l = it.y;
  if (!ba.active[p]) return;
  const PLevel<float>& P = ba.lv[p * kMaxLevels + l];
  const bool finest = l == ba.Lp[p];
  SweepArgs<float> a{};
  a.L = P.d;
  a.u = bvec(ba, P, p, l, src);
  a.b = finest ? ba.bfin[p] : P.b;
  a.out = bvec(ba, P, p, l, dst);
  a.eps = P.eps;
  a.ahat = P.ahat;
  a.ascale = P.ascale;
  a.omega = ba.omega;
  a.R = B;  // whole bricks
  if (finest)
    sweep_pair_item<float, 0, B, B>(a, it.z, 0);
  else
    sweep_pair_item<float, AMC, B, B>(a, it.z, 0);
}

void blaunch_sweep_pair_2d_f32(const BatchArgs<float>& ba, const BatchGroup& g, int amc, int src, int dst,
                               cudaStream_t s) {
  const unsigned grid = static_cast<unsigned>(g.count);
#define MG_BP(B)                                                                    \
  do {                                                                              \
    if (amc == 2) k_bsweep_pair<2, B><<<grid, 256, 0, s>>>(ba, g.items, src, dst);  \
    else if (amc == 3) k_bsweep_pair<3, B><<<grid, 256, 0, s>>>(ba, g.items, src, dst); \
    else k_bsweep_pair<0, B><<<grid, 256, 0, s>>>(ba, g.items, src, dst);           \
  } while (0)
  if (g.B == 9) MG_BP(9);
  else MG_BP(27);
#undef MG_BP
}
}  // namespace mg
