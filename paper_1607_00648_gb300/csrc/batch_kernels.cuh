// Kernels of the batched solve: one launch per phase and brick edge, one CTA per
// work item of any problem in the batch (see batch.cu for the phase schedule).
#pragma once

#include <type_traits>

#include "kernels.cuh"
#include "persist.cuh"
#include "sweep_fast.cuh"

namespace mg {

enum BatchSel { kSelU = 0, kSelT = 1, kSelR = 2 };

template <typename T>
struct BatchArgs {
  const PLevel<T>* lv;   // [p * kMaxLevels + l]
  T* const* ufin;        // finest-level iterate per problem
  const T* const* bfin;  // finest-level right-hand side per problem
  const int* Lp;         // finest level per problem
  const int* active;     // 1 while problem p still iterates
  double* partial;       // per item of a norm phase (nullable)
  T omega;
  // paired smoothing of a lockstep FP32 cycle: the iterate of 2D levels of brick edge 27
  // or 9 sits in t between pre- and post-smoothing, so the prolongation adds into t there
  int pair_t = 0;
};

// per-problem solve state of a batch (device arrays of n entries)
struct BatchState {
  int* active;
  int* cycles;
  int* status;  // 0 converged, 1 not converged, 2 non-finite, 3 diverged
  double* r0;
  double* rel;
  double* sigma;
  const double* invc;
  int* n_active;
  const int2* prange;
  const double* partial;
  const double* tol;     // per problem
  const int* max_cycles; // per problem
  int inc;
  int n;
};

// convergence test of problem p from the partial sums of its norm sweep: first call
// (r0 < 0) records r0; retires the problem on convergence, a non-finite or diverged
// residual, or max_cycles; otherwise counts the cycles, stores sigma (mixed scaling)
// and counts the problem active
__device__ inline void bcheck_one(const BatchState& s, int p) {
  if (!s.active[p]) return;
  double n2 = 0.0;
  for (int i = s.prange[p].x; i < s.prange[p].y; ++i) n2 += s.partial[i];
  double rel;
  if (s.r0[p] < 0.0) {
    s.r0[p] = sqrt(n2);
    rel = s.r0[p] > 0.0 ? 1.0 : 0.0;
  } else {
    rel = sqrt(n2) / s.r0[p];
  }
  s.rel[p] = rel;
  int st = -1;
  if (!(rel == rel) || isinf(rel)) st = 2;
  else if (rel <= s.tol[p]) st = 0;
  else if (rel > 1e6) st = 3;
  else if (s.cycles[p] >= s.max_cycles[p]) st = 1;
  if (st >= 0) {
    s.status[p] = st;
    s.active[p] = 0;
    return;
  }
  s.cycles[p] += s.inc;
  s.sigma[p] = sqrt(n2 * s.invc[p]);
  atomicAdd(s.n_active, 1);
}

// coarsest level of problem p by its FP64 Cholesky factor (one thread)
template <typename T>
__device__ void bcoarse_one(const PLevel<T>* lv, const int* cp, const double* const* chol,
                            const int32_t* const* cslots, const int* nc, int p) {
  const PLevel<T>& P = lv[p * kMaxLevels + cp[p]];
  const double* Lm = chol[p];
  const int32_t* cs = cslots[p];
  const int m = nc[p];
  double y[64];
  for (int i = 0; i < m; ++i) {
    double v = static_cast<double>(P.b[cs[i]]);
    for (int j = 0; j < i; ++j) v -= Lm[i * m + j] * y[j];
    y[i] = v / Lm[i * m + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double v = y[i];
    for (int j = i + 1; j < m; ++j) v -= Lm[j * m + i] * y[j];
    y[i] = v / Lm[i * m + i];
  }
  for (int i = 0; i < m; ++i) P.u[cs[i]] = static_cast<T>(y[i]);
}

// a launch group: items of one phase sharing the brick edge(s)
struct BatchGroup {
  int B, BC, BF;   // sweep: B; transfer: coarse / fine brick edge
  int4* items;     // device
  int count;
  int part_off;    // offset of this group's items in the partial buffer (norm phases)
};

template <typename T>
__device__ __forceinline__ T* bvec(const BatchArgs<T>& ba, const PLevel<T>& P, int p, int l, int sel) {
  if (sel == kSelU) return l == ba.Lp[p] ? ba.ufin[p] : P.u;
  if (sel == kSelT) return P.t;
  return P.r;
}

// item = (problem, level, brick, slab)
template <int DIM, typename T, int AMC, int OP, int B>
__global__ void __launch_bounds__(kBlock) k_bsweep(BatchArgs<T> ba, const int4* items, int part_off, int src,
                                                     int dst) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int4 it = items[blockIdx.x];
  const int p = it.x, l = it.y;
  if (!ba.active[p]) return;
  const PLevel<T>& P = ba.lv[p * kMaxLevels + l];
  const bool finest = l == ba.Lp[p];
  SweepArgs<T> a{};
  a.L = P.d;
  a.u = bvec(ba, P, p, l, src);
  a.b = finest ? ba.bfin[p] : P.b;
  a.out = bvec(ba, P, p, l, dst);
  a.eps = P.eps;
  a.ahat = P.ahat;
  a.ascale = P.ascale;
  a.omega = ba.omega;
  a.R = P.R;
  double part;
  if (finest)
    part = sweep_item<DIM, T, 0, OP, B>(a, it.z, it.w, smem);
  else
    part = sweep_item<DIM, T, AMC, OP, B>(a, it.z, it.w, smem);
  if constexpr (OP == kJacobiNorm || OP == kResidual) {
    if (ba.partial) {
      const double s = block_sum(part);
      if (threadIdx.x == 0) ba.partial[part_off + blockIdx.x] = s;
    }
  }
}

// FP32 at the fine brick edges (2D 27, 3D 9): the column kernels, 128 threads
template <int DIM, typename T, int AMC, int OP>
__global__ void __launch_bounds__(128, 6) k_bsweep_col(BatchArgs<T> ba, const int4* items, int part_off, int src,
                                                         int dst) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int4 it = items[blockIdx.x];
  const int p = it.x, l = it.y;
  if (!ba.active[p]) return;
  const PLevel<T>& P = ba.lv[p * kMaxLevels + l];
  const bool finest = l == ba.Lp[p];
  SweepArgs<T> a{};
  a.L = P.d;
  a.u = bvec(ba, P, p, l, src);
  a.b = finest ? ba.bfin[p] : P.b;
  a.out = bvec(ba, P, p, l, dst);
  a.eps = P.eps;
  a.ahat = P.ahat;
  a.ascale = P.ascale;
  a.omega = ba.omega;
  a.R = P.R;
  double part;
  if (finest)
    part = sweep_col_item<DIM, T, 0, OP>(a, it.z, it.w, smem);
  else
    part = sweep_col_item<DIM, T, AMC, OP>(a, it.z, it.w, smem);
  if constexpr (OP == kJacobiNorm || OP == kResidual) {
    if (ba.partial) {
      const double s = block_sum(part);
      if (threadIdx.x == 0) ba.partial[part_off + blockIdx.x] = s;
    }
  }
}

// item = (problem, coarse level, chunk of kBlock coarse slots); also zeroes the
// coarse iterate (the coarse-grid correction starts from 0)
template <int DIM, typename T, int PM, int BC, int BF>
__global__ void __launch_bounds__(kBlock) k_brestrict(BatchArgs<T> ba, const int4* items) {
  const int4 it = items[blockIdx.x];
  const int p = it.x, lc = it.y;
  if (!ba.active[p]) return;
  const PLevel<T>& C = ba.lv[p * kMaxLevels + lc];
  const PLevel<T>& F = ba.lv[p * kMaxLevels + lc + 1];
  const int64_t cs = static_cast<int64_t>(it.z) * kBlock + threadIdx.x;
  if (cs >= C.d.n_slots) return;
  restrict_one<DIM, T, PM, BC, BF>(C.d, F.d, F.r, C.b, C.phat, C.pscale, cs);
  C.u[cs] = T(0);
}

// item = (problem, fine level, chunk of kBlock fine slots)
template <int DIM, typename T, int PM, int BC, int BF>
__global__ void __launch_bounds__(kBlock) k_bprolong(BatchArgs<T> ba, const int4* items) {
  const int4 it = items[blockIdx.x];
  const int p = it.x, lf = it.y;
  if (!ba.active[p]) return;
  const PLevel<T>& C = ba.lv[p * kMaxLevels + lf - 1];
  const PLevel<T>& F = ba.lv[p * kMaxLevels + lf];
  const int64_t fs = static_cast<int64_t>(it.z) * kBlock + threadIdx.x;
  if (fs >= F.d.n_slots) return;
  T* uf = (DIM == 2 && ba.pair_t && (F.d.B == 27 || F.d.B == 9)) ? F.t : (lf == ba.Lp[p] ? ba.ufin[p] : F.u);
  prolong_one<DIM, T, PM, BC, BF>(C.d, F.d, C.u, uf, C.phat, C.pscale, fs);
}

// item = (problem, level, chunk): dst = src
template <typename T>
__global__ void __launch_bounds__(kBlock) k_bcopy(BatchArgs<T> ba, const int4* items, int src, int dst) {
  const int4 it = items[blockIdx.x];
  const int p = it.x, l = it.y;
  if (!ba.active[p]) return;
  const PLevel<T>& P = ba.lv[p * kMaxLevels + l];
  const int64_t i = static_cast<int64_t>(it.z) * kBlock + threadIdx.x;
  if (i >= P.d.n_slots) return;
  bvec(ba, P, p, l, dst)[i] = bvec(ba, P, p, l, src)[i];
}

template <int DIM, typename T>
void blaunch_sweep(const BatchArgs<T>& ba, const BatchGroup& g, int op, int amc, int src, int dst, cudaStream_t s);

// two Jacobi sweeps src -> dst per item (whole bricks) of a 2D FP32 group of brick edge 27
// or 9 (sweep_pair.cuh; bit for bit two k_bsweep_col / k_bsweep sweeps)
void blaunch_sweep_pair_2d_f32(const BatchArgs<float>& ba, const BatchGroup& g, int amc, int src, int dst,
                               cudaStream_t s);

template <int DIM, typename T>
void blaunch_transfer(const BatchArgs<T>& ba, const BatchGroup& g, bool restrict_op, int pm, cudaStream_t s);

// ---- launcher bodies (instantiated in batch_{2,3}d_{f64,f32}.cu) ----

template <int DIM, typename T, int B>
static void bsweep_b(const BatchArgs<T>& ba, const BatchGroup& g, int op, int amc, int src, int dst, cudaStream_t s) {
  constexpr int VOL = DIM == 2 ? B * B : B * B * B;
  constexpr bool col = std::is_same<T, float>::value && ((DIM == 2 && B == 27) || (DIM == 3 && B == 9));
  int threads = ((VOL + 31) / 32) * 32;
  if (threads > kBlock) threads = kBlock;
  const size_t smem = col ? (DIM == 2 ? 0 : sweep_tile_bytes<DIM, T>(B, B, true)) : sweep_tile_bytes<DIM, T>(B, B);
  const unsigned grid = static_cast<unsigned>(g.count);
#define MG_BS(AM, OP)                                                                                 \
  do {                                                                                                \
    if constexpr (col)                                                                                \
      k_bsweep_col<DIM, T, AM, OP><<<grid, 128, smem, s>>>(ba, g.items, g.part_off, src, dst);         \
    else                                                                                              \
      k_bsweep<DIM, T, AM, OP, B><<<grid, threads, smem, s>>>(ba, g.items, g.part_off, src, dst);      \
  } while (0)
#define MG_BS_OPS(AM)                          \
  do {                                         \
    if (op == kJacobi) MG_BS(AM, kJacobi);     \
    else if (op == kJacobiNorm) MG_BS(AM, kJacobiNorm); \
    else MG_BS(AM, kResidual);                 \
  } while (0)
  if constexpr (std::is_same<T, double>::value) {
    if (amc == 1) MG_BS_OPS(1); else MG_BS_OPS(0);
  } else {
    if (amc == 2) MG_BS_OPS(2); else if (amc == 3) MG_BS_OPS(3); else MG_BS_OPS(0);
  }
#undef MG_BS_OPS
#undef MG_BS
}

template <int DIM, typename T, int BC, int BF>
static void btransfer_b(const BatchArgs<T>& ba, const BatchGroup& g, bool r, int pm, cudaStream_t s) {
  const unsigned grid = static_cast<unsigned>(g.count);
#define MG_BT(PM)                                                                       \
  do {                                                                                  \
    if (r) k_brestrict<DIM, T, PM, BC, BF><<<grid, kBlock, 0, s>>>(ba, g.items);        \
    else k_bprolong<DIM, T, PM, BC, BF><<<grid, kBlock, 0, s>>>(ba, g.items);           \
  } while (0)
  if constexpr (std::is_same<T, double>::value) {
    if (pm == 1) MG_BT(1); else MG_BT(0);
  } else {
    if (pm == 2) MG_BT(2); else if (pm == 3) MG_BT(3); else MG_BT(0);
  }
#undef MG_BT
}

}  // namespace mg

#define MG_BATCH_INSTANTIATE(DIM, T)                                                                          \
  namespace mg {                                                                                              \
  template <>                                                                                                 \
  void blaunch_sweep<DIM, T>(const BatchArgs<T>& ba, const BatchGroup& g, int op, int amc, int src, int dst,  \
                             cudaStream_t s) {                                                                \
    if (g.B == 3) bsweep_b<DIM, T, 3>(ba, g, op, amc, src, dst, s);                                           \
    else if (g.B == 9) bsweep_b<DIM, T, 9>(ba, g, op, amc, src, dst, s);                                      \
    else MG_BSWEEP_27(DIM, T)                                                                                 \
  }                                                                                                           \
  template <>                                                                                                 \
  void blaunch_transfer<DIM, T>(const BatchArgs<T>& ba, const BatchGroup& g, bool r, int pm, cudaStream_t s) { \
    if (g.BC == 3 && g.BF == 9) btransfer_b<DIM, T, 3, 9>(ba, g, r, pm, s);                                    \
    else if (g.BC == 9 && g.BF == 9) btransfer_b<DIM, T, 9, 9>(ba, g, r, pm, s);                               \
    else MG_BTRANSFER_27(DIM, T)                                                                              \
  }                                                                                                           \
  }
