// A batch step in one persistent launch: the work of every problem of the batch (its
// sweeps by brick, transfers and copies by chunk of slots, coarsest solve and
// convergence test) is one device work queue in phase order, and each problem carries a
// progress counter instead of the per-phase launches of the lockstep schedule.
//
// The CTAs of one launch take queue entries in order (an atomic ticket).  An entry of
// problem p in its phase k waits until p's counter shows all of p's entries of phases
// < k done, runs, and counts itself done.  Waits are only on entries with smaller
// tickets, all of them already taken by CTAs that run to completion, so the queue always
// makes progress; problems advance independently, so the small problems of a batch do
// not wait at every phase for the largest ones.  Every wait is bounded: past the limit
// the CTA raises the error word, and every later entry is skipped (still counted), so
// the launch always ends.
#pragma once

#include "batch_kernels.cuh"

namespace mg {

enum QOp : int {
  kQSweep = 0,    // Jacobi / Jacobi + norm / residual sweep of one brick (FP64 or FP32)
  kQCopy = 1,     // dst = src on a chunk of kBlock slots
  kQRestrict = 2, // b_c = R r_f on a chunk of kBlock coarse slots (and u_c = 0 there)
  kQProlong = 3,  // u_f += P u_c on a chunk of kBlock fine slots
  kQCoarse = 4,   // the problem's coarsest level by its FP64 Cholesky factor
  kQCheck = 5,    // the problem's convergence test from the norm sweep's partial sums
  kQUpdate = 6,   // mixed: u64 += sigma e32 on a chunk of finest slots
  kQScale = 7     // mixed: b32 = r64 / sigma, e32 = 0 on a chunk of finest slots
};

// one queue entry; op packs the QOp (bits 0-3), the arithmetic type (bit 4: FP32), the
// sweep operation (bits 8-11) and the source / destination vector selectors (bits
// 12-15 / 16-19)
struct QItem {
  int op, p, l, idx;
  int need;  // entries of problem p in earlier phases (its counter must reach this)
  int aux;   // norm / residual sweeps: the partial-sum slot
};

struct QueueArgs {
  BatchArgs<double> b64;
  BatchArgs<float> b32;  // mixed batches
  BatchState st;
  const int* cp;                 // coarsest level per problem
  const double* const* chol;     // coarsest Cholesky factor per problem
  const int32_t* const* cslots;  // coarsest DoF slots per problem
  const int* nc;                 // coarsest DoFs per problem
  const QItem* items;
  int n_items;
  unsigned* head;  // next ticket
  int* prog;       // per problem: entries done
  int* err;        // 0, or 2: a wait ran out (the launch skipped the rest)
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// one brick of a sweep with the level's compile-time brick edge and the batch's delta mode
template <int DIM, typename T, int AM, int OP>
__device__ __forceinline__ double q_sweep_b(const SweepArgs<T>& a, int brick, unsigned char* smem) {
  const int B = a.L.B;
  if constexpr (std::is_same<T, float>::value) {
    if ((DIM == 2 && B == 27) || (DIM == 3 && B == 9)) return sweep_col_item<DIM, T, AM, OP>(a, brick, 0, smem);
  }
  if (B == 3) return sweep_item<DIM, T, AM, OP, 3>(a, brick, 0, smem);
  if constexpr (DIM == 2) {
    if (B == 9) return sweep_item<DIM, T, AM, OP, 9>(a, brick, 0, smem);
    return sweep_item<DIM, T, AM, OP, 27>(a, brick, 0, smem);
  } else {
    return sweep_item<DIM, T, AM, OP, 9>(a, brick, 0, smem);
  }
}

template <int DIM, typename T, int AMC>
__device__ void q_sweep(const BatchArgs<T>& ba, const QItem& it, unsigned char* smem) {
  const int p = it.p, l = it.l;
  if (!ba.active[p]) return;
  const PLevel<T>& P = ba.lv[p * kMaxLevels + l];
  const bool finest = l == ba.Lp[p];
  const int op = (it.op >> 8) & 15, src = (it.op >> 12) & 15, dst = (it.op >> 16) & 15;
  SweepArgs<T> a{};
  a.L = P.d;
  a.u = bvec(ba, P, p, l, src);
  a.b = finest ? ba.bfin[p] : P.b;
  a.out = bvec(ba, P, p, l, dst);
  a.eps = P.eps;
  a.ahat = P.ahat;
  a.ascale = P.ascale;
  a.omega = ba.omega;
  a.R = P.d.B;  // whole bricks
  double part = 0.0;
#define MG_QS(AM)                                                                               \
  do {                                                                                          \
    if (op == kJacobi) part = q_sweep_b<DIM, T, AM, kJacobi>(a, it.idx, smem);                   \
    else if constexpr (std::is_same<T, double>::value) {                                        \
      if (op == kJacobiNorm) part = q_sweep_b<DIM, T, AM, kJacobiNorm>(a, it.idx, smem);         \
      else part = q_sweep_b<DIM, T, AM, kResidual>(a, it.idx, smem);                             \
    } else {                                                                                    \
      part = q_sweep_b<DIM, T, AM, kResidual>(a, it.idx, smem);                                  \
    }                                                                                           \
  } while (0)
  if (finest || AMC == 0) MG_QS(0); else MG_QS(AMC);
#undef MG_QS
  if (op != kJacobi && ba.partial && it.aux >= 0) {  // norm sweeps only: cycle residuals carry no slot
    const double s = block_sum(part);
    if (threadIdx.x == 0) ba.partial[it.aux] = s;
  }
}

template <int DIM, typename T, int PM>
__device__ void q_transfer(const BatchArgs<T>& ba, const QItem& it, bool restrict_op) {
  const int p = it.p;
  if (!ba.active[p]) return;
  if (restrict_op) {
    const PLevel<T>& C = ba.lv[p * kMaxLevels + it.l];
    const PLevel<T>& F = ba.lv[p * kMaxLevels + it.l + 1];
    for (int t = threadIdx.x; t < kBlock; t += blockDim.x) {
      const int64_t cs = static_cast<int64_t>(it.idx) * kBlock + t;
      if (cs >= C.d.n_slots) break;
      if (C.d.B == 3 && F.d.B == 9) restrict_one<DIM, T, PM, 3, 9>(C.d, F.d, F.r, C.b, C.phat, C.pscale, cs);
      else if (C.d.B == 9 && F.d.B == 9) restrict_one<DIM, T, PM, 9, 9>(C.d, F.d, F.r, C.b, C.phat, C.pscale, cs);
      else if constexpr (DIM == 2) {
        if (C.d.B == 9) restrict_one<DIM, T, PM, 9, 27>(C.d, F.d, F.r, C.b, C.phat, C.pscale, cs);
        else restrict_one<DIM, T, PM, 27, 27>(C.d, F.d, F.r, C.b, C.phat, C.pscale, cs);
      }
      C.u[cs] = T(0);
    }
  } else {
    const PLevel<T>& C = ba.lv[p * kMaxLevels + it.l - 1];
    const PLevel<T>& F = ba.lv[p * kMaxLevels + it.l];
    T* uf = it.l == ba.Lp[p] ? ba.ufin[p] : F.u;
    for (int t = threadIdx.x; t < kBlock; t += blockDim.x) {
      const int64_t fs = static_cast<int64_t>(it.idx) * kBlock + t;
      if (fs >= F.d.n_slots) break;
      if (C.d.B == 3 && F.d.B == 9) prolong_one<DIM, T, PM, 3, 9>(C.d, F.d, C.u, uf, C.phat, C.pscale, fs);
      else if (C.d.B == 9 && F.d.B == 9) prolong_one<DIM, T, PM, 9, 9>(C.d, F.d, C.u, uf, C.phat, C.pscale, fs);
      else if constexpr (DIM == 2) {
        if (C.d.B == 9) prolong_one<DIM, T, PM, 9, 27>(C.d, F.d, C.u, uf, C.phat, C.pscale, fs);
        else prolong_one<DIM, T, PM, 27, 27>(C.d, F.d, C.u, uf, C.phat, C.pscale, fs);
      }
    }
  }
}

template <typename T>
__device__ void q_copy(const BatchArgs<T>& ba, const QItem& it) {
  const int p = it.p, l = it.l;
  if (!ba.active[p]) return;
  const PLevel<T>& P = ba.lv[p * kMaxLevels + l];
  const int src = (it.op >> 12) & 15, dst = (it.op >> 16) & 15;
  for (int t = threadIdx.x; t < kBlock; t += blockDim.x) {
    const int64_t i = static_cast<int64_t>(it.idx) * kBlock + t;
    if (i >= P.d.n_slots) break;
    bvec(ba, P, p, l, dst)[i] = bvec(ba, P, p, l, src)[i];
  }
}

template <typename T>
__device__ void q_coarse(const QueueArgs& q, const BatchArgs<T>& ba, int p) {
  if (threadIdx.x == 0 && ba.active[p]) bcoarse_one<T>(ba.lv, q.cp, q.chol, q.cslots, q.nc, p);
}

__device__ inline void q_update_scale(const QueueArgs& q, const QItem& it, bool update) {
  const int p = it.p;
  if (!q.st.active[p]) return;
  const PLevel<double>& G = q.b64.lv[p * kMaxLevels + it.l];
  const double sg = q.st.sigma[p];
  double* u64 = q.b64.ufin[p];
  float* e32 = q.b32.ufin[p];
  float* b32 = const_cast<float*>(q.b32.bfin[p]);
  for (int t = threadIdx.x; t < kBlock; t += blockDim.x) {
    const int64_t i = static_cast<int64_t>(it.idx) * kBlock + t;
    if (i >= G.d.n_slots) break;
    if (update) {
      u64[i] = fma(sg, static_cast<double>(e32[i]), u64[i]);
    } else {
      b32[i] = static_cast<float>(sg > 0.0 ? G.r[i] / sg : 0.0);
      e32[i] = 0.0f;
    }
  }
}

template <int DIM, int AMC64, int PM64, int AMC32, int PM32>
__global__ void __launch_bounds__(128, 6) k_bpersist(QueueArgs q) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_t, s_ok;
  for (;;) {
    __syncthreads();  // the previous entry's work is done before the next ticket
    if (threadIdx.x == 0) s_t = static_cast<int>(atomicAdd(q.head, 1u));
    __syncthreads();
    const int t = s_t;
    if (t >= q.n_items) return;
    const QItem it = q.items[t];
    if (threadIdx.x == 0) {
      int ok = 1;
      unsigned spins = 0;
      while (ld_acquire_gpu(q.prog + it.p) < it.need) {
        if (*static_cast<volatile int*>(q.err)) {
          ok = 0;
          break;
        }
        if (++spins > (1u << 24)) {  // about a second of waiting: give up
          atomicExch(q.err, 2);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
      s_ok = ok && !*static_cast<volatile int*>(q.err);
    }
    __syncthreads();
    if (s_ok) {
      const int op = it.op & 15;
      const bool f32 = (it.op >> 4) & 1;
      switch (op) {
        case kQSweep:
          if (f32) q_sweep<DIM, float, AMC32>(q.b32, it, smem);
          else q_sweep<DIM, double, AMC64>(q.b64, it, smem);
          break;
        case kQCopy:
          if (f32) q_copy<float>(q.b32, it); else q_copy<double>(q.b64, it);
          break;
        case kQRestrict:
        case kQProlong:
          if (f32) q_transfer<DIM, float, PM32>(q.b32, it, op == kQRestrict);
          else q_transfer<DIM, double, PM64>(q.b64, it, op == kQRestrict);
          break;
        case kQCoarse:
          if (f32) q_coarse<float>(q, q.b32, it.p); else q_coarse<double>(q, q.b64, it.p);
          break;
        case kQCheck:
          if (threadIdx.x == 0) bcheck_one(q.st, it.p);
          break;
        default:
          q_update_scale(q, it, op == kQUpdate);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // this entry's results before its count
      atomicAdd(q.prog + it.p, 1);
    }
  }
}

// the dynamic shared memory an entry may need: the largest sweep tile of the dimension
template <int DIM>
inline size_t bpersist_smem() {
  if constexpr (DIM == 2) return sweep_tile_bytes<2, double>(27, 27);
  return std::max(sweep_tile_bytes<3, double>(9, 9), sweep_tile_bytes<3, float>(9, 9, true));
}

// launch of one step's queue (instantiated in batch_persist.cu); modes: the batch's
// delta / transfer modes (FP64 A_hat, FP64 P_hat, FP32 A_hat, FP32 P_hat)
template <int DIM>
cudaError_t bpersist_launch(const QueueArgs& q, int amc64, int pm64, int amc32, int pm32, cudaStream_t s);

}  // namespace mg
