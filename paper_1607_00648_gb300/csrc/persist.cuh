// Persistent solve: the whole FP64 solve, or the whole mixed FP64-refinement solve,
// in one cooperative launch.  Every phase of a V-cycle (a sweep of one level, a
// restriction, the coarsest solve, a prolongation) is spread over the resident
// grid and followed by a grid-wide barrier, so a cycle costs no kernel launches
// and the convergence test needs no host round trip.  The residual norm of the
// current iterate is a by-product of the first Jacobi sweep of the next cycle
// (that sweep computes b - A u anyway and writes to the other buffer), so no
// separate residual pass is spent on the test.
#pragma once

#include <cooperative_groups.h>

#include "kernels.cuh"

namespace mg {

constexpr int kMaxLevels = 9;

template <typename T>
struct PLevel {
  LevelDesc d;
  const T* eps;
  const void* ahat;
  const float* ascale;
  const void* phat;  // P_hat for the transfer to the next finer level (stored here)
  const float* pscale;
  T* u;
  T* b;
  T* r;
  T* t;
  int R;
  int nitems;  // sweep work items (brick, slab)
};

template <typename T>
struct PSolve {
  int L, c, nu1, nu2;
  T omega;
  PLevel<T> lv[kMaxLevels];
  const double* chol;
  int n_c;
  const int32_t* c_slots;
  double* partial;   // >= max nitems
  double* hist;      // relative residual after each cycle / refinement step
  int hist_cap;
  int* out_int;      // [0] cycles, [1] outer steps, [2] status (0 ok, 1 not converged, 2 non-finite, 3 diverged)
  double* out_dbl;   // [0] r0, [1] final relative residual
  double tol;
  int max_cycles;
  // mixed path
  PLevel<double> f64;  // finest FP64 level (u = solution, b = rhs, r = FP64 residual)
  double inv_count;    // 1 / n_dofs
};

// deterministic sum of partial[0..n) by one CTA (every CTA may call it; all get the same value)
__device__ __forceinline__ double cta_sum_partials(const double* partial, int n) {
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += static_cast<const volatile double*>(partial)[i];
  const double s = block_sum(t);
  __shared__ double bcast;
  if (threadIdx.x == 0) bcast = s;
  __syncthreads();
  const double v = bcast;
  __syncthreads();
  return v;
}

template <int DIM, typename T, int AM, int OP>
__device__ __forceinline__ double sweep_any_b(const SweepArgs<T>& a, int64_t brick, int slab, unsigned char* smem) {
  if constexpr (DIM == 2) {
    if (a.L.B == 27) return sweep_item<2, T, AM, OP, 27>(a, brick, slab, smem);
    if (a.L.B == 9) return sweep_item<2, T, AM, OP, 9>(a, brick, slab, smem);
    return sweep_item<2, T, AM, OP, 3>(a, brick, slab, smem);
  } else {
    if (a.L.B == 9) return sweep_item<3, T, AM, OP, 9>(a, brick, slab, smem);
    return sweep_item<3, T, AM, OP, 3>(a, brick, slab, smem);
  }
}

// One sweep of a level over the grid; partial sums of r^2 per item when `partial`.
template <int DIM, typename T, int AM, int OP>
__device__ void phase_sweep(const PLevel<T>& P, const T* u, const T* b, T* out, T omega, double* partial,
                            unsigned char* smem) {
  SweepArgs<T> a{};
  a.L = P.d;
  a.u = u;
  a.b = b;
  a.out = out;
  a.eps = P.eps;
  a.ahat = P.ahat;
  a.ascale = P.ascale;
  a.omega = omega;
  a.R = P.R;
  const int per = P.d.B / P.R;
  for (int it = blockIdx.x; it < P.nitems; it += gridDim.x) {
    const double part = sweep_any_b<DIM, T, AM, OP>(a, it / per, it % per, smem);
    if (partial) {
      const double s = block_sum(part);
      if (threadIdx.x == 0) partial[it] = s;
    }
  }
}

template <int DIM, typename T, int PM>
__device__ void phase_restrict(const PLevel<T>& C, const PLevel<T>& F, const T* rf, T* bc, T* uc_zero) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t cs = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; cs < C.d.n_slots; cs += stride) {
    if constexpr (DIM == 2) {
      if (C.d.B == 27) restrict_one<2, T, PM, 27, 27>(C.d, F.d, rf, bc, C.phat, C.pscale, cs);
      else if (C.d.B == 9) restrict_one<2, T, PM, 9, 27>(C.d, F.d, rf, bc, C.phat, C.pscale, cs);
      else restrict_one<2, T, PM, 3, 9>(C.d, F.d, rf, bc, C.phat, C.pscale, cs);
    } else {
      if (C.d.B == 9) restrict_one<3, T, PM, 9, 9>(C.d, F.d, rf, bc, C.phat, C.pscale, cs);
      else restrict_one<3, T, PM, 3, 9>(C.d, F.d, rf, bc, C.phat, C.pscale, cs);
    }
    uc_zero[cs] = T(0);
  }
}

template <int DIM, typename T, int PM>
__device__ void phase_prolong(const PLevel<T>& C, const PLevel<T>& F, const T* ec, T* uf) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t fs = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; fs < F.d.n_slots; fs += stride) {
    if constexpr (DIM == 2) {
      if (C.d.B == 27) prolong_one<2, T, PM, 27, 27>(C.d, F.d, ec, uf, C.phat, C.pscale, fs);
      else if (C.d.B == 9) prolong_one<2, T, PM, 9, 27>(C.d, F.d, ec, uf, C.phat, C.pscale, fs);
      else prolong_one<2, T, PM, 3, 9>(C.d, F.d, ec, uf, C.phat, C.pscale, fs);
    } else {
      if (C.d.B == 9) prolong_one<3, T, PM, 9, 9>(C.d, F.d, ec, uf, C.phat, C.pscale, fs);
      else prolong_one<3, T, PM, 3, 9>(C.d, F.d, ec, uf, C.phat, C.pscale, fs);
    }
  }
}

// coarsest level by the FP64 Cholesky factor, on CTA 0
template <typename T>
__device__ void phase_coarse(const double* Lm, int n, const int32_t* c_slots, const T* b, T* u) {
  __shared__ double y[64];
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int i = 0; i < n; ++i) {
    double v = static_cast<double>(b[c_slots[i]]);
    for (int j = 0; j < i; ++j) v -= Lm[i * n + j] * y[j];
    y[i] = v / Lm[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = y[i];
    for (int j = i + 1; j < n; ++j) v -= Lm[j * n + i] * y[j];
    y[i] = v / Lm[i * n + i];
  }
  for (int i = 0; i < n; ++i) u[c_slots[i]] = static_cast<T>(y[i]);
}

template <typename T>
__device__ void phase_copy(T* dst, const T* src, int64_t n) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

// The rest of a V(nu1, nu2) cycle on the finest level after its first Jacobi sweep
// (which went u -> t); ends with the new iterate in u.
template <int DIM, typename T, int AMC, int PM>
__device__ void cycle_rest(const PSolve<T>& p, unsigned char* smem) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  // pre-smoothing (remaining sweeps) and restriction, level by level downwards
  for (int l = p.L; l > p.c; --l) {
    const PLevel<T>& F = p.lv[l];
    T* cur = F.u;
    T* oth = F.t;
    int first = 0;
    if (l == p.L) {  // first sweep already done: iterate is in t
      cur = F.t;
      oth = F.u;
      first = 1;
    }
    for (int k = first; k < p.nu1; ++k) {
      if (l == p.L)
        phase_sweep<DIM, T, 0, kJacobi>(F, cur, F.b, oth, p.omega, nullptr, smem);
      else
        phase_sweep<DIM, T, AMC, kJacobi>(F, cur, F.b, oth, p.omega, nullptr, smem);
      grid.sync();
      T* tt = cur;
      cur = oth;
      oth = tt;
    }
    if (cur != F.u) {
      phase_copy<T>(F.u, cur, F.d.n_slots);
      grid.sync();
    }
    if (l == p.L)
      phase_sweep<DIM, T, 0, kResidual>(F, F.u, F.b, F.r, T(0), nullptr, smem);
    else
      phase_sweep<DIM, T, AMC, kResidual>(F, F.u, F.b, F.r, T(0), nullptr, smem);
    grid.sync();
    phase_restrict<DIM, T, PM>(p.lv[l - 1], F, F.r, p.lv[l - 1].b, p.lv[l - 1].u);
    grid.sync();
  }
  phase_coarse<T>(p.chol, p.n_c, p.c_slots, p.lv[p.c].b, p.lv[p.c].u);
  grid.sync();
  for (int l = p.c + 1; l <= p.L; ++l) {
    const PLevel<T>& F = p.lv[l];
    phase_prolong<DIM, T, PM>(p.lv[l - 1], F, p.lv[l - 1].u, F.u);
    grid.sync();
    T* cur = F.u;
    T* oth = F.t;
    for (int k = 0; k < p.nu2; ++k) {
      if (l == p.L)
        phase_sweep<DIM, T, 0, kJacobi>(F, cur, F.b, oth, p.omega, nullptr, smem);
      else
        phase_sweep<DIM, T, AMC, kJacobi>(F, cur, F.b, oth, p.omega, nullptr, smem);
      grid.sync();
      T* tt = cur;
      cur = oth;
      oth = tt;
    }
    if (cur != F.u) {
      phase_copy<T>(F.u, cur, F.d.n_slots);
      grid.sync();
    }
  }
}

// FP64 solve from u = 0 (the caller zeroes u): V-cycles until the relative residual
// drops below tol (Sect. 4.1; ||r||_2 / ||r_0||_2 over the DoFs, u_0 = 0).
template <int DIM, int AMC, int PM>
__global__ void __launch_bounds__(kBlock) k_persist_fp64(const PSolve<double>* __restrict__ pp) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char smem[];
  const PSolve<double>& p = *pp;
  const PLevel<double>& F = p.lv[p.L];
  double r0 = 0.0, rel = 1.0;
  int cycles = 0, status = 1;
  for (;;) {
    // first pre-smoothing sweep; its b - A u is the residual of the current iterate
    phase_sweep<DIM, double, 0, kJacobiNorm>(F, F.u, F.b, F.t, p.omega, p.partial, smem);
    grid.sync();
    const double n2 = cta_sum_partials(p.partial, F.nitems);
    if (cycles == 0) {
      r0 = sqrt(n2);
      rel = r0 > 0.0 ? 1.0 : 0.0;
    } else {
      rel = sqrt(n2) / r0;
      if (blockIdx.x == 0 && threadIdx.x == 0 && cycles - 1 < p.hist_cap) p.hist[cycles - 1] = rel;
    }
    if (!(rel == rel) || !(r0 == r0) || isinf(rel)) {
      status = 2;
      break;
    }
    if (rel > 1e6) {
      status = 3;
      break;
    }
    if (rel <= p.tol) {
      status = 0;
      break;
    }
    if (cycles >= p.max_cycles) {
      status = 1;
      break;
    }
    cycle_rest<DIM, double, AMC, PM>(p, smem);
    ++cycles;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    p.out_int[0] = cycles;
    p.out_int[1] = cycles;
    p.out_int[2] = status;
    p.out_dbl[0] = r0;
    p.out_dbl[1] = rel;
  }
}

// Mixed solve: FP64 iterative refinement (residual, scaling, update in FP64 on the
// finest level) around FP32 V-cycles whose coarse operators are rebuilt from 16-bit
// delta codes.  An inner solve stops at the first sweep whose FP32 residual is below
// max(1e-5, 0.3 tol / rel) of its start, or when it stagnates (ratio > 0.9 per cycle
// averaged over 8 cycles).
template <int DIM, int AMC, int PM>
__global__ void __launch_bounds__(kBlock) k_persist_mixed(const PSolve<float>* __restrict__ pp) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char smem[];
  const PSolve<float>& p = *pp;
  const PLevel<double>& G = p.f64;
  const PLevel<float>& F = p.lv[p.L];
  const int64_t n = G.d.n_slots;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t gtid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  double r0 = 0.0, rel = 1.0, sigma = 0.0;
  int cycles = 0, outer = 0, status = 1;
  for (;;) {
    // u64 += sigma e32 (sigma = 0 on the first step), then r64 = b - A u64 in FP64
    if (outer > 0)
      for (int64_t i = gtid; i < n; i += stride) G.u[i] = fma(sigma, static_cast<double>(F.u[i]), G.u[i]);
    grid.sync();
    phase_sweep<DIM, double, 0, kResidual>(G, G.u, G.b, G.r, 0.0, p.partial, smem);
    grid.sync();
    const double n2 = cta_sum_partials(p.partial, G.nitems);
    if (outer == 0) {
      r0 = sqrt(n2);
      rel = r0 > 0.0 ? 1.0 : 0.0;
    } else {
      rel = sqrt(n2) / r0;
      if (blockIdx.x == 0 && threadIdx.x == 0 && outer - 1 < p.hist_cap) p.hist[outer - 1] = rel;
    }
    ++outer;
    if (!(rel == rel) || isinf(rel)) {
      status = 2;
      break;
    }
    if (rel > 1e6) {
      status = 3;
      break;
    }
    if (rel <= p.tol) {
      status = 0;
      break;
    }
    if (cycles >= p.max_cycles) {
      status = 1;
      break;
    }
    // correction equation A e = r / sigma in FP32
    sigma = sqrt(n2 * p.inv_count);
    const double inv = sigma > 0.0 ? 1.0 / sigma : 0.0;
    for (int64_t i = gtid; i < n; i += stride) {
      F.b[i] = static_cast<float>(G.r[i] * inv);
      F.u[i] = 0.0f;
    }
    grid.sync();
    const double target = fmax(1e-5, 0.3 * p.tol / rel);
    double inner0 = 0.0, prev8 = 0.0;
    for (int k = 0;; ++k) {
      phase_sweep<DIM, float, 0, kJacobiNorm>(F, F.u, F.b, F.t, static_cast<float>(p.omega), p.partial, smem);
      grid.sync();
      const double m2 = sqrt(cta_sum_partials(p.partial, F.nitems));
      if (k == 0) {
        inner0 = m2;
        prev8 = m2;
      }
      const double irel = inner0 > 0.0 ? m2 / inner0 : 0.0;
      if (k > 0 && (irel <= target || !(m2 == m2))) break;
      if (k > 0 && k % 8 == 0) {  // stagnation: less than 10% gained over 8 cycles
        if (m2 > 0.9 * prev8) break;
        prev8 = m2;
      }
      if (cycles >= p.max_cycles) break;
      cycle_rest<DIM, float, AMC, PM>(p, smem);
      ++cycles;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    p.out_int[0] = cycles;
    p.out_int[1] = outer;
    p.out_int[2] = status;
    p.out_dbl[0] = r0;
    p.out_dbl[1] = rel;
  }
}

// ---- host launch helpers (instantiated in persist_2d.cu / persist_3d.cu) ----

template <typename K, typename P>
static cudaError_t coop_launch(K kernel, const P* p, size_t smem, cudaStream_t s, int* grid_out) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  if (per_sm > 4) per_sm = 4;
  const int grid = sms * per_sm;
  *grid_out = grid;
  void* args[] = {const_cast<P**>(&p)};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kernel), dim3(grid), dim3(kBlock), args, smem, s);
}

template <int DIM>
cudaError_t persist_launch_fp64(const PSolve<double>* p, int amc, int pm, size_t smem, cudaStream_t s, int* grid) {
  if (amc == 1 && pm == 1) return coop_launch(k_persist_fp64<DIM, 1, 1>, p, smem, s, grid);
  if (amc == 1) return coop_launch(k_persist_fp64<DIM, 1, 0>, p, smem, s, grid);
  if (pm == 1) return coop_launch(k_persist_fp64<DIM, 0, 1>, p, smem, s, grid);
  return coop_launch(k_persist_fp64<DIM, 0, 0>, p, smem, s, grid);
}

template <int DIM>
cudaError_t persist_launch_mixed(const PSolve<float>* p, int amc, int pm, size_t smem, cudaStream_t s, int* grid) {
  if (amc == 2 && pm == 2) return coop_launch(k_persist_mixed<DIM, 2, 2>, p, smem, s, grid);
  if (amc == 3 && pm == 3) return coop_launch(k_persist_mixed<DIM, 3, 3>, p, smem, s, grid);
  if (amc == 2 && pm == 0) return coop_launch(k_persist_mixed<DIM, 2, 0>, p, smem, s, grid);
  if (amc == 3 && pm == 0) return coop_launch(k_persist_mixed<DIM, 3, 0>, p, smem, s, grid);
  if (amc == 0 && pm == 2) return coop_launch(k_persist_mixed<DIM, 0, 2>, p, smem, s, grid);
  if (amc == 0 && pm == 3) return coop_launch(k_persist_mixed<DIM, 0, 3>, p, smem, s, grid);
  return coop_launch(k_persist_mixed<DIM, 0, 0>, p, smem, s, grid);
}

}  // namespace mg
