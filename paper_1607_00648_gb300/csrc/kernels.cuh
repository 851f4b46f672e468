// Hot-path kernels: in-situ stencil sweeps (A2-A4), restriction (A5), prolongation
// (A6), hanging interpolation (A7) and reductions, templated on dimension,
// arithmetic type and delta storage.
#pragma once

#include "device.cuh"

namespace mg {

enum SweepOp { kJacobi = 0, kResidual = 1 };

template <typename T>
struct SweepArgs {
  LevelDesc L;
  const T* u;
  const T* b;
  T* out;
  const T* eps;         // cell coefficients (cell slots)
  const void* ahat;     // A_hat planes (3^d per vertex) or nullptr
  const float* ascale;  // per-vertex scale of 16-bit codes
  T omega;
  double* partial;      // per-CTA partial sum of r^2 (residual op), nullable
};

// Deterministic CTA reduction of one double per thread into partial[blockIdx.x].
__device__ __forceinline__ void block_reduce_store(double v, double* partial) {
  __shared__ double warp_sums[kBlock / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_sums[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kBlock / 32; ++w) s += warp_sums[w];
    partial[blockIdx.x] = s;
  }
}

// One CTA per brick.  The brick's vertex values with a one-vertex halo and the
// coefficients of all cells touching the brick are staged in shared memory;
// each DoF vertex then rebuilds its 3^d stencil from the 2^d adjacent cells
// (element-wise split of Sect. 4, summed per Hamming class), adds the stored
// delta A_hat on coarse levels (Sect. 5), and applies either the damped
// Jacobi update (Alg. 1) or the residual b - A u.
template <int DIM, typename T, int AMODE, int OP>
__global__ void __launch_bounds__(kBlock) k_sweep(SweepArgs<T> a) {
  constexpr int N3 = cpow(3, DIM);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const LevelDesc& L = a.L;
  const int B = L.B, Bu = B + 2, Be = B + 1;
  const int nu_tile = DIM == 2 ? Bu * Bu : Bu * Bu * Bu;
  const int ne_tile = DIM == 2 ? Be * Be : Be * Be * Be;
  T* su = reinterpret_cast<T*>(smem_raw);
  T* se = su + nu_tile;
  const int64_t brick = blockIdx.x;
  const int32_t* bn = L.brick_nbr + brick * N3;

  // vertex values, local coordinates -1 .. B
  for (int t = threadIdx.x; t < nu_tile; t += kBlock) {
    int rem = t, nidx = 0, mul = 1, lm = 1;
    int64_t li = 0;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      int l = rem % Bu - 1;
      rem /= Bu;
      const int o = l < 0 ? -1 : (l >= B ? 1 : 0);
      l -= o * B;
      nidx += (o + 1) * mul;
      mul *= 3;
      li += static_cast<int64_t>(l) * lm;
      lm *= B;
    }
    const int32_t nb = bn[nidx];
    su[t] = nb >= 0 ? a.u[static_cast<int64_t>(nb) * L.S + li] : T(0);
  }
  // cell coefficients, local cell coordinates -1 .. B-1
  for (int t = threadIdx.x; t < ne_tile; t += kBlock) {
    int rem = t, nidx = 0, mul = 1, lm = 1;
    int64_t li = 0;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      int l = rem % Be - 1;
      rem /= Be;
      const int o = l < 0 ? -1 : 0;
      l -= o * B;
      nidx += (o + 1) * mul;
      mul *= 3;
      li += static_cast<int64_t>(l) * lm;
      lm *= B;
    }
    const int32_t nb = bn[nidx];
    se[t] = nb >= 0 ? a.eps[static_cast<int64_t>(nb) * L.S + li] : T(0);
  }
  __syncthreads();

  const int nloc = brick_vol<DIM>(B);
  const T hscale = DIM == 3 ? static_cast<T>(L.h) : T(1);
  double part = 0.0;
  for (int s = threadIdx.x; s < nloc; s += kBlock) {
    const int64_t slot = brick * L.S + s;
    T res = T(0);
    if (is_dof(L.vflags[slot])) {
      int x[DIM];
      int rem = s;
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        x[i] = rem % B;
        rem /= B;
      }
      int cu = 0, ce = 0, su_mul = 1, se_mul = 1;
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        cu += (x[i] + 1) * su_mul;
        ce += (x[i] + 1) * se_mul;
        su_mul *= Bu;
        se_mul *= Be;
      }
      // per Hamming-class accumulators: sum over offsets of (sum of eps of the
      // cells shared by v and v+o) * u(v+o)
      T acc[DIM + 1];
#pragma unroll
      for (int c = 0; c <= DIM; ++c) acc[c] = T(0);
      T es_centre = T(0);
#pragma unroll
      for (int k = 0; k < N3; ++k) {
        int o[DIM];
        int ham = 0, kk = k;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          o[i] = kk % 3 - 1;
          kk /= 3;
          ham += o[i] != 0;
        }
        if (elem_k(DIM, ham) == 0.0) continue;
        T es = T(0);
#pragma unroll
        for (int e = 0; e < (1 << DIM); ++e) {
          bool ok = true;
          int cidx = ce, m = 1;
#pragma unroll
          for (int i = 0; i < DIM; ++i) {
            const int ei = (e >> i) & 1;
            const int t = ei + o[i];
            ok = ok && t >= 0 && t <= 1;
            cidx -= ei * m;
            m *= Be;
          }
          if (ok) es += se[cidx];
        }
        int uidx = cu, m = 1;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          uidx += o[i] * m;
          m *= Bu;
        }
        acc[ham] = fma(es, su[uidx], acc[ham]);
        if (ham == 0) es_centre = es;
      }
      T Au = T(0);
#pragma unroll
      for (int c = 0; c <= DIM; ++c)
        if (elem_k(DIM, c) != 0.0) Au = fma(static_cast<T>(elem_k(DIM, c)), acc[c], Au);
      Au *= hscale;
      T D = static_cast<T>(elem_k(DIM, 0)) * es_centre * hscale;
      if constexpr (AMODE != 0) {
#pragma unroll
        for (int k = 0; k < N3; ++k) {
          int uidx = cu, m = 1, kk = k;
#pragma unroll
          for (int i = 0; i < DIM; ++i) {
            uidx += (kk % 3 - 1) * m;
            kk /= 3;
            m *= Bu;
          }
          const T d = load_delta<AMODE, T>(a.ahat, a.ascale, (brick * N3 + k) * L.S + s, slot);
          Au = fma(d, su[uidx], Au);
          if (k == N3 / 2) D += d;
        }
      }
      const T r = a.b[slot] - Au;
      if constexpr (OP == kJacobi) {
        res = su[cu] + a.omega * r / D;
      } else {
        res = r;
        part += static_cast<double>(r) * static_cast<double>(r);
      }
    }
    a.out[slot] = res;
  }
  if constexpr (OP == kResidual) {
    if (a.partial) block_reduce_store(part, a.partial);
  }
}

// P(V, o) = P_dlin(o) + P_hat_V(o), o in [-2,2]^d lexicographic (5^d planes on the coarse level)
template <int DIM, int PMODE, typename T>
__device__ __forceinline__ T p_entry(const LevelDesc& Lc, const void* phat, const float* pscale, int64_t cs,
                                     const int* o) {
  constexpr int N5 = cpow(5, DIM);
  double w = 1.0;
  int k = 0, m = 1;
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    w *= wlin1(o[i]);
    k += (o[i] + 2) * m;
    m *= 5;
  }
  T p = static_cast<T>(w);
  if constexpr (PMODE != 0) p += load_delta<PMODE, T>(phat, pscale, plane_index(Lc, cs, k, N5), cs);
  return p;
}

// b_c(V) = sum_o P(V,o) r_f(3V + o): restriction with R = P^T (Sect. 4.4).
// One thread per coarse slot; zero on non-DoF coarse slots.
template <int DIM, typename T, int PMODE>
__global__ void __launch_bounds__(kBlock) k_restrict(LevelDesc Lc, LevelDesc Lf, const T* rf, T* bc,
                                                       const void* phat, const float* pscale) {
  const int64_t cs = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (cs >= Lc.n_slots) return;
  int X[DIM];
  if (!coords_of<DIM>(Lc, cs, X) || !is_dof(Lc.vflags[cs])) {
    bc[cs] = T(0);
    return;
  }
  constexpr int N5 = cpow(5, DIM);
  T acc = T(0);
#pragma unroll 5
  for (int k = 0; k < N5; ++k) {
    int o[DIM], y[DIM];
    int kk = k;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      o[i] = kk % 5 - 2;
      kk /= 5;
      y[i] = 3 * X[i] + o[i];
    }
    const int64_t fs = slot_of<DIM>(Lf, y);
    if (fs < 0) continue;
    acc = fma(p_entry<DIM, PMODE, T>(Lc, phat, pscale, cs, o), rf[fs], acc);
  }
  bc[cs] = acc;
}

// u_f(v) += sum over coarse parents V of P(V, v - 3V) e_c(V) (coarse-grid
// correction of Alg. 1).  One thread per fine slot; non-DoF slots untouched.
template <int DIM, typename T, int PMODE>
__global__ void __launch_bounds__(kBlock) k_prolong(LevelDesc Lc, LevelDesc Lf, const T* ec, T* uf,
                                                      const void* phat, const float* pscale) {
  const int64_t fs = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (fs >= Lf.n_slots) return;
  int x[DIM];
  if (!coords_of<DIM>(Lf, fs, x) || !is_dof(Lf.vflags[fs])) return;
  int lo[DIM], cnt[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    lo[i] = x[i] / 3;
    cnt[i] = (x[i] % 3 == 0) ? 1 : 2;
  }
  T acc = T(0);
#pragma unroll
  for (int e = 0; e < (1 << DIM); ++e) {
    int X[DIM], o[DIM];
    bool ok = true;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      const int ei = (e >> i) & 1;
      if (ei >= cnt[i]) ok = false;
      X[i] = lo[i] + ei;
      o[i] = x[i] - 3 * X[i];
    }
    if (!ok) continue;
    const int64_t cs = slot_of<DIM>(Lc, X);
    if (cs < 0 || !is_dof(Lc.vflags[cs])) continue;
    acc = fma(p_entry<DIM, PMODE, T>(Lc, phat, pscale, cs, o), ec[cs], acc);
  }
  uf[fs] += acc;
}

// u_f on HANGING slots = d-linear interpolant of the coarser level (Sect. 3, rule 2)
template <int DIM, typename T>
__global__ void __launch_bounds__(kBlock) k_hanging(LevelDesc Lf, const int32_t* hang_idx, const double* hang_w,
                                                      const T* uc, T* uf) {
  const int64_t fs = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (fs >= Lf.n_slots) return;
  if (!(Lf.vflags[fs] & MG_V_HANGING)) return;
  T acc = T(0);
#pragma unroll
  for (int e = 0; e < (1 << DIM); ++e) {
    const int32_t c = hang_idx[fs * (1 << DIM) + e];
    if (c >= 0) acc = fma(static_cast<T>(hang_w[fs * (1 << DIM) + e]), uc[c], acc);
  }
  uf[fs] = acc;
}

// sum of partial[0..n) in a fixed order by one CTA -> *out
__global__ void __launch_bounds__(kBlock) k_reduce_partials(const double* partial, int64_t n, double* out);

}  // namespace mg
