// Hierarchy, setup sequence, V-cycle and solve drivers, and the C-ABI entry points
// of libmg (everything except the grid builder).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "boxmg3.cuh"
#include "bpa.cuh"
#include "hier.h"
#include "internal.h"
#include "kernels.cuh"
#include "persist.cuh"
#include "rap3.cuh"
#include "setup.cuh"

namespace mg {

extern template cudaError_t persist_launch_fp64<2>(const PSolve<double>*, int, int, size_t, cudaStream_t, int*);
extern template cudaError_t persist_launch_fp64<3>(const PSolve<double>*, int, int, size_t, cudaStream_t, int*);
extern template cudaError_t persist_launch_mixed<2>(const PSolve<float>*, int, int, size_t, cudaStream_t, int*);
extern template cudaError_t persist_launch_mixed<3>(const PSolve<float>*, int, int, size_t, cudaStream_t, int*);

// ----------------------------------------------------------------------------- small kernels

// binary64 -> (h, l) float pair rounded to nearest twice (h = fl32(v), l = fl32(v - h)),
// packed into a binary64 container (low word h, high word l) for the float-float sweeps
__global__ void k_split_pairs(int64_t n, const double* v, double* out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const double x = v[i];
  const float h = __double2float_rn(x);
  const float l = __double2float_rn(x - static_cast<double>(h));
  out[i] = __hiloint2double(__float_as_int(l), __float_as_int(h));
}

__global__ void k_leaf_eps(LevelDesc L, const uint8_t* cflags, const double* eps_in, double* eps) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (s >= L.n_slots) return;
  const uint8_t f = cflags[s];
  eps[s] = ((f & MG_C_EXISTS) && !(f & MG_C_REFINED)) ? eps_in[s] : 0.0;
}

__global__ void __launch_bounds__(kBlock) k_reduce_partials(const double* partial, int64_t n, double* out) {
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kBlock) v += partial[i];
  __shared__ double warp_sums[kBlock / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) s += warp_sums[w];
    out[0] = s;
  }
}

__global__ void k_to_f32(int64_t n, const double* in, float* out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (i < n) out[i] = static_cast<float>(in[i]);
}

// b32 = fl32(r64 / sigma), sigma = sqrt(norm2 / n_dofs) (keeps the FP32 correction O(1))
__global__ void k_scale_to_f32(int64_t n, const double* r, const double* norm2, double inv_count, float* out,
                               double* sigma_out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  const double sigma = sqrt(norm2[0] * inv_count);
  const double inv = sigma > 0.0 ? 1.0 / sigma : 0.0;
  if (i == 0) sigma_out[0] = sigma;
  if (i < n) out[i] = static_cast<float>(r[i] * inv);
}

// u64 += sigma * e32 (iterative-refinement update; e32 is zero off the DoFs)
__global__ void k_update_f64(int64_t n, double* u, const float* e, const double* sigma) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (i < n) u[i] = fma(sigma[0], static_cast<double>(e[i]), u[i]);
}

// ---- composite (adaptive) grid kernels: level t = L - 1 of a tree refined to L in part

// u_t(V) = u_L(3V) at refined level-t DoFs (Sect. 3, rule 1: injection)
template <typename T>
__global__ void k_inject(LevelDesc Lt, const int32_t* child, const T* uL, T* ut) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (s >= Lt.n_slots) return;
  const uint8_t f = Lt.vflags[s];
  if (is_dof(f) && (f & MG_V_REFINED)) ut[s] = uL[child[s]];
}

// additive cycle (Alg. 2), element-wise steps: d = omega D^-1 r on DoFs (zero elsewhere)
// and u += d; the negated copy of a vector; injection u_c = I u_f on every coarse DoF
__global__ void k_add_correct(LevelDesc L, const double* dinv, const double* r, double* d, double* u) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (s >= L.n_slots) return;
  const double c = is_dof(L.vflags[s]) ? dinv[s] * r[s] : 0.0;
  d[s] = c;
  u[s] += c;
}
// BPX (Alg. 3) ascent on a level above the coarsest: d = omega D^-1 r on DoFs; the
// c-points (every coordinate a multiple of 3) skip their own update, keep d = 0 and
// leave the skipped update in r for the injection i_{l-1} = I d_l
template <int DIM>
__global__ void k_bpx_correct(LevelDesc L, const double* dinv, double* r, double* d, double* u) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (s >= L.n_slots) return;
  const double c = is_dof(L.vflags[s]) ? dinv[s] * r[s] : 0.0;
  int x[DIM];
  bool cp = coords_of<DIM>(L, s, x);
#pragma unroll
  for (int i = 0; i < DIM; ++i) cp = cp && x[i] % 3 == 0;
  r[s] = c;
  d[s] = cp ? 0.0 : c;
  if (!cp) u[s] += c;
}
// BPX descent at the c-points: x_f += i_c at the fine slot coinciding with each coarse
// DoF (the prolongation of x = d - i left P i out there, and P is the injection at
// c-points), for the correction d and the iterate u
__global__ void k_bpx_cpoints(LevelDesc Lc, const int32_t* child, const double* ic, double* df, double* uf) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (s >= Lc.n_slots || !is_dof(Lc.vflags[s]) || child[s] < 0) return;
  df[child[s]] += ic[s];
  uf[child[s]] += ic[s];
}
__global__ void k_sub(int64_t n, const double* x, const double* y, double* z) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (s < n) z[s] = x[s] - y[s];
}
__global__ void k_negate(int64_t n, const double* x, double* y) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (s < n) y[s] = -x[s];
}
__global__ void k_inject_level(LevelDesc Lc, const int32_t* child, const double* uf, double* uc) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (s >= Lc.n_slots) return;
  uc[s] = (is_dof(Lc.vflags[s]) && child[s] >= 0) ? uf[child[s]] : 0.0;
}

// coarse-correction right-hand side off the refined vertices: the level-t residual
// at unrefined DoFs, zero at non-DoFs (the restriction fills the refined DoFs)
template <typename T>
__global__ void k_compose_rhs(LevelDesc Lt, const T* r_t, T* rhs) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (s >= Lt.n_slots) return;
  const uint8_t f = Lt.vflags[s];
  if (!is_dof(f))
    rhs[s] = T(0);
  else if (!(f & MG_V_REFINED))
    rhs[s] = r_t[s];
}

// u_t += e_t at unrefined level-t DoFs
template <typename T>
__global__ void k_add_unrefined(LevelDesc Lt, const T* e, T* ut) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (s >= Lt.n_slots) return;
  const uint8_t f = Lt.vflags[s];
  if (is_dof(f) && !(f & MG_V_REFINED)) ut[s] += e[s];
}

// r_t = 0 off the unrefined level-t DoFs, and the sum of r_t^2 over them into
// *norm2 (fixed-order CTA partials, grid-stride over the level)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_masked_norm(LevelDesc Lt, T* r, double* partial, unsigned* counter,
                                                          double* norm2) {
  double part = 0.0;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * kBlock;
  for (int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x; s < Lt.n_slots; s += stride) {
    const uint8_t f = Lt.vflags[s];
    if (is_dof(f) && !(f & MG_V_REFINED)) {
      const double v = static_cast<double>(r[s]);
      part += v * v;
    } else {
      r[s] = T(0);
    }
  }
  store_partial_and_finish(part, partial, counter, norm2);
}

__global__ void k_sum2(const double* a, const double* b, double* out) { out[0] = a[0] + b[0]; }

// Round an FP64 value to the nearest (ties to even) BF16 (FMT 1) or FP16 (FMT 2)
// value, from the IEEE 754 definition of the target format: the quantum is
// 2^(max(E, Emin) - fraction bits) for the leading-bit exponent E.
template <int FMT>
__device__ uint16_t round_to_16(double t) {
  constexpr int frac = FMT == 1 ? 7 : 10;
  constexpr int emin = FMT == 1 ? -126 : -14;
  constexpr int bias = FMT == 1 ? 127 : 15;
  const uint16_t sign = t < 0.0 ? 0x8000u : 0u;
  const double a = fabs(t);
  if (a == 0.0) return sign;
  int e;
  frexp(a, &e);
  int E = e - 1;
  if (E < emin) E = emin;
  const double m = rint(ldexp(a, frac - E));  // integer mantissa incl. leading bit, ties to even
  long long mi = static_cast<long long>(m);
  if (mi >= (1LL << (frac + 1))) {  // rounding carried into the next binade
    mi >>= 1;
    ++E;
  }
  if (mi < (1LL << frac)) return sign | static_cast<uint16_t>(mi);  // subnormal (E == emin)
  return sign | static_cast<uint16_t>(((E + bias) << frac) | (mi - (1LL << frac)));
}

// per row: scale = fl32(max |delta|), codes = round_to_16(delta / scale)
template <int FMT>
__global__ void k_encode_rows(int64_t n, int K, const double* delta, uint16_t* codes, float* scale) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (i >= n) return;
  double m = 0.0;
  for (int k = 0; k < K; ++k) m = fmax(m, fabs(delta[i * K + k]));
  const float s = __double2float_rn(m);
  scale[i] = s;
  const double sd = static_cast<double>(s);
  for (int k = 0; k < K; ++k) codes[i * K + k] = sd > 0.0 ? round_to_16<FMT>(delta[i * K + k] / sd) : 0;
}

// Promotion rule of a row (Sect. 5 cancellation, the dtype counterpart of the paper's
// per-vertex choice against eps_mf): half a unit of the 16-bit format relative to the
// scale, h s (h = 2^-9 for BF16, 2^-12 for FP16), exceeds 2^-8 of the reconstructed
// diagonal |A_vv|.  Products by powers of two: the comparison is exact.
template <int FMT>
__device__ __forceinline__ bool promote_row(float sc, double diag) {
  constexpr double h = FMT == 1 ? 0x1p-9 : 0x1p-12;
  return static_cast<double>(sc) * h > 0x1p-8 * fabs(diag);
}

// codes of one row: plain 16-bit codes, or (promoted) the FP32 bit pattern of
// fl32(delta / s) split into the code (high half) and lo (low half)
template <int FMT>
__device__ __forceinline__ void put_codes(double d, double sd, bool prom, uint16_t* code, uint16_t* lo) {
  if (prom) {
    const uint32_t bits = __float_as_uint(__double2float_rn(d / sd));
    *code = static_cast<uint16_t>(bits >> 16);
    *lo = static_cast<uint16_t>(bits & 0xffffu);
  } else {
    *code = sd > 0.0 ? round_to_16<FMT>(d / sd) : 0;
    if (lo) *lo = 0;
  }
}

// per row with promotion against diag[i]: the flag is the sign of scale[i]
template <int FMT>
__global__ void k_encode_rows_promote(int64_t n, int K, const double* delta, const double* diag, uint16_t* codes,
                                      uint16_t* lo, float* scale) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (i >= n) return;
  double m = 0.0;
  for (int k = 0; k < K; ++k) m = fmax(m, fabs(delta[i * K + k]));
  const float s = __double2float_rn(m);
  const bool prom = s > 0.0f && promote_row<FMT>(s, diag[i]);
  scale[i] = prom ? -s : s;
  const double sd = static_cast<double>(s);
  for (int k = 0; k < K; ++k) put_codes<FMT>(delta[i * K + k], sd, prom, codes + i * K + k, lo + i * K + k);
}

// same on brick-major planes of a level.  promote (A_hat only): the row's reconstructed
// diagonal A_redisc + A_hat is formed from the level's coefficients (full_stencil) and
// promoted rows write their low halves n_slots * K entries after the code planes
template <int DIM, int FMT>
__global__ void k_encode_planes(LevelDesc L, int K, const double* delta, uint16_t* codes, float* scale,
                                const double* eps, int promote) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (s >= L.n_slots) return;
  double m = 0.0;
  for (int k = 0; k < K; ++k) m = fmax(m, fabs(delta[plane_index(L, s, k, K)]));
  const float sc = __double2float_rn(m);
  bool prom = false;
  if (promote && sc > 0.0f) {
    int x[DIM];
    if (coords_of<DIM>(L, s, x)) {
      double st[cpow(3, DIM)];
      full_stencil<DIM>(L, eps, delta, x, s, st);
      prom = promote_row<FMT>(sc, st[cpow(3, DIM) / 2]);
    }
  }
  scale[s] = prom ? -sc : sc;
  const double sd = static_cast<double>(sc);
  uint16_t* lo = promote ? codes + L.n_slots * K : nullptr;
  for (int k = 0; k < K; ++k) {
    const int64_t idx = plane_index(L, s, k, K);
    put_codes<FMT>(delta[idx], sd, prom, codes + idx, lo ? lo + idx : nullptr);
  }
}

// reconstructed stencils (offset-major export) and the diagonal audit (Sect. 4.3)
template <int DIM>
__global__ void k_export_stencils(LevelDesc L, const double* eps, const double* ahat, double* out, int* status,
                                  const double* aniso = nullptr) {
  constexpr int N3 = cpow(3, DIM);
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (s >= L.n_slots) return;
  int x[DIM];
  double st[N3];
  if (!coords_of<DIM>(L, s, x)) {
    if (out)
      for (int k = 0; k < N3; ++k) out[k * L.n_slots + s] = 0.0;
    return;
  }
  full_stencil<DIM>(L, eps, ahat, x, s, st, aniso);
  if (out)
    for (int k = 0; k < N3; ++k) out[k * L.n_slots + s] = st[k];
  if (status && is_dof(L.vflags[s]) && !(st[N3 / 2] > 0.0)) atomicExch(status, 2);
}

// diagonal-tensor coefficients of the finest level (d level-concatenated arrays, one per
// axis, stride n_total): the per-cell mean into eps, the deviations d_i = eps_i - mean
// into aniso (axis-major)
template <int DIM>
__global__ void k_tensor_split(LevelDesc L, const double* axes, int64_t n_total, double* eps, double* aniso) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (s >= L.n_slots) return;
  double e[DIM], m = 0.0;
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    e[i] = axes[i * n_total + s];
    m += e[i];
  }
  m /= DIM;
  eps[s] = m;
#pragma unroll
  for (int i = 0; i < DIM; ++i) aniso[i * L.n_slots + s] = e[i] - m;
}

// The anisotropic part B u of a diagonal-tensor operator on the finest level (the
// sweeps apply the per-cell mean coefficient): after a Jacobi sweep out -= dinv B u
// (FP64: omega / diag from the setup; FP32: omega / D with D from the mean coefficients;
// B has no diagonal), after a residual sweep out -= B u with the squared norm of the
// result (the sweep itself then runs without its norm).  u is the sweep's input.
template <int DIM, typename T, int OP>
__global__ void __launch_bounds__(kBlock) k_aniso_fix(LevelDesc L, const T* u, T* out, const T* aniso, const T* eps,
                                                       const double* dinv, T omega, double* partial, unsigned* counter,
                                                       double* norm2) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  double part = 0.0;
  int x[DIM];
  if (s < L.n_slots && is_dof(L.vflags[s]) && coords_of<DIM>(L, s, x)) {
    double Bu = 0.0, es = 0.0;
#pragma unroll
    for (int e = 0; e < (1 << DIM); ++e) {
      int c[DIM];
#pragma unroll
      for (int i = 0; i < DIM; ++i) c[i] = x[i] - ((e >> i) & 1);
      const int64_t cs = slot_of<DIM>(L, c);
      if (cs < 0) continue;
      double dv[DIM];
#pragma unroll
      for (int i = 0; i < DIM; ++i) dv[i] = static_cast<double>(aniso[i * L.n_slots + cs]);
      es += static_cast<double>(eps[cs]);
      // the cell's other corners: offsets o_i in {0, 1 - 2 e_i}
#pragma unroll
      for (int m = 1; m < (1 << DIM); ++m) {
        int o[DIM], y[DIM];
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          o[i] = ((m >> i) & 1) ? 1 - 2 * ((e >> i) & 1) : 0;
          y[i] = x[i] + o[i];
        }
        const double w = aniso_entry<DIM>(dv, o, L.h);
        if (w == 0.0) continue;
        const int64_t ns = slot_of<DIM>(L, y);
        if (ns >= 0) Bu += w * static_cast<double>(u[ns]);
      }
    }
    if constexpr (OP == kJacobi) {
      double f;
      if (dinv) {
        f = dinv[s];
      } else {
        const double D = DIM == 2 ? elem_k(2, 0) * es : elem_k(3, 0) * L.h * es;
        f = static_cast<double>(omega) / D;
      }
      out[s] = static_cast<T>(static_cast<double>(out[s]) - f * Bu);
    } else {
      const T r = static_cast<T>(static_cast<double>(out[s]) - Bu);
      out[s] = r;
      part = static_cast<double>(r) * static_cast<double>(r);
    }
  }
  if constexpr (OP == kResidual) {
    if (partial) store_partial_and_finish(part, partial, counter, norm2);
  }
}

// Sect. 4.3 audit of one level for the dynamic coarsest level: *fail = 1 if a DoF row
// has a non-positive diagonal or is not diagonally dominant over the unknowns (sum of
// |off-diagonal| over DoF neighbours > (1 + 1e-12) |diagonal|); entries towards
// Dirichlet vertices multiply zero and are left out
template <int DIM>
__global__ void k_audit(LevelDesc L, const double* eps, const double* ahat, int* fail) {
  constexpr int N3 = cpow(3, DIM);
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (s >= L.n_slots || !is_dof(L.vflags[s])) return;
  int x[DIM];
  if (!coords_of<DIM>(L, s, x)) return;
  double st[N3];
  full_stencil<DIM>(L, eps, ahat, x, s, st);
  double off = 0.0;
  for (int k = 0; k < N3; ++k) {
    if (k == N3 / 2) continue;
    int y[DIM], kk = k;
    for (int i = 0; i < DIM; ++i) {
      y[i] = x[i] + kk % 3 - 1;
      kk /= 3;
    }
    const int64_t ns = slot_of<DIM>(L, y);
    if (ns >= 0 && is_dof(L.vflags[ns])) off += fabs(st[k]);
  }
  const double d = st[N3 / 2];
  if (!(d > 0.0) || off > (1.0 + 1e-12) * fabs(d)) *fail = 1;
}

// dense coarsest operator over its DoFs
template <int DIM>
__global__ void k_coarse_assemble(LevelDesc L, const double* eps, const double* ahat, const int32_t* c_slots,
                                  const int32_t* c_map, int n, double* M) {
  constexpr int N3 = cpow(3, DIM);
  const int i = blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  const int64_t s = c_slots[i];
  int x[DIM];
  coords_of<DIM>(L, s, x);
  double st[N3];
  full_stencil<DIM>(L, eps, ahat, x, s, st);
  for (int j = 0; j < n; ++j) M[static_cast<int64_t>(i) * n + j] = 0.0;
  for (int k = 0; k < N3; ++k) {
    int y[DIM], kk = k;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      y[a] = x[a] + kk % 3 - 1;
      kk /= 3;
    }
    const int64_t t = slot_of<DIM>(L, y);
    if (t < 0) continue;
    const int j = c_map[t];
    if (j >= 0) M[static_cast<int64_t>(i) * n + j] = st[k];
  }
}

// in-place lower Cholesky factor of the SPD coarsest operator (one CTA); status 3 on failure
__global__ void __launch_bounds__(kBlock) k_cholesky(double* M, int n, int* status) {
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double d = M[static_cast<int64_t>(k) * n + k];
      if (!(d > 0.0)) {
        fail = 1;
      } else {
        M[static_cast<int64_t>(k) * n + k] = sqrt(d);
      }
    }
    __syncthreads();
    if (fail) break;
    const double dk = M[static_cast<int64_t>(k) * n + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += kBlock) M[static_cast<int64_t>(i) * n + k] /= dk;
    __syncthreads();
    const int m = n - k - 1;
    for (int t = threadIdx.x; t < m * m; t += kBlock) {
      const int i = k + 1 + t / m, j = k + 1 + t % m;
      if (j <= i) M[static_cast<int64_t>(i) * n + j] -= M[static_cast<int64_t>(i) * n + k] * M[static_cast<int64_t>(j) * n + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && fail) atomicExch(status, 3);
}

// u(coarsest DoFs) = A^-1 b by the Cholesky factor, in FP64 for both precisions
template <typename T>
__global__ void __launch_bounds__(kBlock) k_coarse_solve(const double* Lm, int n, const int32_t* c_slots, const T* b,
                                                           T* u) {
  extern __shared__ double y[];
  pdl_enter();
  for (int i = threadIdx.x; i < n; i += kBlock) y[i] = static_cast<double>(b[c_slots[i]]);
  __syncthreads();
  for (int k = 0; k < n; ++k) {  // L y = b
    if (threadIdx.x == 0) y[k] /= Lm[static_cast<int64_t>(k) * n + k];
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < n; i += kBlock) y[i] -= Lm[static_cast<int64_t>(i) * n + k] * y[k];
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {  // L^T x = y
    if (threadIdx.x == 0) y[k] /= Lm[static_cast<int64_t>(k) * n + k];
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += kBlock) y[i] -= Lm[static_cast<int64_t>(k) * n + i] * y[k];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += kBlock) u[c_slots[i]] = static_cast<T>(y[i]);
}

// the same for at most 32 unknowns: one thread, no barriers
template <typename T>
__global__ void k_coarse_solve_small(const double* Lm, int n, const int32_t* c_slots, const T* b, T* u) {
  pdl_enter();
  if (threadIdx.x != 0) return;
  double y[32];
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

// ----------------------------------------------------------------------------- hierarchy

#define MG_TRY_CUDA(call)                                                         \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      set_error(std::string(#call) + " failed: " + cudaGetErrorString(e_));       \
      return MG_ERR_CUDA;                                                         \
    }                                                                             \
  } while (0)

#define MG_CHECK(expr)               \
  do {                               \
    mg_status st_ = (expr);          \
    if (st_ != MG_OK) return st_;    \
  } while (0)

static mg_status last_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  return MG_OK;
}

// ---- pooled device memory and pinned slots ----

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};
std::vector<void*> g_pinned_free;
}  // namespace

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_pools[dev]) {
      cudaMemPoolProps props{};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&g_pools[dev], &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = ~0ull;
      e = cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) return e;
    }
    pool = g_pools[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

void pool_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

void* pinned_slot() {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_pinned_free.empty()) {
    constexpr size_t kSlot = 128, kSlab = 512;
    char* slab = nullptr;
    if (cudaMallocHost(&slab, kSlot * kSlab) != cudaSuccess) return nullptr;
    for (size_t i = 0; i < kSlab; ++i) g_pinned_free.push_back(slab + i * kSlot);
  }
  void* p = g_pinned_free.back();
  g_pinned_free.pop_back();
  std::memset(p, 0, 128);
  return p;
}

void pinned_release(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  g_pinned_free.push_back(p);
}

template <typename T>
static mg_status dalloc(Hier& H, T** p, size_t n) {
  *p = nullptr;
  if (n == 0) return MG_OK;
  void* q = nullptr;
  const cudaError_t e = pool_alloc(&q, n * sizeof(T), H.own);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("device allocation of ") + std::to_string(n * sizeof(T)) + " bytes: " +
              cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA;
  }
  H.allocs.push_back(q);
  MG_TRY_CUDA(cudaMemsetAsync(q, 0, n * sizeof(T), H.own));
  *p = static_cast<T*>(q);
  return MG_OK;
}

template <typename T>
static mg_status upload(Hier& H, T** p, const std::vector<T>& v) {
  MG_CHECK(dalloc(H, p, v.size()));
  if (!v.empty()) MG_TRY_CUDA(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, H.own));
  return MG_OK;
}

// device_sync: wait for all device work first (public destroy: a hierarchy may still be
// in use on any stream, as cudaFree would have waited for); the server passes false
static void free_hier(Hier* H, bool device_sync) {
  if (!H) return;
  if (device_sync) cudaDeviceSynchronize();
  H->g_cycle64.reset();
  H->g_cycle_ff.reset();
  for (auto& gr : H->g_fused)
    for (Graph& g : gr) g.reset();
  H->g_comp_ff.reset();
  H->g_outer.reset();
  H->g_inner.reset();
  H->g_comp64.reset();
  H->g_comp_outer.reset();
  H->g_comp_inner.reset();
  H->g_add.reset();
  for (void* p : H->allocs) pool_free(p, H->own);
  pinned_release(H->h_pin);
  if (H->own) cudaStreamDestroy(H->own);
  delete H;
}

void hier_release(Hier* H) { free_hier(H, false); }

static inline unsigned nblk(int64_t n) { return static_cast<unsigned>((n + kBlock - 1) / kBlock); }

static mg_status create(const Grid* g, const mg_options& o, Hier** out, int priority, bool blocking) {
  Hier* H = new (std::nothrow) Hier();
  if (!H) {
    set_error("mg_hier_create: out of host memory");
    return MG_ERR_OOM;
  }
  H->g = g;
  H->opt = o;
  H->L = g->L;
  H->c = o.coarsest_level;
  H->adaptive = !g->uniform;
  H->top = H->adaptive ? g->L - 1 : g->L;
  H->dim = g->dim;
  H->galerkin = o.coarse == MG_COARSE_GALERKIN;
  H->tensor = o.tensor_coefficients != 0;
  H->boxmg = o.transfer == MG_TRANSFER_BOXMG;
  H->mixed = o.precision != MG_PREC_FP64;
  H->fmt = o.precision == MG_PREC_MIXED_FP16 ? 2 : (o.precision == MG_PREC_MIXED_BPA ? 4 : 1);
  auto fail = [&](mg_status s) {
    free_hier(H, true);
    return s;
  };
  // public hierarchies: a blocking stream, so that work given stream NULL runs here
  // ordered with the legacy default stream as the interface's stream convention
  // promises; the server's hierarchies (only ever used on its own streams) take a
  // non-blocking one, so that their creation does not wait on unrelated work
  if (cudaStreamCreateWithPriority(&H->own, blocking ? cudaStreamDefault : cudaStreamNonBlocking, priority) !=
      cudaSuccess) {
    set_error("mg_hier_create: cudaStreamCreate failed");
    return fail(MG_ERR_CUDA);
  }
  const int d = g->dim;
  const int n3 = ipow(3, d), n5 = ipow(5, d);
  H->lv.resize(H->L + 1);
  mg_status st;
  if (d == 3 && H->galerkin && H->top > H->c && g->levels[H->top].B == 9) {
    // two-stage 3D Galerkin product: AP scratch of the largest fine level (rap3.cuh)
    H->ap3_len = static_cast<int64_t>(g->levels[H->top].n_bricks) * kApPerBrick;
    if ((st = dalloc(*H, &H->ap3, static_cast<size_t>(H->ap3_len))) != MG_OK) return fail(st);
  }
  for (int l = H->c; l <= H->L; ++l) {
    const HostLevel& hl = g->levels[l];
    DevLevel& D = H->lv[l];
    if ((st = upload(*H, &D.brick_nbr, hl.brick_nbr)) != MG_OK) return fail(st);
    if ((st = upload(*H, &D.brick_roots, hl.brick_roots)) != MG_OK) return fail(st);
    if ((st = upload(*H, &D.brick_rank, hl.brick_rank)) != MG_OK) return fail(st);
    if ((st = upload(*H, &D.vflags, hl.vflags)) != MG_OK) return fail(st);
    if ((st = upload(*H, &D.cflags, hl.cflags)) != MG_OK) return fail(st);
    if (l > 0 && hl.n_hanging > 0) {  // levels without hanging vertices need no interpolation tables
      if ((st = upload(*H, &D.hang_idx, hl.hang_idx)) != MG_OK) return fail(st);
      if ((st = upload(*H, &D.hang_w, hl.hang_w)) != MG_OK) return fail(st);
    }
    const size_t ns = static_cast<size_t>(hl.n_slots);
    D.n_dofs = hl.n_dofs;
    D.d = LevelDesc{d, l, hl.n, hl.B, hl.S, hl.nb_axis, hl.n_bricks, hl.n_slots, hl.h,
                    D.brick_nbr, D.brick_roots, D.brick_rank, D.vflags};
    if ((st = dalloc(*H, &D.eps, ns)) != MG_OK) return fail(st);
    if ((st = dalloc(*H, &D.r, ns)) != MG_OK) return fail(st);
    if ((st = dalloc(*H, &D.t, ns)) != MG_OK) return fail(st);
    if (o.cycle != MG_CYCLE_V) {
      if ((st = dalloc(*H, &D.ad, ns)) != MG_OK) return fail(st);
      if ((st = dalloc(*H, &D.ar, ns)) != MG_OK) return fail(st);
      if (o.cycle == MG_CYCLE_BPX && l < H->L && (st = dalloc(*H, &D.ai, ns)) != MG_OK) return fail(st);
      if (l < H->L) {  // injection map: the level-(l+1) slot at position 3x
        const HostLevel& hf = g->levels[l + 1];
        std::vector<int32_t> child(hl.n_slots, -1);
        int x[3];
        for (int64_t q = 0; q < hl.n_slots; ++q) {
          hl.coords_of(q, x);
          if (x[0] < 0) continue;
          for (int i = 0; i < d; ++i) x[i] *= 3;
          child[q] = static_cast<int32_t>(hf.slot_of(x));
        }
        if ((st = upload(*H, &D.child, child)) != MG_OK) return fail(st);
      }
    }
    if (o.tensor_coefficients && l == H->L) {  // per-axis deviations of a diagonal-tensor coefficient
      if ((st = dalloc(*H, &D.aniso, ns * d)) != MG_OK) return fail(st);
      if (H->mixed && (st = dalloc(*H, &D.aniso32, ns * d)) != MG_OK) return fail(st);
    }
    if ((st = dalloc(*H, &D.partial, static_cast<size_t>(hl.n_bricks) * hl.B)) != MG_OK) return fail(st);
    if (!H->mixed && (st = dalloc(*H, &D.dinv, ns)) != MG_OK) return fail(st);
    if (!H->mixed && o.ff_sweeps && l == H->L) {  // float-float finest sweeps: split coefficients
      if ((st = dalloc(*H, &D.eps_pair, ns)) != MG_OK) return fail(st);
      if ((st = dalloc(*H, &D.dinv_pair, ns)) != MG_OK) return fail(st);
    }
    if ((st = dalloc(*H, &D.counter, 1)) != MG_OK) return fail(st);
    if (l < H->L) {
      if ((st = dalloc(*H, &D.u, ns)) != MG_OK) return fail(st);
      if ((st = dalloc(*H, &D.b, ns)) != MG_OK) return fail(st);
    }
    if (l < H->top) {
      if (H->galerkin && (st = dalloc(*H, &D.ahat, ns * n3)) != MG_OK) return fail(st);
      if (H->boxmg && (st = dalloc(*H, &D.phat, ns * n5)) != MG_OK) return fail(st);
    }
    if (H->mixed) {
      if ((st = dalloc(*H, &D.eps32, ns)) != MG_OK) return fail(st);
      if ((st = dalloc(*H, &D.u32, ns)) != MG_OK) return fail(st);
      if ((st = dalloc(*H, &D.b32, ns)) != MG_OK) return fail(st);
      if ((st = dalloc(*H, &D.r32, ns)) != MG_OK) return fail(st);
      if ((st = dalloc(*H, &D.t32, ns)) != MG_OK) return fail(st);
      if (l < H->top && H->fmt == 4) {  // bpa streams at their worst case (8 bytes per entry)
        if (H->galerkin) {
          if ((st = dalloc(*H, &D.abpa_rec, ns)) != MG_OK) return fail(st);
          if ((st = dalloc(*H, &D.abpa, ns * n3 * 8)) != MG_OK) return fail(st);
        }
        if (H->boxmg) {
          if ((st = dalloc(*H, &D.pbpa_rec, ns)) != MG_OK) return fail(st);
          if ((st = dalloc(*H, &D.pbpa, ns * n5 * 8)) != MG_OK) return fail(st);
        }
      } else if (l < H->top) {
        if (H->galerkin) {
          // code planes followed by the low-half planes of promoted vertices
          if ((st = dalloc(*H, &D.a16, 2 * ns * n3)) != MG_OK) return fail(st);
          if ((st = dalloc(*H, &D.ascale, ns)) != MG_OK) return fail(st);
        }
        if (H->boxmg) {
          if ((st = dalloc(*H, &D.p16, ns * n5)) != MG_OK) return fail(st);
          if ((st = dalloc(*H, &D.pscale, ns)) != MG_OK) return fail(st);
        }
      }
    }
  }
  if (H->adaptive) {  // injection map of the composite solve and the FP32 composite vectors
    const HostLevel& ht = g->levels[H->top];
    const HostLevel& hf = g->levels[H->L];
    std::vector<int32_t> child(ht.n_slots, -1);
    int x[3];
    for (int64_t s = 0; s < ht.n_slots; ++s) {
      ht.coords_of(s, x);
      if (x[0] < 0) continue;
      for (int i = 0; i < d; ++i) x[i] *= 3;
      child[s] = static_cast<int32_t>(hf.slot_of(x));
    }
    if ((st = upload(*H, &H->child_top, child)) != MG_OK) return fail(st);
    int64_t unref = 0;
    std::vector<int32_t> ref, dofL, hangL;
    for (int64_t s = 0; s < ht.n_slots; ++s) {
      const uint8_t f = ht.vflags[s];
      if (!(f & MG_V_EXISTS) || (f & (MG_V_BOUNDARY | MG_V_HANGING))) continue;
      if (f & MG_V_REFINED)
        ref.push_back(static_cast<int32_t>(s));
      else
        ++unref;
    }
    for (int64_t s = 0; s < hf.n_slots; ++s) {
      const uint8_t f = hf.vflags[s];
      if (!(f & MG_V_EXISTS) || (f & MG_V_BOUNDARY)) continue;
      ((f & MG_V_HANGING) ? hangL : dofL).push_back(static_cast<int32_t>(s));
    }
    H->n_comp_dofs = hf.n_dofs + unref;
    H->n_ref_top = static_cast<int64_t>(ref.size());
    H->n_dof_L = static_cast<int64_t>(dofL.size());
    H->n_hang_L = static_cast<int64_t>(hangL.size());
    if (!ref.empty() && (st = upload(*H, &H->ref_top, ref)) != MG_OK) return fail(st);
    if (!dofL.empty() && (st = upload(*H, &H->dof_L, dofL)) != MG_OK) return fail(st);
    if (!hangL.empty() && (st = upload(*H, &H->hang_L, hangL)) != MG_OK) return fail(st);
    if (H->mixed) {
      if ((st = dalloc(*H, &H->c32, static_cast<size_t>(ht.n_slots))) != MG_OK) return fail(st);
      if ((st = dalloc(*H, &H->cb32, static_cast<size_t>(ht.n_slots))) != MG_OK) return fail(st);
    }
  }
  // coarsest dense system; with the dynamic coarsest level, the slot lists of every level
  // that may become the coarsest one (up to kMaxDynCoarse unknowns) and a matrix buffer
  // for the largest of them, so that mg_setup and mg_solve allocate nothing
  H->c_user = H->c_setup = H->c;
  H->c_max = H->c;
  if (o.dynamic_coarsest)
    while (H->c_max + 1 < H->L && g->levels[H->c_max + 1].n_dofs <= kMaxDynCoarse) ++H->c_max;
  H->cs_lv.assign(H->L + 1, nullptr);
  H->cm_lv.assign(H->L + 1, nullptr);
  H->nc_lv.assign(H->L + 1, 0);
  int nc_big = 0;
  for (int l = H->c; l <= H->c_max; ++l) {
    const HostLevel& hc = g->levels[l];
    std::vector<int32_t> slots, map(hc.n_slots, -1);
    for (int64_t s = 0; s < hc.n_slots; ++s) {
      const uint8_t f = hc.vflags[s];
      if ((f & MG_V_EXISTS) && !(f & (MG_V_BOUNDARY | MG_V_HANGING))) {
        map[s] = static_cast<int32_t>(slots.size());
        slots.push_back(static_cast<int32_t>(s));
      }
    }
    const int n = static_cast<int>(slots.size());
    if (n == 0 || n > 4096) {
      set_error("mg_hier_create: coarsest level has " + std::to_string(n) + " DoFs (need 1..4096)");
      return fail(MG_ERR_INVALID_ARG);
    }
    if ((st = upload(*H, &H->cs_lv[l], slots)) != MG_OK) return fail(st);
    if ((st = upload(*H, &H->cm_lv[l], map)) != MG_OK) return fail(st);
    H->nc_lv[l] = n;
    nc_big = std::max(nc_big, n);
  }
  H->n_c = H->nc_lv[H->c];
  H->c_slots = H->cs_lv[H->c];
  H->c_map = H->cm_lv[H->c];
  if ((st = dalloc(*H, &H->c_mat, static_cast<size_t>(nc_big) * nc_big)) != MG_OK) return fail(st);
  if (o.dynamic_coarsest && (st = dalloc(*H, &H->d_audit, H->L + 1)) != MG_OK) return fail(st);
  if ((st = dalloc(*H, &H->d_status, 1)) != MG_OK) return fail(st);
  if (H->fmt == 4 && (st = dalloc(*H, &H->bpa_used, 2 * (H->L + 1))) != MG_OK) return fail(st);
  if ((st = dalloc(*H, &H->d_scal, 16)) != MG_OK) return fail(st);
  if ((st = dalloc(*H, &H->d_hist, kHistCap)) != MG_OK) return fail(st);
  if ((st = dalloc(*H, &H->d_pint, 4)) != MG_OK) return fail(st);
  if ((st = dalloc(*H, &H->d_pdbl, 4)) != MG_OK) return fail(st);
  {
    unsigned char* ps = nullptr;
    if ((st = dalloc(*H, &ps, std::max(sizeof(PSolve<double>), sizeof(PSolve<float>)))) != MG_OK) return fail(st);
    H->d_psolve = ps;
  }
  H->h_pin = static_cast<double*>(pinned_slot());
  if (!H->h_pin) {
    set_error("mg_hier_create: pinned host memory unavailable");
    return fail(MG_ERR_OOM);
  }
  // the buffers were allocated, zeroed and filled in order on H->own: complete that
  // before any other stream uses them
  if (cudaStreamSynchronize(H->own) != cudaSuccess) {
    set_error(std::string("mg_hier_create: ") + cudaGetErrorString(cudaGetLastError()));
    return fail(MG_ERR_CUDA);
  }
  *out = H;
  return MG_OK;
}

// options and grid checks of mg_hier_create, then create() with the hierarchy's own
// stream at the given priority (the server gives small requests the highest)
mg_status hier_create(const Grid* g, const mg_options& o, int priority, Hier** out, bool blocking) {
  *out = nullptr;
  if (o.coarsest_level < 1 || o.coarsest_level >= g->L || o.nu1 < 0 || o.nu2 < 0 || !(o.omega > 0.0) ||
      o.transfer < 0 || o.transfer > 1 || o.coarse < 0 || o.coarse > 1 || o.precision < 0 || o.precision > 3 || o.smoother < 0 || o.smoother > 1 ||
      (o.smoother == MG_SMOOTH_BLOCK && (o.gs_sweeps < 1 || o.gs_sweeps > 64)) || o.cycle < 0 || o.cycle > 2 ||
      (o.cycle != MG_CYCLE_V && (o.precision != MG_PREC_FP64 || o.smoother != MG_SMOOTH_JACOBI)) ||
      o.dynamic_coarsest < 0 || o.dynamic_coarsest > 1 || (o.dynamic_coarsest && o.cycle != MG_CYCLE_V) ||
      o.tensor_coefficients < 0 || o.tensor_coefficients > 1 ||
      (o.tensor_coefficients && (o.coarse != MG_COARSE_GALERKIN || o.smoother != MG_SMOOTH_JACOBI || o.persistent ||
                                 o.precision == MG_PREC_MIXED_BPA)) ||
      o.ff_sweeps < 0 || o.ff_sweeps > 1 || (o.ff_sweeps && (o.precision != MG_PREC_FP64 || o.cycle != MG_CYCLE_V)) ||
      (o.precision == MG_PREC_MIXED_BPA && !(o.eps_mf >= 0.0 && o.eps_mf < 1e300))) {
    set_error("mg_hier_create: invalid options");
    return MG_ERR_INVALID_ARG;
  }
  if (!g->uniform) {
    // composite solve: levels 0 .. L - 2 present and refined everywhere, so level
    // L - 1 is complete and only its refinement towards level L is partial
    for (int l = 0; l + 1 < g->L; ++l)
      for (size_t c = 0; c < g->cells[l].size(); ++c)
        if (!g->cells[l][c] || !g->refined[l][c]) {
          set_error("mg_hier_create: adaptive grids must be complete up to level max_level - 1");
          return MG_ERR_UNSUPPORTED;
        }
    if (o.coarsest_level >= g->L - 1) {
      set_error("mg_hier_create: the coarsest level must lie below the finest complete level");
      return MG_ERR_INVALID_ARG;
    }
    if (o.cycle != MG_CYCLE_V || o.dynamic_coarsest || o.tensor_coefficients) {
      set_error("mg_hier_create: adaptive grids run the composite V-cycle with a fixed coarsest level and "
                "scalar coefficients");
      return MG_ERR_UNSUPPORTED;
    }
  }
  try {
    return create(g, o, out, priority, blocking);
  } catch (const std::bad_alloc&) {
    set_error("mg_hier_create: out of host memory");
    return MG_ERR_OOM;
  }
}

// device bytes mg_hier_create allocates for a grid and options (admission by HBM footprint)
size_t hier_footprint(const Grid& g, const mg_options& o) {
  const int d = g.dim;
  const size_t n3 = ipow(3, d), n5 = ipow(5, d), full = 1u << d;
  const bool galerkin = o.coarse == MG_COARSE_GALERKIN, boxmg = o.transfer == MG_TRANSFER_BOXMG;
  const bool mixed = o.precision != MG_PREC_FP64;
  const int top = g.uniform ? g.L : g.L - 1;
  size_t bytes = 64 * 1024;  // small fixed buffers (status, scalars, history, parameter block)
  for (int l = o.coarsest_level; l <= g.L; ++l) {
    const HostLevel& hl = g.levels[l];
    const size_t ns = static_cast<size_t>(hl.n_slots), nb = static_cast<size_t>(hl.n_bricks);
    bytes += nb * n3 * 4 + nb * d * 4 + hl.brick_rank.size() * 4 + 2 * ns + (hl.n_hanging > 0 ? ns * full * 12 : 0);
    bytes += 3 * ns * 8 + nb * hl.B * 8 + 4 + (mixed ? 0 : ns * 8);
    if (l < g.L) bytes += 2 * ns * 8;
    if (o.cycle != MG_CYCLE_V) bytes += 2 * ns * 8 + (l < g.L ? ns * 4 : 0);
    if (o.cycle == MG_CYCLE_BPX && l < g.L) bytes += ns * 8;
    if (o.tensor_coefficients && l == g.L) bytes += ns * d * (mixed ? 12 : 8);
    if (!mixed && o.ff_sweeps && l == g.L) bytes += 2 * ns * 8;  // split coefficients and omega / D
    if (l < top) bytes += (galerkin ? ns * n3 * 8 : 0) + (boxmg ? ns * n5 * 8 : 0);
    if (d == 3 && galerkin && l == top && top > o.coarsest_level && hl.B == 9) bytes += nb * kApPerBrick * 8;
    if (mixed) {
      bytes += 5 * ns * 4;
      const size_t per = o.precision == MG_PREC_MIXED_BPA ? 8 : 2, sc = o.precision == MG_PREC_MIXED_BPA ? 8 : 4;
      const size_t per_a = o.precision == MG_PREC_MIXED_BPA ? 8 : 4;  // 16-bit codes + low halves
      if (l < top) bytes += (galerkin ? ns * n3 * per_a + ns * sc : 0) + (boxmg ? ns * n5 * per + ns * sc : 0);
    }
    if (l == top && top < g.L) bytes += ns * 4 + (mixed ? 2 * ns * 4 : 0);  // injection map, FP32 composite vectors
  }
  const size_t nc = static_cast<size_t>(g.levels[o.coarsest_level].n_dofs);
  return bytes + nc * nc * 8 + g.levels[o.coarsest_level].n_slots * 4 + nc * 4;
}

// ----------------------------------------------------------------------------- kernel dispatch

constexpr int64_t kSweepTargetCtas = 4 * 152;  // spread small levels over the SMs

template <typename T>
static SweepArgs<T> sweep_args(const Hier& H, int l, const T* u, const T* b, T* out, int* amode) {
  const DevLevel& D = H.lv[l];
  const bool coarse = l < H.top && H.galerkin;
  SweepArgs<T> a{};
  a.L = D.d;
  a.u = u;
  a.b = b;
  a.out = out;
  a.omega = static_cast<T>(H.opt.omega);
  const int tuned = std::is_same<T, double>::value ? D.R64 : D.R32;
  a.R = tuned > 0 ? tuned : sweep_slab<T>(H.dim, D.d.B, D.d.n_bricks);
  *amode = 0;
  if constexpr (std::is_same<T, double>::value) {
    a.eps = D.eps;
    a.dinv = D.dinv;
    if (H.ff_active) {
      a.eps_pair = D.eps_pair;
      a.dinv_pair = D.dinv_pair;
    }
    if (coarse) {
      *amode = 1;
      a.ahat = D.ahat;
    }
  } else {
    a.eps = D.eps32;
    if (coarse && H.fmt == 4) {
      *amode = 4;
      a.ahat = D.abpa;
      a.ascale = D.abpa_rec;
    } else if (coarse) {
      *amode = H.fmt == 1 ? 2 : 3;
      a.ahat = D.a16;
      a.ascale = D.ascale;
    }
  }
  return a;
}

template <typename T>
static void launch(const Hier& H, SweepArgs<T> a, int op, int amode, cudaStream_t s) {
  if (H.dim == 2)
    launch_sweep<2, T>(a, op, amode, s);
  else
    launch_sweep<3, T>(a, op, amode, s);
}

template <typename T>
static void sweep(const Hier& H, int l, int op, const T* u, const T* b, T* out, double* norm2, cudaStream_t s) {
  int amode = 0;
  SweepArgs<T> a = sweep_args<T>(H, l, u, b, out, &amode);
  const DevLevel& D = H.lv[l];
  const bool tensor = H.tensor && l == H.L;
  if (norm2 && !tensor) {
    a.partial = D.partial;
    a.counter = D.counter;
    a.norm2 = norm2;
  }
  launch<T>(H, a, op, amode, s);
  if (tensor) {  // the anisotropic part of a diagonal-tensor coefficient (finest level)
    const T* an;
    const T* ep;
    if constexpr (std::is_same<T, double>::value) {
      an = D.aniso;
      ep = D.eps;
    } else {
      an = D.aniso32;
      ep = D.eps32;
    }
    const double* dinv = std::is_same<T, double>::value ? D.dinv : nullptr;
    const unsigned g = static_cast<unsigned>((D.d.n_slots + kBlock - 1) / kBlock);
    const T om = static_cast<T>(H.opt.omega);
    if (op == kJacobi) {
      if (H.dim == 2) k_aniso_fix<2, T, kJacobi><<<g, kBlock, 0, s>>>(D.d, u, out, an, ep, dinv, om, nullptr, nullptr, nullptr);
      else k_aniso_fix<3, T, kJacobi><<<g, kBlock, 0, s>>>(D.d, u, out, an, ep, dinv, om, nullptr, nullptr, nullptr);
    } else {
      double* pa = norm2 ? D.partial : nullptr;
      unsigned* ct = norm2 ? D.counter : nullptr;
      if (H.dim == 2) k_aniso_fix<2, T, kResidual><<<g, kBlock, 0, s>>>(D.d, u, out, an, ep, dinv, om, pa, ct, norm2);
      else k_aniso_fix<3, T, kResidual><<<g, kBlock, 0, s>>>(D.d, u, out, an, ep, dinv, om, pa, ct, norm2);
    }
  }
}

template <typename T>
static void transfer(const Hier& H, int fine, bool restrict_op, const T* in, T* out, cudaStream_t s,
                     const int32_t* list = nullptr, int64_t n_list = 0, T* zero_c = nullptr) {
  const DevLevel& F = H.lv[fine];
  const DevLevel& C = H.lv[fine - 1];
  int pmode = 0;
  const void* ph = nullptr;
  const void* ps = nullptr;
  if (H.boxmg && fine <= H.top) {
    if constexpr (std::is_same<T, double>::value) {
      pmode = 1;
      ph = C.phat;
    } else if (H.fmt == 4) {
      pmode = 4;
      ph = C.pbpa;
      ps = C.pbpa_rec;
    } else {
      pmode = H.fmt == 1 ? 2 : 3;
      ph = C.p16;
      ps = C.pscale;
    }
  }
  if (H.dim == 2)
    launch_transfer<2, T>(C.d, F.d, restrict_op, pmode, in, out, ph, ps, s, list, n_list, zero_c);
  else
    launch_transfer<3, T>(C.d, F.d, restrict_op, pmode, in, out, ph, ps, s, list, n_list, zero_c);
}

template <typename T>
static void coarse_solve(const Hier& H, const T* b, T* u, cudaStream_t s) {
  if (H.n_c <= 32)
    launch_pdl(k_coarse_solve_small<T>, 1, 32, 0, s, static_cast<const double*>(H.c_mat), H.n_c,
               static_cast<const int32_t*>(H.c_slots), b, u);
  else
    launch_pdl(k_coarse_solve<T>, 1, kBlock, H.n_c * sizeof(double), s, static_cast<const double*>(H.c_mat),
               H.n_c, static_cast<const int32_t*>(H.c_slots), b, u);
}

// nu smoothing steps, ping-pong through tmp, result in u: damped Jacobi sweeps, or block
// Jacobi steps (Sect. 4.2: Gauss-Seidel on the patches' iota vertices in place, then the
// Jacobi sweep with the iota values kept) on the uniform levels of a block hierarchy
// first_done: the first sweep (u -> tmp) has already run (the fused FP64 solve runs it
// with the previous cycle, beside its convergence norm)
template <typename T>
static void smooth(const Hier& H, int l, T* u, const T* b, T* tmp, int nu, cudaStream_t s, bool first_done = false) {
  T* src = first_done ? tmp : u;
  T* dst = first_done ? u : tmp;
  const bool block = H.opt.smoother == MG_SMOOTH_BLOCK && l <= H.top;
  for (int k = first_done ? 1 : 0; k < nu; ++k) {
    if (block) {
      int amode = 0;
      SweepArgs<T> g = sweep_args<T>(H, l, src, b, src, &amode);
      const int gs = H.opt.gs_sweeps;
      if (H.dim == 2) launch_patch_gs<2, T>(g, amode, gs, s); else launch_patch_gs<3, T>(g, amode, gs, s);
      SweepArgs<T> a = sweep_args<T>(H, l, src, b, dst, &amode);
      a.block = 1;
      launch<T>(H, a, kJacobi, amode, s);
    } else {
      sweep<T>(H, l, kJacobi, src, b, dst, nullptr, s);
    }
    T* t = src;
    src = dst;
    dst = t;
  }
  if (src != u) cudaMemcpyAsync(u, src, H.lv[l].d.n_slots * sizeof(T), cudaMemcpyDeviceToDevice, s);
}

template <typename T>
static T* lvec(Hier& H, int l, int which) {  // 0 u, 1 b, 2 r, 3 t
  DevLevel& D = H.lv[l];
  if constexpr (std::is_same<T, double>::value) {
    return which == 0 ? D.u : which == 1 ? D.b : which == 2 ? D.r : D.t;
  } else {
    return which == 0 ? D.u32 : which == 1 ? D.b32 : which == 2 ? D.r32 : D.t32;
  }
}

// V-cycle smoothing of a 2D level of brick edge 27 or 9 (damped Jacobi, no anisotropy pass): nu
// sweeps from the iterate in cur, two per launch where nu allows (launch_sweep_pair_2d_*,
// bit for bit two sweeps); returns the buffer holding the result
static bool pair_smoothing(const Hier& H, int l) {
  return H.dim == 2 && (H.lv[l].d.B == 27 || H.lv[l].d.B == 9) && H.opt.smoother == MG_SMOOTH_JACOBI &&
         !(H.tensor && l == H.L) && !(H.fmt == 4 && l < H.top);
}

template <typename T>
static T* smooth_pairs(const Hier& H, int l, T* cur, T* oth, const T* b, int nu, cudaStream_t s) {
  for (int k = 0; k < nu;) {
    int amode = 0;
    SweepArgs<T> a = sweep_args<T>(H, l, cur, b, oth, &amode);
    if (nu - k >= 2) {
      if constexpr (std::is_same<T, float>::value) launch_sweep_pair_2d_f32(a, amode, s);
      else launch_sweep_pair_2d_f64(a, amode, s);
      k += 2;
    } else {
      launch<T>(H, a, kJacobi, amode, s);
      k += 1;
    }
    T* t = cur;
    cur = oth;
    oth = t;
  }
  return cur;
}

// V(nu1, nu2) cycle on level l (correction scheme; Alg. 1 semantics, Sect. 3 FAS reduced)
template <typename T>
static void vcycle(Hier& H, int l, T* u, const T* b, cudaStream_t s, bool first_done = false) {
  if (l == H.c) {
    coarse_solve<T>(H, b, u, s);
    return;
  }
  T* tmp = lvec<T>(H, l, 3);
  T* r = lvec<T>(H, l, 2);
  T* uc = lvec<T>(H, l - 1, 0);
  T* bc = lvec<T>(H, l - 1, 1);
  // FP32 levels, and the coarse levels of FP64 cycles of FP64 hierarchies (their sweeps
  // take omega / diag(A) from the setup, which mixed hierarchies do not store; the finest
  // FP64 level is bound by the FP64 units: a pair's ring would cost more than the launch
  // it saves)
  if (pair_smoothing(H, l) && (std::is_same<T, float>::value || (l < H.L && H.lv[l].dinv != nullptr))) {
    {  // the iterate moves between u and tmp; it ends in u
      T* cur = smooth_pairs<T>(H, l, u, tmp, b, H.opt.nu1, s);
      sweep<T>(H, l, kResidual, cur, b, r, nullptr, s);
      transfer<T>(H, l, true, r, bc, s, nullptr, 0, uc);
      vcycle<T>(H, l - 1, uc, bc, s);
      transfer<T>(H, l, false, uc, cur, s);
      T* fin = smooth_pairs<T>(H, l, cur, cur == u ? tmp : u, b, H.opt.nu2, s);
      if (fin != u) cudaMemcpyAsync(u, fin, H.lv[l].d.n_slots * sizeof(T), cudaMemcpyDeviceToDevice, s);
      return;
    }
  }
  smooth<T>(H, l, u, b, tmp, H.opt.nu1, s, first_done);
  sweep<T>(H, l, kResidual, u, b, r, nullptr, s);
  transfer<T>(H, l, true, r, bc, s, nullptr, 0, uc);  // also zeroes the coarse correction uc
  vcycle<T>(H, l - 1, uc, bc, s);
  transfer<T>(H, l, false, uc, u, s);
  smooth<T>(H, l, u, b, tmp, H.opt.nu2, s);
}

// finest residual r = b - A u with its squared norm into d_scal[slot]
template <typename T>
static void residual_norm(Hier& H, const T* u, const T* b, T* r, int slot, cudaStream_t s) {
  sweep<T>(H, H.L, kResidual, u, b, r, H.d_scal + slot, s);
}

static mg_status additive_reset(Hier& H, double* u, cudaStream_t s);

// make level c the directly solved one (its slot lists were prepared at creation);
// captured cycles of another coarsest level are dropped
static void set_coarsest(Hier& H, int c) {
  if (c == H.c && H.c_slots == H.cs_lv[c]) return;
  H.c = c;
  H.n_c = H.nc_lv[c];
  H.c_slots = H.cs_lv[c];
  H.c_map = H.cm_lv[c];
  for (Graph* gr : {&H.g_cycle64, &H.g_cycle_ff, &H.g_comp_ff, &H.g_outer, &H.g_inner, &H.g_comp64, &H.g_comp_outer, &H.g_comp_inner, &H.g_add,
                    &H.g_fused[0][0], &H.g_fused[0][1], &H.g_fused[1][0], &H.g_fused[1][1]})
    gr->reset();
}

// dense FP64 operator of the coarsest level and its Cholesky factor (status 3 if the
// operator is not positive definite)
static void coarse_factor(Hier& H, cudaStream_t s) {
  DevLevel& C = H.lv[H.c];
  const double* ah = (H.c < H.top && H.galerkin) ? C.ahat : nullptr;
  if (H.dim == 2)
    k_coarse_assemble<2><<<nblk(H.n_c), kBlock, 0, s>>>(C.d, C.eps, ah, H.c_slots, H.c_map, H.n_c, H.c_mat);
  else
    k_coarse_assemble<3><<<nblk(H.n_c), kBlock, 0, s>>>(C.d, C.eps, ah, H.c_slots, H.c_map, H.n_c, H.c_mat);
  k_cholesky<<<1, kBlock, 0, s>>>(H.c_mat, H.n_c, H.d_status);
}

// Sect. 4.3, dynamic coarsest level, rule (a): audit the coarse levels and make the level
// above the finest failing one the coarsest
static mg_status dynamic_coarsest_setup(Hier& H, cudaStream_t s) {
  MG_TRY_CUDA(cudaMemsetAsync(H.d_audit, 0, static_cast<size_t>(H.L + 1) * sizeof(int), s));
  for (int l = H.c_user; l < H.top; ++l) {
    DevLevel& D = H.lv[l];
    const double* ah = H.galerkin ? D.ahat : nullptr;
    if (H.dim == 2)
      k_audit<2><<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, D.eps, ah, H.d_audit + l);
    else
      k_audit<3><<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, D.eps, ah, H.d_audit + l);
  }
  MG_CHECK(last_launch("setup: coarse-level audit"));
  std::vector<int> fail(H.L + 1, 0);
  MG_TRY_CUDA(cudaMemcpyAsync(fail.data(), H.d_audit, fail.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
  MG_TRY_CUDA(cudaStreamSynchronize(s));
  int cn = H.c_user;
  for (int l = H.c_user; l < H.top; ++l)
    if (fail[l]) cn = std::max(cn, l + 1);
  if (cn > H.c_max) {
    set_error("mg_setup: the dynamic coarsest level (Sect. 4.3) would be level " + std::to_string(cn) +
              ": beyond the finest level or the " + std::to_string(kMaxDynCoarse) +
              " unknowns of the direct coarse solve");
    return MG_ERR_INDEFINITE_COARSE;
  }
  set_coarsest(H, cn);
  H.c_setup = cn;
  return MG_OK;
}

// eps_in: level-concatenated leaf coefficients; tensor_axes (instead, tensor hierarchies):
// d such arrays, one per axis, of a diagonal-tensor coefficient on the finest level
static mg_status run_setup(Hier& H, const double* eps_in, cudaStream_t s, bool check_now = true,
                           const double* tensor_axes = nullptr) {
  const Grid& g = *H.g;
  const int d = H.dim;
  if (H.opt.dynamic_coarsest) {
    if (!check_now) {
      set_error("mg_setup: the dynamic coarsest level needs a synchronous setup (single hierarchies)");
      return MG_ERR_UNSUPPORTED;
    }
    set_coarsest(H, H.c_user);  // every setup starts again from the requested level
  }
  if (tensor_axes) {  // uniform grid: the leaves are the finest level's cells
    DevLevel& D = H.lv[H.L];
    const int64_t nt = g.levels[H.L].slot_offset + g.levels[H.L].n_slots;
    const double* ax = tensor_axes + g.levels[H.L].slot_offset;
    if (d == 2)
      k_tensor_split<2><<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, ax, nt, D.eps, D.aniso);
    else
      k_tensor_split<3><<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, ax, nt, D.eps, D.aniso);
  } else {
    for (int l = H.c; l <= H.L; ++l) {
      DevLevel& D = H.lv[l];
      k_leaf_eps<<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, D.cflags, eps_in + g.levels[l].slot_offset, D.eps);
    }
    if (H.tensor)  // a scalar coefficient on a tensor hierarchy: no anisotropy
      MG_TRY_CUDA(cudaMemsetAsync(H.lv[H.L].aniso, 0, sizeof(double) * d * H.lv[H.L].d.n_slots, s));
  }
  for (int l = H.L - 1; l >= H.c; --l) {
    DevLevel& C = H.lv[l];
    DevLevel& F = H.lv[l + 1];
    if (d == 2)
      k_mean_eps<2><<<nblk(C.d.n_slots), kBlock, 0, s>>>(C.d, F.d, C.cflags, F.eps, C.eps);
    else
      k_mean_eps<3><<<nblk(C.d.n_slots), kBlock, 0, s>>>(C.d, F.d, C.cflags, F.eps, C.eps);
  }
  MG_CHECK(last_launch("setup: coefficients"));
  MG_TRY_CUDA(cudaMemsetAsync(H.d_status, 0, sizeof(int), s));
  for (int l = H.top; l > H.c; --l) {  // BoxMG / Galerkin on the complete levels
    DevLevel& F = H.lv[l];
    DevLevel& C = H.lv[l - 1];
    const double* ahat_f = (l < H.top && H.galerkin) ? F.ahat : nullptr;
    if (H.boxmg) {
      const unsigned gp = static_cast<unsigned>(((C.d.n_slots << d) + 63) / 64);
      if (d == 2)
        k_boxmg<2><<<gp, 64, 0, s>>>(C.d, F.d, F.eps, ahat_f, C.phat, H.d_status, F.aniso);
      else
        k_boxmg3c<<<static_cast<unsigned>((C.d.n_slots + kBoxCells - 1) / kBoxCells), 8 * kBoxCells, 0, s>>>(
            C.d, F.d, F.eps, ahat_f, C.phat, H.d_status, F.aniso);
    }
    if (H.galerkin) {
      // 128-thread CTAs: 4 coarse vertices (2D) or 1 (3D) per CTA
      const unsigned gr = static_cast<unsigned>((C.d.n_slots + (128 / rap_tpv<2>()) - 1) / (128 / rap_tpv<2>()));
      static const bool smem_opt_in = [] {  // the 3D kernel stages 27 KB of P
        return cudaFuncSetAttribute(k_rap<3, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(rap_dyn_smem<3, 1>())) == cudaSuccess &&
               cudaFuncSetAttribute(k_rap<3, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(rap_dyn_smem<3, 0>())) == cudaSuccess;
      }();
      (void)smem_opt_in;
      if (d == 2) {
        if (H.boxmg)
          k_rap<2, 1><<<gr, 128, rap_dyn_smem<2, 1>(), s>>>(C.d, F.d, F.eps, ahat_f, C.eps, C.phat, C.ahat, F.aniso);
        else
          k_rap<2, 0><<<gr, 128, rap_dyn_smem<2, 0>(), s>>>(C.d, F.d, F.eps, ahat_f, C.eps, C.phat, C.ahat, F.aniso);
      } else if (H.ap3 && F.d.B == 9 && F.d.n_bricks * kApPerBrick <= H.ap3_len) {
        // two stages: AP = A_f P per fine vertex into the scratch, then P^T (AP) per coarse one
        const unsigned g1 = static_cast<unsigned>((ap_threads(F.d.n_bricks) + 127) / 128);
        const unsigned g2 = static_cast<unsigned>((C.d.n_slots + kRapPtSlots - 1) / kRapPtSlots);
        static const bool pt_opt_in = [] {
          return cudaFuncSetAttribute(k_rap3_pt<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(rap3_pt_smem())) == cudaSuccess &&
                 cudaFuncSetAttribute(k_rap3_pt<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(rap3_pt_smem())) == cudaSuccess;
        }();
        (void)pt_opt_in;
        if (H.boxmg) {
          k_rap3_ap<1><<<g1, 128, 0, s>>>(C.d, F.d, F.eps, ahat_f, C.phat, H.ap3, F.aniso);
          k_rap3_pt<1><<<g2, 27 * 32, rap3_pt_smem(), s>>>(C.d, F.d, C.eps, C.phat, H.ap3, C.ahat);
        } else {
          k_rap3_ap<0><<<g1, 128, 0, s>>>(C.d, F.d, F.eps, ahat_f, C.phat, H.ap3, F.aniso);
          k_rap3_pt<0><<<g2, 27 * 32, rap3_pt_smem(), s>>>(C.d, F.d, C.eps, C.phat, H.ap3, C.ahat);
        }
      } else {
        const unsigned g3 = static_cast<unsigned>(C.d.n_slots);
        if (H.boxmg)
          k_rap<3, 1><<<g3, 128, rap_dyn_smem<3, 1>(), s>>>(C.d, F.d, F.eps, ahat_f, C.eps, C.phat, C.ahat, F.aniso);
        else
          k_rap<3, 0><<<g3, 128, rap_dyn_smem<3, 0>(), s>>>(C.d, F.d, F.eps, ahat_f, C.eps, C.phat, C.ahat, F.aniso);
      }
    }
    MG_CHECK(last_launch("setup: BoxMG / Galerkin"));
  }
  if (H.opt.dynamic_coarsest) MG_CHECK(dynamic_coarsest_setup(H, s));
  // diagonal audit of every level (Sect. 4.3 definiteness check), Jacobi factors,
  // coarsest factor
  for (int l = H.c; l <= H.L; ++l) {
    DevLevel& D = H.lv[l];
    const double* ah = (l < H.top && H.galerkin) ? D.ahat : nullptr;
    if (d == 2)
      k_export_stencils<2><<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, D.eps, ah, nullptr, H.d_status, D.aniso);
    else
      k_export_stencils<3><<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, D.eps, ah, nullptr, H.d_status, D.aniso);
    if (D.dinv) {
      if (d == 2)
        k_jacobi_dinv<2><<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, D.eps, ah, H.opt.omega, D.dinv);
      else
        k_jacobi_dinv<3><<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, D.eps, ah, H.opt.omega, D.dinv);
    }
    if (D.eps_pair) {
      k_split_pairs<<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d.n_slots, D.eps, D.eps_pair);
      k_split_pairs<<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d.n_slots, D.dinv, D.dinv_pair);
    }
  }
  coarse_factor(H, s);
  MG_CHECK(last_launch("setup: coarse factor"));
  if (H.mixed) {
    const int n3 = ipow(3, d), n5 = ipow(5, d);
    if (H.tensor) {
      DevLevel& F = H.lv[H.L];
      k_to_f32<<<nblk(d * F.d.n_slots), kBlock, 0, s>>>(d * F.d.n_slots, F.aniso, F.aniso32);
    }
    for (int l = H.c; l <= H.L; ++l) {
      DevLevel& D = H.lv[l];
      k_to_f32<<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d.n_slots, D.eps, D.eps32);
      if (l < H.top && H.fmt == 4) {
        const int64_t ns = D.d.n_slots;
        if (H.galerkin)
          bpa_encode_enqueue(BpaSrc{D.ahat, n3, true, D.d}, ns, H.opt.eps_mf, D.abpa_rec, D.abpa,
                             H.bpa_used + 2 * l, H.d_status, 4, 5, s);
        if (H.boxmg)
          bpa_encode_enqueue(BpaSrc{D.phat, n5, true, D.d}, ns, H.opt.eps_mf, D.pbpa_rec, D.pbpa,
                             H.bpa_used + 2 * l + 1, H.d_status, 4, 5, s);
      } else if (l < H.top) {
        const unsigned g = nblk(D.d.n_slots);
#define MG_ENC(DIM, FMT)                                                                          \
  do {                                                                                            \
    if (H.galerkin) k_encode_planes<DIM, FMT><<<g, kBlock, 0, s>>>(D.d, n3, D.ahat, D.a16, D.ascale, D.eps, 1); \
    if (H.boxmg) k_encode_planes<DIM, FMT><<<g, kBlock, 0, s>>>(D.d, n5, D.phat, D.p16, D.pscale, D.eps, 0);    \
  } while (0)
        if (d == 2) {
          if (H.fmt == 1) MG_ENC(2, 1); else MG_ENC(2, 2);
        } else {
          if (H.fmt == 1) MG_ENC(3, 1); else MG_ENC(3, 2);
        }
#undef MG_ENC
      }
    }
    MG_CHECK(last_launch("setup: encode"));
  }
  if (H.opt.cycle != MG_CYCLE_V) MG_CHECK(additive_reset(H, nullptr, s));
  if (!check_now) {  // the caller reads d_status after one synchronisation for many hierarchies
    H.ready = true;
    return MG_OK;
  }
  int status = 0;
  MG_TRY_CUDA(cudaMemcpyAsync(&status, H.d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  MG_TRY_CUDA(cudaStreamSynchronize(s));
  return setup_status(H, status);
}

mg_status setup_status(Hier& H, int status) {
  if (status == 1) {
    set_error("mg_setup: a BoxMG patch system is singular");
    return MG_ERR_INDEFINITE_COARSE;
  }
  if (status == 2) {
    set_error("mg_setup: a level operator has a non-positive diagonal (Sect. 4.3 definiteness check)");
    return MG_ERR_INDEFINITE_COARSE;
  }
  if (status == 3) {
    set_error("mg_setup: the coarsest operator is not positive definite");
    return MG_ERR_INDEFINITE_COARSE;
  }
  if (status == 4 || status == 5) {
    set_error(status == 4 ? "mg_setup: a hierarchical delta is not finite"
                          : "mg_setup: a hierarchical delta is beyond the bpa codec's exponent range");
    return MG_ERR_NONFINITE;
  }
  H.ready = true;
  return MG_OK;
}

mg_status setup_enqueue(Hier& H, const double* eps, cudaStream_t s) { return run_setup(H, eps, s, false); }

static cudaStream_t pick(Hier& H, void* stream) {
  return stream ? static_cast<cudaStream_t>(stream) : H.own;
}

// Slab depth per level and sweep type by measurement: every divisor R of the brick edge
// (B, B/3, ..., 1) is timed on the level's own buffers (Jacobi sweeps, CUDA events on
// s) and the fastest kept.  The sweeps compute the same values for every R; only the
// work split over CTAs changes.
template <typename T>
static mg_status tune_level(Hier& H, int l, cudaStream_t s, int* best_out) {
  DevLevel& D = H.lv[l];
  T* u = lvec<T>(H, l, 2);
  T* out = lvec<T>(H, l, 3);
  const T* b = std::is_same<T, double>::value ? reinterpret_cast<const T*>(D.eps) : reinterpret_cast<const T*>(D.eps32);
  cudaEvent_t e0, e1;
  MG_TRY_CUDA(cudaEventCreate(&e0));
  MG_TRY_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 0.0f;
  for (int R = D.d.B; R >= 1; R /= 3) {
    int amode = 0;
    SweepArgs<T> a = sweep_args<T>(H, l, u, b, out, &amode);
    a.R = R;
    for (int k = 0; k < 2; ++k) launch<T>(H, a, kJacobi, amode, s);
    cudaEventRecord(e0, s);
    constexpr int reps = 5;
    for (int k = 0; k < reps; ++k) launch<T>(H, a, kJacobi, amode, s);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best == 0 || ms < best_ms) {
      best = R;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  MG_CHECK(last_launch("mg_autotune"));
  *best_out = best;
  return MG_OK;
}

// capture fn() on stream s into g (re-captured when the key pointers change)
template <typename F>
static mg_status graph_launch(Hier& H, Graph& g, const void* k0, const void* k1, cudaStream_t s, F fn) {
  if (!H.opt.use_graphs) {
    fn(s);
    return last_launch("cycle");
  }
  if (!g.exec || g.key0 != k0 || g.key1 != k1) {
    g.reset();
    cudaGraph_t graph = nullptr;
    MG_TRY_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    fn(s);
    const cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error(std::string("graph capture: ") + cudaGetErrorString(e));
      return MG_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      g.exec = nullptr;
      set_error(std::string("graph instantiate: ") + cudaGetErrorString(ei));
      return MG_ERR_CUDA;
    }
    g.key0 = k0;
    g.key1 = k1;
  }
  MG_TRY_CUDA(cudaGraphLaunch(g.exec, s));
  return MG_OK;
}

// FP64 solves with float-float finest sweeps switch to FP64 sweeps below this multiple of
// the tolerance (their own residual floor is ~1e-10 on the 2D level-6 checkerboard, 1e-9
// on level 7: a 1e-10 solve switches at 1e-7)
constexpr double kFfSwitch = 1e3;

static mg_status solve_fp64(Hier& H, double* u, const double* b, double tol, int max_cycles, mg_solve_stats* st,
                            cudaStream_t s) {
  DevLevel& F = H.lv[H.L];
  // float-float finest sweeps (mg_options.ff_sweeps) carry the cycles while the residual
  // is far above the tolerance; the last cycles run in FP64, whose residual floor lies
  // ~2^6 below theirs (iterative refinement: the final iterate is the FP64 one)
  const bool ff = F.eps_pair != nullptr;
  struct Restore {
    Hier& h;
    ~Restore() { h.ff_active = true; }
  } restore{H};
  H.ff_active = false;  // r0 in FP64
  MG_TRY_CUDA(cudaMemsetAsync(u, 0, F.d.n_slots * sizeof(double), s));
  residual_norm<double>(H, u, b, F.r, 0, s);
  MG_TRY_CUDA(cudaMemcpyAsync(H.h_pin, H.d_scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  MG_TRY_CUDA(cudaStreamSynchronize(s));
  const double r0 = std::sqrt(H.h_pin[0]);
  if (st) {
    st->r0_norm = r0;
    st->history_len = 0;
  }
  if (!std::isfinite(r0)) {
    set_error("mg_solve: non-finite initial residual");
    return MG_ERR_NONFINITE;
  }
  double rel = r0 > 0 ? 1.0 : 0.0;
  int cycles = 0;
  if (H.opt.dynamic_coarsest && H.c != H.c_setup) {
    // rule (b) raised the coarsest level in an earlier solve: every solve starts from
    // the level the setup chose (rule (a))
    set_coarsest(H, H.c_setup);
    coarse_factor(H, s);
  }
  H.ff_active = ff && rel > kFfSwitch * tol;
  // Fused convergence test: the first Jacobi sweep of a cycle forms b - A u at every DoF
  // anyway, so cycle k's graph ends with the first sweep of cycle k + 1 (u_k -> F.t, u_k
  // kept in u) and takes ||b - A u_k|| from it instead of a separate residual sweep; the
  // next graph starts from that sweep.  A solve that stops after cycle k leaves the sweep
  // unused.  The iterates are those of the plain loop.  Needs the finest level's column
  // kernel, damped Jacobi with nu1 >= 1 and no anisotropy correction pass.
  const int Bf = F.d.B;
  const bool fused = H.opt.use_graphs && H.opt.smoother == MG_SMOOTH_JACOBI && H.opt.nu1 >= 1 && !H.tensor &&
                     ((H.dim == 2 && Bf == 27) || (H.dim == 3 && Bf == 9));
  bool pending = false;  // F.t holds the first sweep of the next cycle, formed from u
  while (rel > tol && cycles < max_cycles) {
    if (fused) {
      const bool lead = !pending;
      MG_CHECK(graph_launch(H, H.g_fused[H.ff_active ? 1 : 0][lead ? 1 : 0], u, b, s, [&](cudaStream_t ss) {
        if (lead) sweep<double>(H, H.L, kJacobi, u, b, F.t, nullptr, ss);
        vcycle<double>(H, H.L, u, b, ss, true);
        sweep<double>(H, H.L, kJacobiNorm, u, b, F.t, H.d_scal, ss);
        cudaMemcpyAsync(H.h_pin, H.d_scal, sizeof(double), cudaMemcpyDeviceToHost, ss);
      }));
      pending = true;
    } else {
      MG_CHECK(graph_launch(H, H.ff_active ? H.g_cycle_ff : H.g_cycle64, u, b, s, [&](cudaStream_t ss) {
        vcycle<double>(H, H.L, u, b, ss);
        residual_norm<double>(H, u, b, F.r, 0, ss);
        cudaMemcpyAsync(H.h_pin, H.d_scal, sizeof(double), cudaMemcpyDeviceToHost, ss);
      }));
    }
    MG_TRY_CUDA(cudaStreamSynchronize(s));
    ++cycles;
    const double prev = rel;
    rel = std::sqrt(H.h_pin[0]) / r0;
    // leave float-float near the tolerance, or once its cycles stop contracting (the
    // pending first sweep was a float-float one: the next FP64 cycle forms its own)
    if (H.ff_active && (rel <= kFfSwitch * tol || rel > 0.95 * prev)) {
      H.ff_active = false;
      pending = false;
    }
    if (H.opt.dynamic_coarsest && rel > tol && rel > 0.95 * prev && H.c < H.c_max) {
      // Sect. 4.3, rule (b): the residual stagnated or grew, raise the coarsest level
      set_coarsest(H, H.c + 1);
      MG_TRY_CUDA(cudaMemsetAsync(H.d_status, 0, sizeof(int), s));
      coarse_factor(H, s);
      int status = 0;
      MG_TRY_CUDA(cudaMemcpyAsync(&status, H.d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
      MG_TRY_CUDA(cudaStreamSynchronize(s));
      if (status != 0) {
        set_error("mg_solve: the raised coarsest level is not positive definite");
        return MG_ERR_INDEFINITE_COARSE;
      }
    }
    if (st && st->history && st->history_len < st->history_capacity) st->history[st->history_len++] = rel;
    if (!std::isfinite(rel)) {
      set_error("mg_solve: non-finite residual");
      if (st) st->cycles = cycles;
      return MG_ERR_NONFINITE;
    }
    if (rel > 1e6) {
      set_error("mg_solve: residual grew by more than 1e6 (diverged)");
      if (st) st->cycles = cycles;
      return MG_ERR_DIVERGED;
    }
  }
  if (st) {
    st->cycles = cycles;
    st->outer_steps = cycles;
    st->rel_residual = rel;
  }
  if (rel > tol) {
    set_error("mg_solve: not converged within max_cycles");
    return MG_ERR_NOT_CONVERGED;
  }
  return MG_OK;
}

// One traversal of the additive multigrid of Alg. 2 on level iterates u_l (u, b: the
// finest level's), corrections d_l (D.ad) and surpluses uh_l (D.t).  Descent: d_l +=
// P d_{l-1}, u_l += P d_{l-1}, uh_l = u_l - P u_{l-1}; ascent: r_l = b_l - A_l u_l (D.r),
// rh_l = b_l - A_l uh_l (D.ar), d_l = omega D^-1 r_l, u_l += d_l, u_{l-1} = I u_l,
// b_{l-1} = R rh_l.  The coarse b_l are rebuilt by the restriction every traversal.
//
// BPX (Alg. 3), in the same pass: above the coarsest level the c-points skip their own
// update, which is injected to the coarser level (i_{l-1} = I d_l, D.ai of level l-1)
// and zeroed; the descent applies P d_{l-1} at c-points and P (d_{l-1} - i_{l-1})
// elsewhere (P is the injection at c-points, so P (d - i) + i there); the coarse
// iterates are not overwritten by injection.
static void additive_traversal(Hier& H, double* u, const double* b, cudaStream_t s) {
  auto U = [&](int l) { return l == H.L ? u : H.lv[l].u; };
  auto Bv = [&](int l) { return l == H.L ? b : static_cast<const double*>(H.lv[l].b); };
  const bool bpx = H.opt.cycle == MG_CYCLE_BPX;
  for (int l = H.c; l <= H.L; ++l) {
    DevLevel& D = H.lv[l];
    const size_t bytes = static_cast<size_t>(D.d.n_slots) * sizeof(double);
    if (l > H.c) {
      DevLevel& C = H.lv[l - 1];
      if (bpx) {
        k_sub<<<nblk(C.d.n_slots), kBlock, 0, s>>>(C.d.n_slots, C.ad, C.ai, C.ar);  // x = d - i
        transfer<double>(H, l, false, C.ar, D.ad, s);
        transfer<double>(H, l, false, C.ar, U(l), s);
        k_bpx_cpoints<<<nblk(C.d.n_slots), kBlock, 0, s>>>(C.d, C.child, C.ai, D.ad, U(l));
      } else {
        transfer<double>(H, l, false, C.ad, D.ad, s);
        transfer<double>(H, l, false, C.ad, U(l), s);
      }
      cudaMemcpyAsync(D.t, U(l), bytes, cudaMemcpyDeviceToDevice, s);
      k_negate<<<nblk(C.d.n_slots), kBlock, 0, s>>>(C.d.n_slots, C.u, C.ar);  // rh_{l-1} is formed later
      transfer<double>(H, l, false, C.ar, D.t, s);
    } else {
      cudaMemcpyAsync(D.t, U(l), bytes, cudaMemcpyDeviceToDevice, s);
    }
  }
  for (int l = H.L; l >= H.c; --l) {
    DevLevel& D = H.lv[l];
    sweep<double>(H, l, kResidual, U(l), Bv(l), D.r, nullptr, s);
    sweep<double>(H, l, kResidual, D.t, Bv(l), D.ar, nullptr, s);
    if (bpx && l > H.c) {
      DevLevel& C = H.lv[l - 1];
      if (H.dim == 2)
        k_bpx_correct<2><<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, D.dinv, D.r, D.ad, U(l));
      else
        k_bpx_correct<3><<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, D.dinv, D.r, D.ad, U(l));
      k_inject_level<<<nblk(C.d.n_slots), kBlock, 0, s>>>(C.d, C.child, D.r, C.ai);
      transfer<double>(H, l, true, D.ar, C.b, s);
      continue;
    }
    k_add_correct<<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, D.dinv, D.r, D.ad, U(l));
    if (l > H.c) {
      DevLevel& C = H.lv[l - 1];
      k_inject_level<<<nblk(C.d.n_slots), kBlock, 0, s>>>(C.d, C.child, U(l), C.u);
      transfer<double>(H, l, true, D.ar, C.b, s);
    }
  }
}

// the level iterates and corrections of the additive cycle start from zero
static mg_status additive_reset(Hier& H, double* u, cudaStream_t s) {
  for (int l = H.c; l <= H.L; ++l) {
    DevLevel& D = H.lv[l];
    const size_t bytes = static_cast<size_t>(D.d.n_slots) * sizeof(double);
    MG_TRY_CUDA(cudaMemsetAsync(D.ad, 0, bytes, s));
    if (D.ai) MG_TRY_CUDA(cudaMemsetAsync(D.ai, 0, bytes, s));
    if (l < H.L) MG_TRY_CUDA(cudaMemsetAsync(D.u, 0, bytes, s));
  }
  if (u) MG_TRY_CUDA(cudaMemsetAsync(u, 0, H.lv[H.L].d.n_slots * sizeof(double), s));
  return MG_OK;
}

static mg_status solve_additive(Hier& H, double* u, const double* b, double tol, int max_cycles,
                                mg_solve_stats* st, cudaStream_t s) {
  DevLevel& F = H.lv[H.L];
  MG_CHECK(additive_reset(H, u, s));
  residual_norm<double>(H, u, b, F.r, 0, s);
  MG_TRY_CUDA(cudaMemcpyAsync(H.h_pin, H.d_scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  MG_TRY_CUDA(cudaStreamSynchronize(s));
  const double r0 = std::sqrt(H.h_pin[0]);
  if (st) {
    st->r0_norm = r0;
    st->history_len = 0;
  }
  if (!std::isfinite(r0)) {
    set_error("mg_solve: non-finite initial residual");
    return MG_ERR_NONFINITE;
  }
  double rel = r0 > 0 ? 1.0 : 0.0;
  int cycles = 0;
  while (rel > tol && cycles < max_cycles) {
    MG_CHECK(graph_launch(H, H.g_add, u, b, s, [&](cudaStream_t ss) {
      additive_traversal(H, u, b, ss);
      residual_norm<double>(H, u, b, F.r, 0, ss);
      cudaMemcpyAsync(H.h_pin, H.d_scal, sizeof(double), cudaMemcpyDeviceToHost, ss);
    }));
    MG_TRY_CUDA(cudaStreamSynchronize(s));
    ++cycles;
    rel = std::sqrt(H.h_pin[0]) / r0;
    if (st && st->history && st->history_len < st->history_capacity) st->history[st->history_len++] = rel;
    if (!std::isfinite(rel)) {
      set_error("mg_solve: non-finite residual");
      if (st) st->cycles = cycles;
      return MG_ERR_NONFINITE;
    }
    if (rel > 1e6) {
      set_error("mg_solve: residual grew by more than 1e6 (diverged)");
      if (st) st->cycles = cycles;
      return MG_ERR_DIVERGED;
    }
  }
  if (st) {
    st->cycles = cycles;
    st->outer_steps = cycles;
    st->rel_residual = rel;
  }
  if (rel > tol) {
    set_error("mg_solve: not converged within max_cycles");
    return MG_ERR_NOT_CONVERGED;
  }
  return MG_OK;
}

// FP64 iterative refinement around FP32 V-cycles (Sect. 5 deltas decoded from 16 bits)
static mg_status solve_mixed(Hier& H, double* u, const double* b, double tol, int max_cycles, mg_solve_stats* st,
                             cudaStream_t s) {
  DevLevel& F = H.lv[H.L];
  const int64_t n = F.d.n_slots;
  const double inv_count = F.n_dofs > 0 ? 1.0 / static_cast<double>(F.n_dofs) : 0.0;
  MG_TRY_CUDA(cudaMemsetAsync(u, 0, n * sizeof(double), s));
  MG_TRY_CUDA(cudaMemsetAsync(F.u32, 0, n * sizeof(float), s));
  MG_TRY_CUDA(cudaMemsetAsync(H.d_scal + 2, 0, sizeof(double), s));
  residual_norm<double>(H, u, b, F.r, 0, s);
  MG_TRY_CUDA(cudaMemcpyAsync(H.h_pin, H.d_scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  MG_TRY_CUDA(cudaStreamSynchronize(s));
  const double r0 = std::sqrt(H.h_pin[0]);
  if (st) {
    st->r0_norm = r0;
    st->history_len = 0;
  }
  if (!std::isfinite(r0)) {
    set_error("mg_solve: non-finite initial residual");
    return MG_ERR_NONFINITE;
  }
  double rel = r0 > 0 ? 1.0 : 0.0;
  int cycles = 0, outer = 0;
  const int chunk = H.opt.inner_cycles > 0 ? H.opt.inner_cycles : 8;
  bool first = true;
  while (rel > tol && cycles < max_cycles) {
    // outer step: u += sigma e (skipped the first time), r = b - A u in FP64, b32 = r / sigma
    MG_CHECK(graph_launch(H, H.g_outer, u, b, s, [&](cudaStream_t ss) {
      k_update_f64<<<nblk(n), kBlock, 0, ss>>>(n, u, F.u32, H.d_scal + 2);
      residual_norm<double>(H, u, b, F.r, 0, ss);
      k_scale_to_f32<<<nblk(n), kBlock, 0, ss>>>(n, F.r, H.d_scal, inv_count, F.b32, H.d_scal + 2);
      cudaMemsetAsync(F.u32, 0, n * sizeof(float), ss);
      cudaMemcpyAsync(H.h_pin, H.d_scal, sizeof(double), cudaMemcpyDeviceToHost, ss);
    }));
    MG_TRY_CUDA(cudaStreamSynchronize(s));
    ++outer;
    rel = std::sqrt(H.h_pin[0]) / r0;
    if (!first && st && st->history && st->history_len < st->history_capacity) st->history[st->history_len++] = rel;
    first = false;
    if (!std::isfinite(rel)) {
      set_error("mg_solve: non-finite residual");
      return MG_ERR_NONFINITE;
    }
    if (rel > 1e6) {
      set_error("mg_solve: residual grew by more than 1e6 (diverged)");
      return MG_ERR_DIVERGED;
    }
    if (rel <= tol) break;
    // inner FP32 cycles until the correction equation is solved to what this step needs
    const double target = std::max(1e-5, 0.3 * tol / rel);
    double prev = 1.0;
    while (cycles < max_cycles) {
      MG_CHECK(graph_launch(H, H.g_inner, nullptr, nullptr, s, [&](cudaStream_t ss) {
        for (int k = 0; k < chunk; ++k) vcycle<float>(H, H.L, F.u32, F.b32, ss);
        residual_norm<float>(H, F.u32, F.b32, F.r32, 1, ss);
        cudaMemcpyAsync(H.h_pin + 1, H.d_scal + 1, sizeof(double), cudaMemcpyDeviceToHost, ss);
      }));
      MG_TRY_CUDA(cudaStreamSynchronize(s));
      cycles += chunk;
      const double inner = std::sqrt(H.h_pin[1] * inv_count);  // ||b32|| = sqrt(n_dofs)
      if (!std::isfinite(inner)) {
        set_error("mg_solve: non-finite FP32 inner residual");
        return MG_ERR_NONFINITE;
      }
      if (inner <= target || inner > 0.9 * prev) break;
      prev = inner;
    }
  }
  if (st) {
    st->cycles = cycles;
    st->outer_steps = outer;
    st->rel_residual = rel;
  }
  if (rel > tol) {
    set_error("mg_solve: not converged within max_cycles");
    return MG_ERR_NOT_CONVERGED;
  }
  return MG_OK;
}

// ---- composite grid (Sect. 3): level L refined in part over the complete level t = L - 1

template <typename T>
static void fill_hanging(const Hier& H, const T* ut, T* uL, cudaStream_t s) {
  const DevLevel& F = H.lv[H.L];
  if (H.n_hang_L == 0) return;
  if (H.dim == 2)
    k_hanging<2, T><<<nblk(H.n_hang_L), kBlock, 0, s>>>(F.d, F.hang_idx, F.hang_w, ut, uL, H.hang_L, H.n_hang_L);
  else
    k_hanging<3, T><<<nblk(H.n_hang_L), kBlock, 0, s>>>(F.d, F.hang_idx, F.hang_w, ut, uL, H.hang_L, H.n_hang_L);
}

template <typename T>
static void inject(const Hier& H, const T* uL, T* ut, cudaStream_t s) {
  const DevLevel& D = H.lv[H.top];
  k_inject<T><<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, H.child_top, uL, ut);
}

static inline unsigned norm_blocks(const DevLevel& D) {
  const int64_t cap = D.d.n_bricks * D.d.B;  // entries of D.partial
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(nblk(D.d.n_slots), cap)));
}

// composite residual: r_L = b_L - A_L u_L on level-L DoFs (norm^2 into d_scal[sL]);
// u_t refreshed by injection, r_t = b_t - A_t u_t on unrefined level-t DoFs (zero
// elsewhere, norm^2 into d_scal[st]).  Hanging entries of u_L must be current.
template <typename T>
static void comp_residual_norm(Hier& H, const T* uL, const T* bL, T* ut, const T* bt, int sL, int st,
                               cudaStream_t s) {
  DevLevel& D = H.lv[H.top];
  T* rt = lvec<T>(H, H.top, 2);
  sweep<T>(H, H.L, kResidual, uL, bL, lvec<T>(H, H.L, 2), H.d_scal + sL, s);
  inject<T>(H, uL, ut, s);
  sweep<T>(H, H.top, kResidual, ut, bt, rt, nullptr, s);
  k_masked_norm<T><<<norm_blocks(D), kBlock, 0, s>>>(D.d, rt, D.partial, D.counter, H.d_scal + st);
}

// One composite cycle (FAS two-level scheme on the hierarchical generating system,
// Sect. 3 with Alg. 1's smoother): pre-smooth level L with hanging values from
// level t, inject, form the level-t correction equation (R r_L at refined, the
// level-t residual at unrefined vertices), one V-cycle of the uniform levels
// t .. c for it, correct u_t (unrefined) and u_L (d-linear P), refresh the
// hanging values, post-smooth.  Expects hanging entries of u_L current on entry.
template <typename T>
static void composite_cycle(Hier& H, T* uL, const T* bL, T* ut, const T* bt, cudaStream_t s) {
  const int L = H.L, t = H.top;
  T* tmpL = lvec<T>(H, L, 3);
  T* rL = lvec<T>(H, L, 2);
  T* et = lvec<T>(H, t, 0);
  T* rhs = lvec<T>(H, t, 1);
  T* rt = lvec<T>(H, t, 2);
  const DevLevel& D = H.lv[t];
  smooth<T>(H, L, uL, bL, tmpL, H.opt.nu1, s);
  sweep<T>(H, L, kResidual, uL, bL, rL, nullptr, s);
  inject<T>(H, uL, ut, s);
  sweep<T>(H, t, kResidual, ut, bt, rt, nullptr, s);
  // d-linear R = P^T at refined level-t DoFs (no operator-dependent transfer on
  // level L), the level-t residual at unrefined ones, zero elsewhere
  k_compose_rhs<T><<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, rt, rhs);
  transfer<T>(H, L, true, rL, rhs, s, H.ref_top, H.n_ref_top);
  cudaMemsetAsync(et, 0, D.d.n_slots * sizeof(T), s);
  vcycle<T>(H, t, et, rhs, s);
  k_add_unrefined<T><<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, et, ut);
  transfer<T>(H, L, false, et, uL, s, H.dof_L, H.n_dof_L);
  fill_hanging<T>(H, ut, uL, s);
  smooth<T>(H, L, uL, bL, tmpL, H.opt.nu2, s);
}

struct CompVecs {
  double *uL, *ut;
  const double *bL, *bt;
};

static CompVecs comp_vecs(const Hier& H, double* u, const double* b) {
  const Grid& g = *H.g;
  const int64_t oL = g.levels[H.L].slot_offset, ot = g.levels[H.top].slot_offset;
  return CompVecs{u + oL, u + ot, b + oL, b + ot};
}

static mg_status solve_comp_fp64(Hier& H, double* u, const double* b, double tol, int max_cycles,
                                 mg_solve_stats* st, cudaStream_t s) {
  const CompVecs v = comp_vecs(H, u, b);
  const bool ff = H.lv[H.L].eps_pair != nullptr;  // float-float cycles first, as in solve_fp64
  struct Restore {
    Hier& h;
    ~Restore() { h.ff_active = true; }
  } restore{H};
  H.ff_active = false;
  MG_TRY_CUDA(cudaMemsetAsync(v.uL, 0, H.lv[H.L].d.n_slots * sizeof(double), s));
  MG_TRY_CUDA(cudaMemsetAsync(v.ut, 0, H.lv[H.top].d.n_slots * sizeof(double), s));
  comp_residual_norm<double>(H, v.uL, v.bL, v.ut, v.bt, 0, 4, s);
  MG_TRY_CUDA(cudaMemcpyAsync(H.h_pin, H.d_scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  MG_TRY_CUDA(cudaStreamSynchronize(s));
  const double r0 = std::sqrt(H.h_pin[0] + H.h_pin[4]);
  if (st) {
    st->r0_norm = r0;
    st->history_len = 0;
  }
  if (!std::isfinite(r0)) {
    set_error("mg_solve: non-finite initial residual");
    return MG_ERR_NONFINITE;
  }
  double rel = r0 > 0 ? 1.0 : 0.0;
  int cycles = 0;
  H.ff_active = ff && rel > kFfSwitch * tol;
  while (rel > tol && cycles < max_cycles) {
    MG_CHECK(graph_launch(H, H.ff_active ? H.g_comp_ff : H.g_comp64, u, b, s, [&](cudaStream_t ss) {
      composite_cycle<double>(H, v.uL, v.bL, v.ut, v.bt, ss);
      comp_residual_norm<double>(H, v.uL, v.bL, v.ut, v.bt, 0, 4, ss);
      cudaMemcpyAsync(H.h_pin, H.d_scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, ss);
    }));
    MG_TRY_CUDA(cudaStreamSynchronize(s));
    ++cycles;
    const double prev = rel;
    rel = std::sqrt(H.h_pin[0] + H.h_pin[4]) / r0;
    if (H.ff_active && (rel <= kFfSwitch * tol || rel > 0.95 * prev)) H.ff_active = false;
    if (st && st->history && st->history_len < st->history_capacity) st->history[st->history_len++] = rel;
    if (!std::isfinite(rel)) {
      set_error("mg_solve: non-finite residual");
      if (st) st->cycles = cycles;
      return MG_ERR_NONFINITE;
    }
    if (rel > 1e6) {
      set_error("mg_solve: residual grew by more than 1e6 (diverged)");
      if (st) st->cycles = cycles;
      return MG_ERR_DIVERGED;
    }
  }
  if (st) {
    st->cycles = cycles;
    st->outer_steps = cycles;
    st->rel_residual = rel;
  }
  if (rel > tol) {
    set_error("mg_solve: not converged within max_cycles");
    return MG_ERR_NOT_CONVERGED;
  }
  return MG_OK;
}

// FP64 iterative refinement around FP32 composite cycles: the composite residual
// (r_L, r_t) in FP64, scaled by sigma = sqrt(|r|^2 / n) into the FP32 correction
// equation, solved from zero by FP32 composite cycles, then u += sigma e on both levels
static mg_status solve_comp_mixed(Hier& H, double* u, const double* b, double tol, int max_cycles,
                                  mg_solve_stats* st, cudaStream_t s) {
  const CompVecs v = comp_vecs(H, u, b);
  DevLevel& F = H.lv[H.L];
  DevLevel& D = H.lv[H.top];
  const int64_t nL = F.d.n_slots, nt = D.d.n_slots;
  const double inv_count = H.n_comp_dofs > 0 ? 1.0 / static_cast<double>(H.n_comp_dofs) : 0.0;
  MG_TRY_CUDA(cudaMemsetAsync(v.uL, 0, nL * sizeof(double), s));
  MG_TRY_CUDA(cudaMemsetAsync(v.ut, 0, nt * sizeof(double), s));
  MG_TRY_CUDA(cudaMemsetAsync(F.u32, 0, nL * sizeof(float), s));
  MG_TRY_CUDA(cudaMemsetAsync(H.c32, 0, nt * sizeof(float), s));
  MG_TRY_CUDA(cudaMemsetAsync(H.d_scal + 2, 0, sizeof(double), s));
  comp_residual_norm<double>(H, v.uL, v.bL, v.ut, v.bt, 0, 4, s);
  MG_TRY_CUDA(cudaMemcpyAsync(H.h_pin, H.d_scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  MG_TRY_CUDA(cudaStreamSynchronize(s));
  const double r0 = std::sqrt(H.h_pin[0] + H.h_pin[4]);
  if (st) {
    st->r0_norm = r0;
    st->history_len = 0;
  }
  if (!std::isfinite(r0)) {
    set_error("mg_solve: non-finite initial residual");
    return MG_ERR_NONFINITE;
  }
  double rel = r0 > 0 ? 1.0 : 0.0;
  int cycles = 0, outer = 0;
  const int chunk = H.opt.inner_cycles > 0 ? H.opt.inner_cycles : 8;
  bool first = true;
  while (rel > tol && cycles < max_cycles) {
    MG_CHECK(graph_launch(H, H.g_comp_outer, u, b, s, [&](cudaStream_t ss) {
      k_update_f64<<<nblk(nL), kBlock, 0, ss>>>(nL, v.uL, F.u32, H.d_scal + 2);
      k_update_f64<<<nblk(nt), kBlock, 0, ss>>>(nt, v.ut, H.c32, H.d_scal + 2);
      fill_hanging<double>(H, v.ut, v.uL, ss);
      comp_residual_norm<double>(H, v.uL, v.bL, v.ut, v.bt, 0, 4, ss);
      k_sum2<<<1, 1, 0, ss>>>(H.d_scal, H.d_scal + 4, H.d_scal + 6);
      k_scale_to_f32<<<nblk(nL), kBlock, 0, ss>>>(nL, F.r, H.d_scal + 6, inv_count, F.b32, H.d_scal + 2);
      k_scale_to_f32<<<nblk(nt), kBlock, 0, ss>>>(nt, D.r, H.d_scal + 6, inv_count, H.cb32, H.d_scal + 2);
      cudaMemsetAsync(F.u32, 0, nL * sizeof(float), ss);
      cudaMemsetAsync(H.c32, 0, nt * sizeof(float), ss);
      cudaMemcpyAsync(H.h_pin, H.d_scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, ss);
    }));
    MG_TRY_CUDA(cudaStreamSynchronize(s));
    ++outer;
    rel = std::sqrt(H.h_pin[6]) / r0;
    if (!first && st && st->history && st->history_len < st->history_capacity) st->history[st->history_len++] = rel;
    first = false;
    if (!std::isfinite(rel)) {
      set_error("mg_solve: non-finite residual");
      return MG_ERR_NONFINITE;
    }
    if (rel > 1e6) {
      set_error("mg_solve: residual grew by more than 1e6 (diverged)");
      return MG_ERR_DIVERGED;
    }
    if (rel <= tol) break;
    const double target = std::max(1e-5, 0.3 * tol / rel);
    double prev = 1.0;
    while (cycles < max_cycles) {
      MG_CHECK(graph_launch(H, H.g_comp_inner, nullptr, nullptr, s, [&](cudaStream_t ss) {
        for (int k = 0; k < chunk; ++k) composite_cycle<float>(H, F.u32, F.b32, H.c32, H.cb32, ss);
        comp_residual_norm<float>(H, F.u32, F.b32, H.c32, H.cb32, 1, 5, ss);
        cudaMemcpyAsync(H.h_pin, H.d_scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, ss);
      }));
      MG_TRY_CUDA(cudaStreamSynchronize(s));
      cycles += chunk;
      const double inner = std::sqrt((H.h_pin[1] + H.h_pin[5]) * inv_count);
      if (!std::isfinite(inner)) {
        set_error("mg_solve: non-finite FP32 inner residual");
        return MG_ERR_NONFINITE;
      }
      if (inner <= target || inner > 0.9 * prev) break;
      prev = inner;
    }
  }
  if (st) {
    st->cycles = cycles;
    st->outer_steps = outer;
    st->rel_residual = rel;
  }
  if (rel > tol) {
    set_error("mg_solve: not converged within max_cycles");
    return MG_ERR_NOT_CONVERGED;
  }
  return MG_OK;
}

// ---- persistent cooperative solve -------------------------------------------------

template <typename T>
static PLevel<T> make_plevel(const Hier& H, int l, T* u_fin, const T* b_fin) {
  const DevLevel& D = H.lv[l];
  PLevel<T> P{};
  P.d = D.d;
  const bool coarse = l < H.top;
  if constexpr (std::is_same<T, double>::value) {
    P.eps = D.eps;
    P.ahat = (coarse && H.galerkin) ? D.ahat : nullptr;
    P.phat = (coarse && H.boxmg) ? D.phat : nullptr;
    P.u = coarse ? D.u : u_fin;
    P.b = coarse ? D.b : const_cast<T*>(b_fin);
    P.r = D.r;
    P.t = D.t;
  } else {
    P.eps = D.eps32;
    P.ahat = (coarse && H.galerkin) ? D.a16 : nullptr;
    P.ascale = (coarse && H.galerkin) ? D.ascale : nullptr;
    P.phat = (coarse && H.boxmg) ? D.p16 : nullptr;
    P.pscale = (coarse && H.boxmg) ? D.pscale : nullptr;
    P.u = D.u32;
    P.b = D.b32;
    P.r = D.r32;
    P.t = D.t32;
  }
  P.R = pick_slab(D.d.B, D.d.n_bricks, kSweepTargetCtas);
  P.nitems = static_cast<int>(D.d.n_bricks * (D.d.B / P.R));
  return P;
}

template <typename T>
static size_t tile_bytes(const Hier& H, int l, int R) {
  const int B = H.lv[l].d.B;
  return H.dim == 2 ? sweep_tile_bytes<2, T>(B, R) : sweep_tile_bytes<3, T>(B, R);
}

static mg_status solve_persistent(Hier& H, double* u, const double* b, double tol, int max_cycles,
                                  mg_solve_stats* st, cudaStream_t s) {
  DevLevel& Fd = H.lv[H.L];
  MG_TRY_CUDA(cudaMemsetAsync(u, 0, Fd.d.n_slots * sizeof(double), s));
  const int amc = H.galerkin ? (H.mixed ? (H.fmt == 1 ? 2 : 3) : 1) : 0;
  const int pm = H.boxmg ? (H.mixed ? (H.fmt == 1 ? 2 : 3) : 1) : 0;
  int grid = 0;
  cudaError_t e;
  if (!H.mixed) {
    PSolve<double> p{};
    p.L = H.L;
    p.c = H.c;
    p.nu1 = H.opt.nu1;
    p.nu2 = H.opt.nu2;
    p.omega = H.opt.omega;
    size_t smem = 0;
    for (int l = H.c; l <= H.L; ++l) {
      p.lv[l] = make_plevel<double>(H, l, u, b);
      smem = std::max(smem, tile_bytes<double>(H, l, p.lv[l].R));
    }
    p.chol = H.c_mat;
    p.n_c = H.n_c;
    p.c_slots = H.c_slots;
    p.partial = Fd.partial;
    p.hist = H.d_hist;
    p.hist_cap = kHistCap;
    p.out_int = H.d_pint;
    p.out_dbl = H.d_pdbl;
    p.tol = tol;
    p.max_cycles = max_cycles;
    MG_TRY_CUDA(cudaMemcpyAsync(H.d_psolve, &p, sizeof(p), cudaMemcpyHostToDevice, s));
    e = H.dim == 2 ? persist_launch_fp64<2>(static_cast<const PSolve<double>*>(H.d_psolve), amc, pm, smem, s, &grid)
                   : persist_launch_fp64<3>(static_cast<const PSolve<double>*>(H.d_psolve), amc, pm, smem, s, &grid);
  } else {
    PSolve<float> p{};
    p.L = H.L;
    p.c = H.c;
    p.nu1 = H.opt.nu1;
    p.nu2 = H.opt.nu2;
    p.omega = static_cast<float>(H.opt.omega);
    size_t smem = 0;
    for (int l = H.c; l <= H.L; ++l) {
      p.lv[l] = make_plevel<float>(H, l, nullptr, nullptr);
      smem = std::max(smem, tile_bytes<float>(H, l, p.lv[l].R));
    }
    p.f64 = make_plevel<double>(H, H.L, u, b);
    smem = std::max(smem, tile_bytes<double>(H, H.L, p.f64.R));
    p.chol = H.c_mat;
    p.n_c = H.n_c;
    p.c_slots = H.c_slots;
    p.partial = Fd.partial;
    p.hist = H.d_hist;
    p.hist_cap = kHistCap;
    p.out_int = H.d_pint;
    p.out_dbl = H.d_pdbl;
    p.tol = tol;
    p.max_cycles = max_cycles;
    p.inv_count = Fd.n_dofs > 0 ? 1.0 / static_cast<double>(Fd.n_dofs) : 0.0;
    MG_TRY_CUDA(cudaMemcpyAsync(H.d_psolve, &p, sizeof(p), cudaMemcpyHostToDevice, s));
    e = H.dim == 2 ? persist_launch_mixed<2>(static_cast<const PSolve<float>*>(H.d_psolve), amc, pm, smem, s, &grid)
                   : persist_launch_mixed<3>(static_cast<const PSolve<float>*>(H.d_psolve), amc, pm, smem, s, &grid);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("persistent solve launch: ") + cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  MG_TRY_CUDA(cudaMemcpyAsync(H.h_pin + 8, H.d_pdbl, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  MG_TRY_CUDA(cudaMemcpyAsync(reinterpret_cast<int*>(H.h_pin + 12), H.d_pint, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
  MG_TRY_CUDA(cudaStreamSynchronize(s));
  const int* oi = reinterpret_cast<const int*>(H.h_pin + 12);
  const int cycles = oi[0], outer = oi[1], status = oi[2];
  const double r0 = H.h_pin[8], rel = H.h_pin[9];
  if (st) {
    st->cycles = cycles;
    st->outer_steps = outer;
    st->r0_norm = r0;
    st->rel_residual = rel;
    const int nh = std::min(H.mixed ? std::max(outer - 1, 0) : cycles, std::min(st->history_capacity, kHistCap));
    st->history_len = 0;
    if (st->history && nh > 0) {
      MG_TRY_CUDA(cudaMemcpy(st->history, H.d_hist, nh * sizeof(double), cudaMemcpyDeviceToHost));
      st->history_len = nh;
    }
  }
  if (status == 2) {
    set_error("mg_solve: non-finite residual");
    return MG_ERR_NONFINITE;
  }
  if (status == 3) {
    set_error("mg_solve: residual grew by more than 1e6 (diverged)");
    return MG_ERR_DIVERGED;
  }
  if (status == 1) {
    set_error("mg_solve: not converged within max_cycles");
    return MG_ERR_NOT_CONVERGED;
  }
  return MG_OK;
}

}  // namespace mg

using namespace mg;

// ----------------------------------------------------------------------------- C ABI

static Hier* H_(mg_hier* h) { return reinterpret_cast<Hier*>(h); }

static mg_status check_level(Hier* H, int level, bool need_ready) {
  if (!H) {
    set_error("NULL hierarchy");
    return MG_ERR_INVALID_ARG;
  }
  if (level < H->c || level > H->L) {
    set_error("level outside [coarsest, max_level]");
    return MG_ERR_INVALID_ARG;
  }
  if (need_ready && !H->ready) {
    set_error("hierarchy not set up (call mg_setup)");
    return MG_ERR_INVALID_ARG;
  }
  return MG_OK;
}

extern "C" {

void mg_default_options(mg_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->transfer = MG_TRANSFER_BOXMG;
  o->coarse = MG_COARSE_GALERKIN;
  o->precision = MG_PREC_FP64;
  o->nu1 = 2;
  o->nu2 = 2;
  o->omega = 0.6;
  o->coarsest_level = 1;
  o->inner_cycles = 8;
  o->use_graphs = 1;
  o->persistent = 0;
  o->eps_mf = 1e-4;
  o->smoother = MG_SMOOTH_JACOBI;
  o->gs_sweeps = 1;
  o->cycle = MG_CYCLE_V;
}

mg_status mg_hier_create(const mg_grid* grid, const mg_options* opt, mg_hier** out) {
  if (!grid || !out) {
    set_error("mg_hier_create: NULL argument");
    return MG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  mg_options o;
  if (opt)
    o = *opt;
  else
    mg_default_options(&o);
  return hier_create(reinterpret_cast<const Grid*>(grid), o, 0, reinterpret_cast<Hier**>(out));
}

mg_status mg_hier_footprint(const mg_grid* grid, const mg_options* opt, size_t* bytes) {
  if (!grid || !bytes) {
    set_error("mg_hier_footprint: NULL argument");
    return MG_ERR_INVALID_ARG;
  }
  mg_options o;
  if (opt)
    o = *opt;
  else
    mg_default_options(&o);
  const Grid* g = reinterpret_cast<const Grid*>(grid);
  if (o.coarsest_level < 1 || o.coarsest_level >= g->L) {
    set_error("mg_hier_footprint: invalid coarsest level");
    return MG_ERR_INVALID_ARG;
  }
  *bytes = hier_footprint(*g, o);
  return MG_OK;
}

mg_status mg_setup(mg_hier* h, const double* eps, void* stream) {
  Hier* H = H_(h);
  if (!H || !eps) {
    set_error("mg_setup: NULL argument");
    return MG_ERR_INVALID_ARG;
  }
  H->ready = false;
  return run_setup(*H, eps, pick(*H, stream));
}

mg_status mg_setup_tensor(mg_hier* h, const double* eps_axes, void* stream) {
  Hier* H = H_(h);
  if (!H || !eps_axes) {
    set_error("mg_setup_tensor: NULL argument");
    return MG_ERR_INVALID_ARG;
  }
  if (!H->tensor) {
    set_error("mg_setup_tensor: the hierarchy was created without tensor_coefficients");
    return MG_ERR_INVALID_ARG;
  }
  H->ready = false;
  cudaStream_t s = pick(*H, stream);
  return run_setup(*H, nullptr, s, true, eps_axes);
}

mg_status mg_smooth(mg_hier* h, int level, double* u, const double* b, int nu, void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, level, true));
  if (!u || !b || nu < 0) {
    set_error("mg_smooth: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  smooth<double>(*H, level, u, b, H->lv[level].t, nu, pick(*H, stream));
  return last_launch("mg_smooth");
}

mg_status mg_residual(mg_hier* h, int level, const double* u, const double* b, double* r, double* norm2_host,
                      void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, level, true));
  if (!u || !b || !r) {
    set_error("mg_residual: NULL vector");
    return MG_ERR_INVALID_ARG;
  }
  cudaStream_t s = pick(*H, stream);
  sweep<double>(*H, level, kResidual, u, b, r, norm2_host ? H->d_scal + 3 : nullptr, s);
  if (norm2_host) {
    MG_TRY_CUDA(cudaMemcpyAsync(H->h_pin + 3, H->d_scal + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
    MG_TRY_CUDA(cudaStreamSynchronize(s));
    *norm2_host = H->h_pin[3];
  }
  return last_launch("mg_residual");
}

static mg_status check_mixed(Hier* H, const char* what) {
  if (!H->mixed) {
    set_error(std::string(what) + ": needs a mixed-precision hierarchy");
    return MG_ERR_INVALID_ARG;
  }
  return MG_OK;
}

mg_status mg_smooth_f32(mg_hier* h, int level, float* u, const float* b, int nu, void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, level, true));
  MG_CHECK(check_mixed(H, "mg_smooth_f32"));
  if (!u || !b || nu < 0) {
    set_error("mg_smooth_f32: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  smooth<float>(*H, level, u, b, H->lv[level].t32, nu, pick(*H, stream));
  return last_launch("mg_smooth_f32");
}

mg_status mg_residual_f32(mg_hier* h, int level, const float* u, const float* b, float* r, double* norm2_host,
                          void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, level, true));
  MG_CHECK(check_mixed(H, "mg_residual_f32"));
  if (!u || !b || !r) {
    set_error("mg_residual_f32: NULL vector");
    return MG_ERR_INVALID_ARG;
  }
  cudaStream_t s = pick(*H, stream);
  sweep<float>(*H, level, kResidual, u, b, r, norm2_host ? H->d_scal + 3 : nullptr, s);
  if (norm2_host) {
    MG_TRY_CUDA(cudaMemcpyAsync(H->h_pin + 3, H->d_scal + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
    MG_TRY_CUDA(cudaStreamSynchronize(s));
    *norm2_host = H->h_pin[3];
  }
  return last_launch("mg_residual_f32");
}

mg_status mg_vcycle_f32(mg_hier* h, float* u, const float* b, void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, H ? H->L : 0, true));
  MG_CHECK(check_mixed(H, "mg_vcycle_f32"));
  if (!u || !b) {
    set_error("mg_vcycle_f32: NULL vector");
    return MG_ERR_INVALID_ARG;
  }
  if (H->adaptive) {
    set_error("mg_vcycle_f32: adaptive hierarchies run FP32 composite cycles inside mg_solve only");
    return MG_ERR_UNSUPPORTED;
  }
  vcycle<float>(*H, H->L, u, b, pick(*H, stream));
  return last_launch("mg_vcycle_f32");
}

mg_status mg_restrict(mg_hier* h, int fine_level, const double* r_fine, double* b_coarse, void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, fine_level, true));
  if (fine_level == H->c || !r_fine || !b_coarse) {
    set_error("mg_restrict: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  transfer<double>(*H, fine_level, true, r_fine, b_coarse, pick(*H, stream));
  return last_launch("mg_restrict");
}

mg_status mg_prolong(mg_hier* h, int fine_level, const double* e_coarse, double* u_fine, void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, fine_level, true));
  if (fine_level == H->c || !e_coarse || !u_fine) {
    set_error("mg_prolong: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  transfer<double>(*H, fine_level, false, e_coarse, u_fine, pick(*H, stream));
  return last_launch("mg_prolong");
}

mg_status mg_interpolate_hanging(mg_hier* h, int level, const double* u_coarse, double* u_fine, void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, level, false));
  if (level == H->c || !u_coarse || !u_fine) {
    set_error("mg_interpolate_hanging: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  DevLevel& F = H->lv[level];
  cudaStream_t s = pick(*H, stream);
  if (H->dim == 2)
    k_hanging<2, double><<<nblk(F.d.n_slots), kBlock, 0, s>>>(F.d, F.hang_idx, F.hang_w, u_coarse, u_fine,
                                                              nullptr, 0);
  else
    k_hanging<3, double><<<nblk(F.d.n_slots), kBlock, 0, s>>>(F.d, F.hang_idx, F.hang_w, u_coarse, u_fine,
                                                              nullptr, 0);
  return last_launch("mg_interpolate_hanging");
}

mg_status mg_autotune(mg_hier* h, int32_t* chosen, void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, H ? H->L : 0, true));
  cudaStream_t s = pick(*H, stream);
  for (int l = H->c; l <= H->L; ++l) {
    DevLevel& D = H->lv[l];
    int r64 = 0, r32 = 0;
    if (D.dinv || l == H->L) MG_CHECK(tune_level<double>(*H, l, s, &r64));  // FP64 sweeps of this hierarchy
    if (H->mixed) MG_CHECK(tune_level<float>(*H, l, s, &r32));
    D.R64 = r64;
    D.R32 = r32;
    if (chosen) {
      chosen[2 * l] = r64;
      chosen[2 * l + 1] = r32;
    }
  }
  // captured cycles carry the old launch shapes
  H->g_cycle64.reset();
  H->g_cycle_ff.reset();
  for (auto& gr : H->g_fused)
    for (Graph& g : gr) g.reset();
  H->g_comp_ff.reset();
  H->g_outer.reset();
  H->g_inner.reset();
  H->g_comp64.reset();
  H->g_comp_outer.reset();
  H->g_comp_inner.reset();
  H->g_add.reset();
  return MG_OK;
}

mg_status mg_vcycle(mg_hier* h, double* u, const double* b, void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, H ? H->L : 0, true));
  if (!u || !b) {
    set_error("mg_vcycle: NULL vector");
    return MG_ERR_INVALID_ARG;
  }
  cudaStream_t s = pick(*H, stream);
  if (H->adaptive) {  // one composite cycle on the level-concatenated vectors
    const CompVecs v = comp_vecs(*H, u, b);
    fill_hanging<double>(*H, v.ut, v.uL, s);
    composite_cycle<double>(*H, v.uL, v.bL, v.ut, v.bt, s);
    inject<double>(*H, v.uL, v.ut, s);
  } else if (H->opt.cycle != MG_CYCLE_V) {
    additive_traversal(*H, u, b, s);  // on the stored coarse iterates and corrections
  } else {
    vcycle<double>(*H, H->L, u, b, s);
  }
  return last_launch("mg_vcycle");
}

mg_status mg_solve(mg_hier* h, double* u, const double* b, double rel_tol, int max_cycles, mg_solve_stats* stats,
                   void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, H ? H->L : 0, true));
  if (!u || !b || max_cycles < 0 || !(rel_tol >= 0.0)) {
    set_error("mg_solve: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  cudaStream_t s = pick(*H, stream);
  const auto t0 = std::chrono::steady_clock::now();
  const bool persistent = H->opt.persistent && !H->adaptive && H->fmt != 4 && H->opt.smoother == MG_SMOOTH_JACOBI &&
                          H->opt.cycle == MG_CYCLE_V &&
                          H->n_c <= 64 && H->L < kMaxLevels;
  const mg_status st = H->adaptive ? (H->mixed ? solve_comp_mixed(*H, u, b, rel_tol, max_cycles, stats, s)
                                                 : solve_comp_fp64(*H, u, b, rel_tol, max_cycles, stats, s))
                       : H->opt.cycle != MG_CYCLE_V ? solve_additive(*H, u, b, rel_tol, max_cycles, stats, s)
                       : persistent ? solve_persistent(*H, u, b, rel_tol, max_cycles, stats, s)
                       : H->mixed   ? solve_mixed(*H, u, b, rel_tol, max_cycles, stats, s)
                                    : solve_fp64(*H, u, b, rel_tol, max_cycles, stats, s);
  if (stats)
    stats->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return st;
}

mg_status mg_get_stencils(mg_hier* h, int level, double* st, void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, level, true));
  if (!st) {
    set_error("mg_get_stencils: NULL output");
    return MG_ERR_INVALID_ARG;
  }
  DevLevel& D = H->lv[level];
  const double* ah = (level < H->top && H->galerkin) ? D.ahat : nullptr;
  cudaStream_t s = pick(*H, stream);
  if (H->dim == 2)
    k_export_stencils<2><<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, D.eps, ah, st, nullptr, D.aniso);
  else
    k_export_stencils<3><<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, D.eps, ah, st, nullptr, D.aniso);
  return last_launch("mg_get_stencils");
}

// brick-major planes -> offset-major export
__global__ void k_planes_to_offset_major(mg::LevelDesc L, int K, const double* in, double* out) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(mg::kBlock) + threadIdx.x;
  if (s >= L.n_slots) return;
  for (int k = 0; k < K; ++k) out[k * L.n_slots + s] = in[mg::plane_index(L, s, k, K)];
}
__global__ void k_planes16_to_offset_major(mg::LevelDesc L, int K, const uint16_t* in, uint16_t* out) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(mg::kBlock) + threadIdx.x;
  if (s >= L.n_slots) return;
  for (int k = 0; k < K; ++k) out[k * L.n_slots + s] = in[mg::plane_index(L, s, k, K)];
}

mg_status mg_get_deltas(mg_hier* h, int level, double* a_hat, double* p_hat, void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, level, true));
  if (level >= H->top) {
    set_error("mg_get_deltas: the finest complete level and above store no deltas");
    return MG_ERR_INVALID_ARG;
  }
  DevLevel& D = H->lv[level];
  cudaStream_t s = pick(*H, stream);
  if (a_hat) {
    if (!D.ahat) {
      set_error("mg_get_deltas: no Galerkin deltas (coarse = redisc)");
      return MG_ERR_INVALID_ARG;
    }
    k_planes_to_offset_major<<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, ipow(3, H->dim), D.ahat, a_hat);
  }
  if (p_hat) {
    if (!D.phat) {
      set_error("mg_get_deltas: no BoxMG deltas (transfer = dlinear)");
      return MG_ERR_INVALID_ARG;
    }
    k_planes_to_offset_major<<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, ipow(5, H->dim), D.phat, p_hat);
  }
  return last_launch("mg_get_deltas");
}

mg_status mg_get_codes(mg_hier* h, int level, uint16_t* a_codes, float* a_scale, uint16_t* p_codes, float* p_scale,
                       void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, level, true));
  if (!H->mixed || level >= H->top) {
    set_error("mg_get_codes: no codes (FP64 hierarchy or finest level)");
    return MG_ERR_INVALID_ARG;
  }
  DevLevel& D = H->lv[level];
  cudaStream_t s = pick(*H, stream);
  const size_t ns = static_cast<size_t>(D.d.n_slots);
  if (a_codes && D.a16)
    k_planes16_to_offset_major<<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, ipow(3, H->dim), D.a16, a_codes);
  if (a_scale && D.ascale) MG_TRY_CUDA(cudaMemcpyAsync(a_scale, D.ascale, ns * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (p_codes && D.p16)
    k_planes16_to_offset_major<<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, ipow(5, H->dim), D.p16, p_codes);
  if (p_scale && D.pscale) MG_TRY_CUDA(cudaMemcpyAsync(p_scale, D.pscale, ns * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return last_launch("mg_get_codes");
}

mg_status mg_get_code_lo(mg_hier* h, int level, uint16_t* a_lo, void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, level, true));
  if (!H->mixed || level >= H->top || !H->lv[level].a16 || !a_lo) {
    set_error("mg_get_code_lo: no A_hat codes (FP64 or bpa hierarchy, finest level, or no Galerkin operator)");
    return MG_ERR_INVALID_ARG;
  }
  DevLevel& D = H->lv[level];
  cudaStream_t s = pick(*H, stream);
  k_planes16_to_offset_major<<<nblk(D.d.n_slots), kBlock, 0, s>>>(D.d, ipow(3, H->dim),
                                                                    D.a16 + D.d.n_slots * ipow(3, H->dim), a_lo);
  return last_launch("mg_get_code_lo");
}

mg_status mg_encode_deltas_promote(int64_t n, int k, const double* delta, const double* diag, int fmt,
                                   uint16_t* codes, uint16_t* lo, float* scale, void* stream) {
  if (n < 0 || k <= 0 || (n > 0 && (!delta || !diag || !codes || !lo || !scale)) || (fmt != 1 && fmt != 2)) {
    set_error("mg_encode_deltas_promote: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  if (n == 0) return MG_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (fmt == 1)
    k_encode_rows_promote<1><<<nblk(n), kBlock, 0, s>>>(n, k, delta, diag, codes, lo, scale);
  else
    k_encode_rows_promote<2><<<nblk(n), kBlock, 0, s>>>(n, k, delta, diag, codes, lo, scale);
  return last_launch("mg_encode_deltas_promote");
}

mg_status mg_encode_deltas(int64_t n, int k, const double* delta, int fmt, uint16_t* codes, float* scale,
                           void* stream) {
  if (n < 0 || k <= 0 || (n > 0 && (!delta || !codes || !scale)) || (fmt != 1 && fmt != 2)) {
    set_error("mg_encode_deltas: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  if (n == 0) return MG_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (fmt == 1)
    k_encode_rows<1><<<nblk(n), kBlock, 0, s>>>(n, k, delta, codes, scale);
  else
    k_encode_rows<2><<<nblk(n), kBlock, 0, s>>>(n, k, delta, codes, scale);
  return last_launch("mg_encode_deltas");
}

mg_status mg_bpa_encode(int64_t n, int32_t k, const double* x, double eps_mf, uint64_t* rec, uint8_t* bytes,
                        uint64_t* total_bytes, int32_t* status, void* stream) {
  if (n < 0 || k <= 0 || k > 125 || !(eps_mf >= 0.0) || !total_bytes || (n > 0 && (!x || !rec || !bytes))) {
    set_error("mg_bpa_encode: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (status) MG_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), s));
  BpaSrc src{x, k, false, LevelDesc{}};
  bpa_encode_enqueue(src, n, eps_mf, rec, bytes, total_bytes, status, 1, 2, s);
  return last_launch("mg_bpa_encode");
}

mg_status mg_bpa_decode(int64_t n, int32_t k, const uint64_t* rec, const uint8_t* bytes, int32_t fp32, void* out,
                        void* stream) {
  if (n < 0 || k <= 0 || (n > 0 && (!rec || !bytes || !out))) {
    set_error("mg_bpa_decode: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  if (n == 0) return MG_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (fp32)
    k_bpa_decode<float><<<nblk(n), kBlock, 0, s>>>(n, k, rec, bytes, static_cast<float*>(out));
  else
    k_bpa_decode<double><<<nblk(n), kBlock, 0, s>>>(n, k, rec, bytes, static_cast<double*>(out));
  return last_launch("mg_bpa_decode");
}

mg_status mg_get_bpa(mg_hier* h, int level, uint64_t* a_rec, uint8_t* a_stream, uint64_t* p_rec, uint8_t* p_stream,
                     uint64_t* a_bytes, uint64_t* p_bytes, void* stream) {
  Hier* H = H_(h);
  MG_CHECK(check_level(H, level, true));
  if (H->fmt != 4 || level >= H->top) {
    set_error("mg_get_bpa: no bpa streams (not a MG_PREC_MIXED_BPA hierarchy, or the finest level)");
    return MG_ERR_INVALID_ARG;
  }
  DevLevel& D = H->lv[level];
  cudaStream_t s = pick(*H, stream);
  const size_t ns = static_cast<size_t>(D.d.n_slots);
  const size_t n3 = ipow(3, H->dim), n5 = ipow(5, H->dim);
  uint64_t used[2] = {0, 0};
  MG_TRY_CUDA(cudaMemcpyAsync(used, H->bpa_used + 2 * level, sizeof(used), cudaMemcpyDeviceToHost, s));
  if (a_rec && D.abpa_rec) MG_TRY_CUDA(cudaMemcpyAsync(a_rec, D.abpa_rec, ns * 8, cudaMemcpyDeviceToDevice, s));
  if (a_stream && D.abpa) MG_TRY_CUDA(cudaMemcpyAsync(a_stream, D.abpa, ns * n3 * 8, cudaMemcpyDeviceToDevice, s));
  if (p_rec && D.pbpa_rec) MG_TRY_CUDA(cudaMemcpyAsync(p_rec, D.pbpa_rec, ns * 8, cudaMemcpyDeviceToDevice, s));
  if (p_stream && D.pbpa) MG_TRY_CUDA(cudaMemcpyAsync(p_stream, D.pbpa, ns * n5 * 8, cudaMemcpyDeviceToDevice, s));
  MG_TRY_CUDA(cudaStreamSynchronize(s));
  if (a_bytes) *a_bytes = D.abpa ? used[0] : 0;
  if (p_bytes) *p_bytes = D.pbpa ? used[1] : 0;
  return last_launch("mg_get_bpa");
}

mg_status mg_get_coarsest(mg_hier* h, int32_t* level) {
  Hier* H = H_(h);
  if (!H || !level) {
    set_error("mg_get_coarsest: NULL argument");
    return MG_ERR_INVALID_ARG;
  }
  *level = H->c;
  return MG_OK;
}

void mg_destroy_hier(mg_hier* h) { free_hier(H_(h), true); }

}  // extern "C"
