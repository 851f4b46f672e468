// Setup kernels (A8-A11): coarse coefficients, BoxMG P, Galerkin R A P, delta
// encoding, coarsest-level dense Cholesky, plus stencil export.
#pragma once

#include "device.cuh"

namespace mg {

// Leaf coefficients from the level-concatenated input: existing unrefined cells take
// eps_in, every other slot 0.
__global__ void k_leaf_eps(LevelDesc L, const uint8_t* cflags, const double* eps_in, double* eps);

// Refined cells take the arithmetic mean of their 3^d children (the build's reading
// of the coarse rediscretisation coefficient).
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_mean_eps(LevelDesc Lc, LevelDesc Lf, const uint8_t* cflags_c,
                                                       const double* eps_f, double* eps_c) {
  const int64_t cs = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (cs >= Lc.n_slots) return;
  if (!(cflags_c[cs] & MG_C_REFINED)) return;
  int X[DIM];
  if (!coords_of<DIM>(Lc, cs, X)) return;
  double s = 0.0;
  for (int k = 0; k < cpow(3, DIM); ++k) {
    int y[DIM], kk = k;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      y[i] = 3 * X[i] + kk % 3;
      kk /= 3;
    }
    const int64_t fs = slot_of<DIM>(Lf, y);
    s += eps_f[fs];
  }
  eps_c[cs] = s / static_cast<double>(cpow(3, DIM));
}

// Gaussian elimination with partial pivoting on a small dense system (n <= 8).
template <int NMAX>
__device__ __forceinline__ bool small_solve(double (&M)[NMAX][NMAX], double (&rhs)[NMAX], int n) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    double best = fabs(M[c][c]);
    for (int r = c + 1; r < n; ++r)
      if (fabs(M[r][c]) > best) {
        best = fabs(M[r][c]);
        piv = r;
      }
    if (!(best > 0.0)) return false;
    if (piv != c) {
      for (int j = 0; j < n; ++j) {
        const double t = M[c][j];
        M[c][j] = M[piv][j];
        M[piv][j] = t;
      }
      const double t = rhs[c];
      rhs[c] = rhs[piv];
      rhs[piv] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      const double f = M[r][c] / M[c][c];
      for (int j = c; j < n; ++j) M[r][j] -= f * M[c][j];
      rhs[r] -= f * rhs[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = rhs[r];
    for (int j = r + 1; j < n; ++j) s -= M[r][j] * rhs[j];
    rhs[r] = s / M[r][r];
  }
  return true;
}

// BoxMG prolongation (Sect. 4.4, App. C).  One thread per coarse vertex V and
// patch (sign vector sigma, one of the 2^d cells around V): the 3^d P entries of
// V inside the patch solve C(s) p = f in the reference orientation: c-point p = 1, then for
// each set N of non-zero axes (lines, then faces, then the interior) the
// 2^|N| unknowns with exactly those axes non-zero, from stencils collapsed over
// the other axes; unknowns at reference coordinate 3 vanish.  The system is
// block lower-triangular in that order, so it is solved block by block.  An
// entry lying on a line / face through V is written by the patch with
// sigma_i = +1 on its zero axes.  Output: P_hat = P - P_dlin on 5^d planes.
template <int DIM>
__global__ void __launch_bounds__(64) k_boxmg(LevelDesc Lc, LevelDesc Lf, const double* eps_f,
                                                const double* ahat_f, double* phat_c, int* status) {
  constexpr int N3 = cpow(3, DIM), N5 = cpow(5, DIM);
  // one thread per (coarse slot, patch): the patches of a vertex write disjoint entries
  const int64_t tid = blockIdx.x * static_cast<int64_t>(64) + threadIdx.x;
  const int64_t cs = tid >> DIM;
  const int sg = static_cast<int>(tid & ((1 << DIM) - 1));
  if (cs >= Lc.n_slots) return;
  int V[DIM];
  const bool valid = coords_of<DIM>(Lc, cs, V);
  if (!valid || !is_dof(Lc.vflags[cs])) {
    if (valid && sg == 0)
      for (int k = 0; k < N5; ++k) phat_c[plane_index(Lc, cs, k, N5)] = 0.0;
    return;
  }
  {
    int sigma[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) sigma[i] = ((sg >> i) & 1) ? -1 : 1;
    double p[N3];
    for (int k = 0; k < N3; ++k) p[k] = 0.0;
    p[0] = 1.0;  // reference position 0 is lexicographic index 0 ({0,1,2}^d)
    // subsets of axes ordered by size
    for (int sz = 1; sz <= DIM; ++sz) {
      for (int mask = 1; mask < (1 << DIM); ++mask) {
        if (__popc(mask) != sz) continue;
        const int nunk = 1 << sz;
        double M[8][8], rhs[8];
        int rpos[8][DIM];
        for (int j = 0; j < nunk; ++j) {
          int bit = 0;
#pragma unroll
          for (int i = 0; i < DIM; ++i) {
            if ((mask >> i) & 1) {
              rpos[j][i] = 1 + ((j >> bit) & 1);
              ++bit;
            } else {
              rpos[j][i] = 0;
            }
          }
          for (int q = 0; q < nunk; ++q) M[j][q] = 0.0;
          rhs[j] = 0.0;
        }
        for (int j = 0; j < nunk; ++j) {
          int xf[DIM];
#pragma unroll
          for (int i = 0; i < DIM; ++i) xf[i] = 3 * V[i] + sigma[i] * rpos[j][i];
          const int64_t fsl = slot_of<DIM>(Lf, xf);
          double st[N3];
          full_stencil<DIM>(Lf, eps_f, ahat_f, xf, fsl, st);
          for (int k = 0; k < N3; ++k) {
            int o[DIM], kk = k;
#pragma unroll
            for (int i = 0; i < DIM; ++i) {
              o[i] = kk % 3 - 1;
              kk /= 3;
            }
            // reference offset o looks at actual offset sigma*o
            int ka = 0, m = 1;
#pragma unroll
            for (int i = 0; i < DIM; ++i) {
              ka += (sigma[i] * o[i] + 1) * m;
              m *= 3;
            }
            const double sv = st[ka];
            int t[DIM];
            bool zero = false, inblock = true;
#pragma unroll
            for (int i = 0; i < DIM; ++i) {
              t[i] = ((mask >> i) & 1) ? rpos[j][i] + o[i] : 0;
              if (t[i] == 3) zero = true;
              if (((mask >> i) & 1) && t[i] == 0) inblock = false;
            }
            if (zero) continue;
            if (inblock) {
              int q = 0, bit = 0;
#pragma unroll
              for (int i = 0; i < DIM; ++i)
                if ((mask >> i) & 1) {
                  q |= (t[i] - 1) << bit;
                  ++bit;
                }
              M[j][q] += sv;
            } else {
              int li = 0, m3 = 1;
#pragma unroll
              for (int i = 0; i < DIM; ++i) {
                li += t[i] * m3;
                m3 *= 3;
              }
              rhs[j] -= sv * p[li];
            }
          }
        }
        if (!small_solve<8>(M, rhs, nunk)) atomicExch(status, 1);
        for (int j = 0; j < nunk; ++j) {
          int li = 0, m3 = 1;
#pragma unroll
          for (int i = 0; i < DIM; ++i) {
            li += rpos[j][i] * m3;
            m3 *= 3;
          }
          p[li] = rhs[j];
        }
      }
    }
    // write the entries this patch owns
    for (int k = 0; k < N3; ++k) {
      int r[DIM], kk = k;
      bool own = true;
      int k5 = 0, m5 = 1;
      double w = 1.0;
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        r[i] = kk % 3;
        kk /= 3;
        if (r[i] == 0 && sigma[i] != 1) own = false;
        const int o = sigma[i] * r[i];
        k5 += (o + 2) * m5;
        m5 *= 5;
        w *= wlin1(o);
      }
      if (own) phat_c[plane_index(Lc, cs, k5, N5)] = p[k] - w;
    }
  }
}

// Galerkin coarse operator A_c = P^T A_f P per coarse vertex V (Sect. 4.3):
// A_c(V, W) = sum_{v in supp P(V)} P(V,v) sum_{w in stencil(v)} A_f(v,w) P(W,w),
// with the fine stencils rebuilt in situ.  Stores A_hat = A_c - A_redisc(eps_c),
// zero on entries pointing to non-DoF vertices (they keep the rediscretised value).
template <int DIM, int PMODE>
__global__ void __launch_bounds__(128) k_rap(LevelDesc Lc, LevelDesc Lf, const double* eps_f, const double* ahat_f,
                                               const double* eps_c, const double* phat_c, double* ahat_c) {
  constexpr int N3 = cpow(3, DIM), N5 = cpow(5, DIM);
  const int64_t cs = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (cs >= Lc.n_slots) return;
  int V[DIM];
  const bool valid = coords_of<DIM>(Lc, cs, V);
  if (!valid || !is_dof(Lc.vflags[cs])) {
    if (valid)
      for (int k = 0; k < N3; ++k) ahat_c[plane_index(Lc, cs, k, N3)] = 0.0;
    return;
  }
  double acc[N3];
  for (int k = 0; k < N3; ++k) acc[k] = 0.0;
  for (int k5 = 0; k5 < N5; ++k5) {
    int o[DIM], v[DIM], kk = k5;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      o[i] = kk % 5 - 2;
      kk /= 5;
      v[i] = 3 * V[i] + o[i];
    }
    const int64_t fs = slot_of<DIM>(Lf, v);
    if (fs < 0 || !is_dof(Lf.vflags[fs])) continue;
    const double pV = p_entry_d<DIM, PMODE>(Lc, phat_c, cs, o);
    double st[N3];
    full_stencil<DIM>(Lf, eps_f, ahat_f, v, fs, st);
    for (int t = 0; t < N3; ++t) {
      int w[DIM], tt = t;
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        w[i] = v[i] + tt % 3 - 1;
        tt /= 3;
      }
      const double a = pV * st[t];
      int lo[DIM], cnt[DIM];
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        lo[i] = w[i] >= 0 ? w[i] / 3 : -1;
        cnt[i] = (w[i] >= 0 && w[i] % 3 == 0) ? 1 : 2;
      }
      for (int e = 0; e < (1 << DIM); ++e) {
        int W[DIM], ow[DIM];
        bool ok = true;
        int q = 0, m = 1;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          const int ei = (e >> i) & 1;
          if (ei >= cnt[i]) ok = false;
          W[i] = lo[i] + ei;
          ow[i] = w[i] - 3 * W[i];
          const int dq = W[i] - V[i];
          if (dq < -1 || dq > 1) ok = false;
          q += (dq + 1) * m;
          m *= 3;
        }
        if (!ok) continue;
        const int64_t ws = slot_of<DIM>(Lc, W);
        if (ws < 0 || !is_dof(Lc.vflags[ws])) continue;
        acc[q] = fma(a, p_entry_d<DIM, PMODE>(Lc, phat_c, ws, ow), acc[q]);
      }
    }
  }
  double sr[N3];
  full_stencil<DIM>(Lc, eps_c, nullptr, V, cs, sr);
  for (int q = 0; q < N3; ++q) {
    int W[DIM], qq = q;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      W[i] = V[i] + qq % 3 - 1;
      qq /= 3;
    }
    const int64_t ws = slot_of<DIM>(Lc, W);
    const bool dofw = ws >= 0 && is_dof(Lc.vflags[ws]);
    ahat_c[plane_index(Lc, cs, q, N3)] = dofw ? acc[q] - sr[q] : 0.0;
  }
}

}  // namespace mg
