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
                                                const double* ahat_f, double* phat_c, int* status,
                                                const double* aniso_f = nullptr) {
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
          full_stencil<DIM>(Lf, eps_f, ahat_f, xf, fsl, st, aniso_f);
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

// omega / diag(A) per DoF (rediscretised diagonal + stored delta), zero elsewhere:
// the damped-Jacobi factor of Alg. 1, formed once per setup
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_jacobi_dinv(LevelDesc L, const double* eps, const double* ahat,
                                                          double omega, double* dinv) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (s >= L.n_slots) return;
  int x[DIM];
  if (!coords_of<DIM>(L, s, x) || !is_dof(L.vflags[s])) {
    dinv[s] = 0.0;
    return;
  }
  double es = 0.0;
  for (int e = 0; e < (1 << DIM); ++e) {
    int c[DIM];
    for (int i = 0; i < DIM; ++i) c[i] = x[i] - ((e >> i) & 1);
    const int64_t cs = slot_of<DIM>(L, c);
    if (cs >= 0) es += eps[cs];
  }
  double D = elem_k(DIM, 0) * es * (DIM == 3 ? L.h : 1.0);
  if (ahat) D += ahat[plane_index(L, s, cpow(3, DIM) / 2, cpow(3, DIM))];
  dinv[s] = omega / D;
}

// Galerkin coarse operator A_c = P^T A_f P (Sect. 4.3), one group of kRapTpv
// threads per coarse vertex V: thread j takes the fine vertex f = 3V + d(j) of the
// support of P(V, .) (5^d of them), rebuilds f's fine stencil in situ and forms its
// contributions P(f,V) A_f(f,g) P(g,W) to the 3^d coarse entries W = V + o; the
// group then adds them in a fixed order (warp shuffles, then warps in order).
// Stores A_hat = A_c - A_redisc(eps_c), zero on entries to non-DoF vertices (they
// keep the rediscretised value), zero planes on non-DoF coarse vertices.
template <int DIM>
constexpr int rap_tpv() { return DIM == 2 ? 32 : 128; }

// dynamic shared memory of k_rap<DIM, PMODE>: the staged P of the coarse neighbours and
// every thread's scaled fine stencil
template <int DIM, int PMODE>
constexpr size_t rap_dyn_smem() {
  return (static_cast<size_t>(128 / rap_tpv<DIM>()) * cpow(3, DIM) * cpow(5, DIM) + 128 * cpow(3, DIM)) *
         sizeof(double);
}

template <int DIM, int PMODE>
__global__ void __launch_bounds__(128) k_rap(LevelDesc Lc, LevelDesc Lf, const double* eps_f, const double* ahat_f,
                                               const double* eps_c, const double* phat_c, double* ahat_c,
                                               const double* aniso_f = nullptr) {
  constexpr int N3 = cpow(3, DIM), N5 = cpow(5, DIM);
  constexpr int TPV = rap_tpv<DIM>(), VPB = 128 / TPV, WPV = TPV / 32;
  __shared__ int64_t pbase[VPB][N3];   // plane-0 index of P_hat(W) for W = V + o if W is a DoF, else -1
  __shared__ double sred[VPB][N3];     // A_redisc(V, V + o)
  __shared__ double part[VPB][N3][WPV];
  __shared__ double plin[N5];          // d-linear weights by 5^d offset
  extern __shared__ double pfull[];    // P(W, .) = d-linear + P_hat of the 3^d coarse neighbours: [VPB][N3][N5]
  const int sub = threadIdx.x / TPV, j = threadIdx.x % TPV;
  const int64_t cs = blockIdx.x * static_cast<int64_t>(VPB) + sub;
  int V[DIM];
  const bool valid = cs < Lc.n_slots && coords_of<DIM>(Lc, cs, V);
  const bool vdof = valid && is_dof(Lc.vflags[cs]);
  for (int k = threadIdx.x; k < N5; k += blockDim.x) {
    double w = 1.0;
    int kk = k;
    for (int i = 0; i < DIM; ++i) {
      w *= wlin1(kk % 5 - 2);
      kk /= 5;
    }
    plin[k] = w;
  }
  if (j < N3) {  // every entry is written (-1 unless W is a DoF): the staging below reads them all
    int64_t pb = -1;
    if (vdof) {
      int W[DIM], jj = j;
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        W[i] = V[i] + jj % 3 - 1;
        jj /= 3;
      }
      const int64_t ws = slot_of<DIM>(Lc, W);
      if (ws >= 0 && is_dof(Lc.vflags[ws])) pb = plane_index(Lc, ws, 0, N5);
    }
    pbase[sub][j] = pb;
  }
  if (vdof && j == 0) {
    double sr[N3];
    full_stencil<DIM>(Lc, eps_c, nullptr, V, cs, sr);
#pragma unroll
    for (int q = 0; q < N3; ++q) sred[sub][q] = sr[q];
  }
  // this thread's fine vertex f = 3V + d, P(f,V) times its fine stencil, and which of
  // its stencil neighbours are DoFs
  int d[DIM];
  uint32_t gdof = 0;
  double st[N3];
  {
    int f[DIM], jj = j;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      d[i] = jj % 5 - 2;
      jj /= 5;
      f[i] = 3 * V[i] + d[i];
    }
    const int64_t fs = (vdof && j < N5) ? slot_of<DIM>(Lf, f) : -1;
    if (fs >= 0 && is_dof(Lf.vflags[fs])) {
      const double pV = p_entry_d<DIM, PMODE>(Lc, phat_c, cs, d);
      full_stencil<DIM>(Lf, eps_f, ahat_f, f, fs, st, aniso_f);
#pragma unroll
      for (int e = 0; e < N3; ++e) {
        int g[DIM], ee = e;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          g[i] = f[i] + ee % 3 - 1;
          ee /= 3;
        }
        const int64_t gs = slot_of<DIM>(Lf, g);
        if (gs >= 0 && is_dof(Lf.vflags[gs])) gdof |= 1u << e;
        st[e] *= pV;
      }
    }
  }
  __syncthreads();
  // stage P(W, .) of the neighbours once per CTA: the loads all in flight together, and
  // the d-linear part added here rather than once per term below (FP64 units are scarce)
  for (int idx = threadIdx.x; idx < VPB * N3 * N5; idx += blockDim.x) {
    const int64_t pb = pbase[idx / (N3 * N5)][(idx / N5) % N3];
    double p = 0.0;
    if (pb >= 0) {
      p = plin[idx % N5];
      if constexpr (PMODE == 1) p += phat_c[pb + (idx % N5) * static_cast<int64_t>(Lc.S)];
    }
    pfull[idx] = p;
  }
  __syncthreads();

  // c[q] = sum over stencil neighbours g = f + eps of f with |g - 3W| <= 2 (W = V + o_q)
  // of P(f,V) A_f(f,g) P(g,W).  The scaled stencil goes to shared memory (zero where g is
  // no DoF) and each target W loops over the admissible eps only: per axis
  // eps in [max(-1, 3 o - 2 - d), min(1, 3 o + 2 - d)] (about 4 of the 3^d per target in
  // 3D), so no fma is issued for a pair that contributes nothing
  double* sst = pfull + VPB * N3 * N5 + threadIdx.x * N3;
#pragma unroll
  for (int e = 0; e < N3; ++e) sst[e] = ((gdof >> e) & 1u) ? st[e] : 0.0;
  double c[N3];
#pragma unroll
  for (int q = 0; q < N3; ++q) c[q] = 0.0;
  if (gdof) {
    const double* pf = pfull + sub * N3 * N5;
#pragma unroll
    for (int q = 0; q < N3; ++q) {
      int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, pb[3] = {0, 0, 0};
      int qq = q;
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        const int o = qq % 3 - 1;
        qq /= 3;
        lo[i] = max(-1, 3 * o - 2 - d[i]);
        hi[i] = min(1, 3 * o + 2 - d[i]);
        pb[i] = d[i] - 3 * o + 2;  // offset index of g - 3W at eps = 0, per axis
      }
      const double* pw = pf + q * N5;
      double acc = 0.0;
      for (int ez = lo[2]; ez <= hi[2]; ++ez)
        for (int ey = lo[1]; ey <= hi[1]; ++ey)
          for (int ex = lo[0]; ex <= hi[0]; ++ex) {
            const int e = (ex + 1) + 3 * (ey + 1) + (DIM == 3 ? 9 * (ez + 1) : 0);
            const int k = (pb[0] + ex) + 5 * (pb[1] + ey) + (DIM == 3 ? 25 * (pb[2] + ez) : 0);
            acc = fma(sst[e], pw[k], acc);
          }
      c[q] = acc;
    }
  }
  // fixed-order reduction over the group: shuffles within each warp, then warps in order
  const int lane = threadIdx.x & 31, wig = j / 32;
#pragma unroll
  for (int q = 0; q < N3; ++q) {
    double v = c[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) part[sub][q][wig] = v;
  }
  __syncthreads();
  if (valid && j < N3) {
    double out = 0.0;
    if (vdof && pbase[sub][j] >= 0) {
      double acc = part[sub][j][0];
#pragma unroll
      for (int w = 1; w < WPV; ++w) acc += part[sub][j][w];
      out = acc - sred[sub][j];
    }
    ahat_c[plane_index(Lc, cs, j, N3)] = out;
  }
}

}  // namespace mg
