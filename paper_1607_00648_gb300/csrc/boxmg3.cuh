// BoxMG prolongation in 3D (Sect. 4.4, App. C) by coarse cell.  The system C(s) p = f of
// a coarse vertex V and one of its 2^3 patches uses the fine stencils of the patch's
// fine points, collapsed over the axes along which its unknowns do not vary: stencils of
// the points on the coarse edges through V collapsed over the two other axes (3 values),
// of the points on the coarse faces through V over the face normal (9 values), and the
// full stencils of the 2^3 points inside the patch (27 values).  A patch is a coarse cell
// and each of its eight corners V solves one such system in it, so one group of eight
// threads per coarse cell builds the cell's 56 stencils once (24 edge, 24 face and 8
// interior points of its closure) in shared memory; then thread e (corner V = C + e)
// solves V's system for this patch with all of its arrays in registers: the blocks in
// order of the number of non-zero reference coordinates (lines, faces, interior), each by
// Gaussian elimination with partial pivoting.  The per-vertex form (k_boxmg) built 26
// stencils in every one of the 8 patch threads of a vertex and indexed its arrays at run
// time (local memory).  Ownership of the written entries as in k_boxmg: an entry on a
// line / face through V is written by the patch with sigma_i = +1 on its zero axes.
#pragma once

#include "device.cuh"

namespace mg {

constexpr int kBoxCells = 8;  // coarse cells per CTA (8 threads each)
// shared doubles per cell: 8 interior points x 27, 24 face points x 9, 24 edge points x 3
constexpr int kBoxIntOff = 0, kBoxFaceOff = 8 * 27, kBoxLineOff = kBoxFaceOff + 24 * 9;
constexpr int kBoxPerCell = kBoxLineOff + 24 * 3;

__host__ __device__ constexpr int bx_popc(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1); }
// reference coordinate along axis i of unknown j of block `mask` (mask axes ascending take
// the bits of j: value 1 + bit), 0 off the mask
__host__ __device__ constexpr int bx_rpos(int mask, int j, int i) {
  int bit = 0;
  for (int a = 0; a < i; ++a) bit += (mask >> a) & 1;
  return ((mask >> i) & 1) ? 1 + ((j >> bit) & 1) : 0;
}
// the two axes other than n, ascending
__host__ __device__ constexpr int bx_other(int n, int which) { return which == 0 ? (n == 0 ? 1 : 0) : (n == 2 ? 1 : 2); }

// Gaussian elimination with partial pivoting (the largest |entry| of the column is moved
// to the pivot row by compare-and-swap, so every index is a compile-time one; every loop
// runs over the full range with a guard, which keeps the arrays in registers); false on a
// zero pivot
template <int N>
__device__ __forceinline__ bool bx_solve(double (&M)[N][N], double (&r)[N]) {
  bool ok = true;
#pragma unroll
  for (int c = 0; c < N; ++c) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (k <= c) continue;
      const bool sw = fabs(M[k][c]) > fabs(M[c][c]);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        if (j < c) continue;
        const double a = M[c][j], b = M[k][j];
        M[c][j] = sw ? b : a;
        M[k][j] = sw ? a : b;
      }
      const double a = r[c], b = r[k];
      r[c] = sw ? b : a;
      r[k] = sw ? a : b;
    }
    ok &= M[c][c] != 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (k <= c) continue;
      const double f = M[k][c] / M[c][c];
#pragma unroll
      for (int j = 0; j < N; ++j)
        if (j > c) M[k][j] -= f * M[c][j];
      r[k] -= f * r[c];
    }
  }
#pragma unroll
  for (int cc = 0; cc < N; ++cc) {
    const int c = N - 1 - cc;
    double s = r[c];
#pragma unroll
    for (int j = 0; j < N; ++j)
      if (j > c) s -= M[c][j] * r[j];
    r[c] = s / M[c][c];
  }
  return ok;
}

// one block of corner e's system (mask: the axes along which its unknowns vary): rows
// from the collapsed stencils in `cell`, read through the mirror sigma (reference offset o
// is actual offset sigma o); entries towards reference coordinate 3 vanish, entries
// towards points of earlier blocks move to the right-hand side with their solved p
template <int MASK>
__device__ __forceinline__ void bx_assemble(const double* cell, const int (&e)[3], const int (&sg)[3],
                                            const double (&p)[27], double (&M)[1 << bx_popc(MASK)][1 << bx_popc(MASK)],
                                            double (&rhs)[1 << bx_popc(MASK)]) {
  constexpr int NU = 1 << bx_popc(MASK);
#pragma unroll
  for (int j = 0; j < NU; ++j) {
#pragma unroll
    for (int q = 0; q < NU; ++q) M[j][q] = 0.0;
    rhs[j] = 0.0;
  }
#pragma unroll
  for (int j = 0; j < NU; ++j) {
    const int r0 = bx_rpos(MASK, j, 0), r1 = bx_rpos(MASK, j, 1), r2 = bx_rpos(MASK, j, 2);
    // local fine coordinates of the unknown's point in the cell (0..3 per axis)
    const int l0 = e[0] ? 3 - r0 : r0, l1 = e[1] ? 3 - r1 : r1, l2 = e[2] ? 3 - r2 : r2;
    const double* rec;
    if constexpr (bx_popc(MASK) == 3) {
      rec = cell + kBoxIntOff + 27 * ((l0 - 1) + 2 * (l1 - 1) + 4 * (l2 - 1));
    } else if constexpr (bx_popc(MASK) == 2) {
      constexpr int n = (MASK & 1) == 0 ? 0 : ((MASK & 2) == 0 ? 1 : 2);
      constexpr int a = bx_other(n, 0), b = bx_other(n, 1);
      const int l[3] = {l0, l1, l2};
      rec = cell + kBoxFaceOff + 9 * (4 * (2 * n + e[n]) + (l[a] - 1) + 2 * (l[b] - 1));
    } else {
      constexpr int ax = (MASK & 1) ? 0 : ((MASK & 2) ? 1 : 2);
      constexpr int b = bx_other(ax, 0), c = bx_other(ax, 1);
      const int l[3] = {l0, l1, l2};
      rec = cell + kBoxLineOff + 3 * (2 * (4 * ax + 2 * e[b] + e[c]) + (l[ax] - 1));
    }
#pragma unroll
    for (int oi = 0; oi < 27; ++oi) {
      const int o0 = oi % 3 - 1, o1 = (oi / 3) % 3 - 1, o2 = oi / 9 - 1;
      if ((!(MASK & 1) && o0 != 0) || (!(MASK & 2) && o1 != 0) || (!(MASK & 4) && o2 != 0)) continue;
      const int t0 = (MASK & 1) ? r0 + o0 : 0, t1 = (MASK & 2) ? r1 + o1 : 0, t2 = (MASK & 4) ? r2 + o2 : 0;
      if (t0 == 3 || t1 == 3 || t2 == 3) continue;
      const int a0 = 1 + sg[0] * o0, a1 = 1 + sg[1] * o1, a2 = 1 + sg[2] * o2;  // actual offset + 1
      int idx;
      if constexpr (bx_popc(MASK) == 3) {
        idx = a0 + 3 * a1 + 9 * a2;
      } else if constexpr (bx_popc(MASK) == 2) {
        idx = (MASK & 1) == 0 ? a1 + 3 * a2 : ((MASK & 2) == 0 ? a0 + 3 * a2 : a0 + 3 * a1);
      } else {
        idx = (MASK & 1) ? a0 : ((MASK & 2) ? a1 : a2);
      }
      const double v = rec[idx];
      const bool inblock = (!(MASK & 1) || t0 >= 1) && (!(MASK & 2) || t1 >= 1) && (!(MASK & 4) || t2 >= 1);
      if (inblock) {
        int q = 0, bit = 0;
        if (MASK & 1) q |= (t0 - 1) << bit++;
        if (MASK & 2) q |= (t1 - 1) << bit++;
        if (MASK & 4) q |= (t2 - 1) << bit++;
        M[j][q] += v;
      } else {
        rhs[j] -= v * p[t0 + 3 * t1 + 9 * t2];
      }
    }
  }
}

template <int MASK>
__device__ __forceinline__ bool bx_block(const double* cell, const int (&e)[3], const int (&sg)[3],
                                         double (&p)[27]) {
  constexpr int NU = 1 << bx_popc(MASK);
  double M[NU][NU], rhs[NU];
  bx_assemble<MASK>(cell, e, sg, p, M, rhs);
  const bool ok = bx_solve<NU>(M, rhs);
#pragma unroll
  for (int j = 0; j < NU; ++j) p[bx_rpos(MASK, j, 0) + 3 * bx_rpos(MASK, j, 1) + 9 * bx_rpos(MASK, j, 2)] = rhs[j];
  return ok;
}

// P_hat entries k (reference position r, lexicographic) of V in this patch that the patch
// owns: entries on a line / face through V belong to the patch with sigma = +1 on the zero
// axes.  interior: the entries with no zero coordinate, else the others.
__device__ __forceinline__ void bx_write(const LevelDesc& Lc, int64_t vs, const int (&e)[3], const int (&sg)[3],
                                         const double (&p)[27], bool interior, double* phat_c) {
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    const int r0 = k % 3, r1 = (k / 3) % 3, r2 = k / 9;
    if ((r0 != 0 && r1 != 0 && r2 != 0) != interior) continue;
    const bool own = (r0 != 0 || e[0] == 0) && (r1 != 0 || e[1] == 0) && (r2 != 0 || e[2] == 0);
    if (!own) continue;
    const int k5 = (sg[0] * r0 + 2) + 5 * (sg[1] * r1 + 2) + 25 * (sg[2] * r2 + 2);
    const double w = wlin1(r0) * wlin1(r1) * wlin1(r2);  // d-linear weight (symmetric in sigma)
    phat_c[plane_index(Lc, vs, k5, 125)] = p[k] - w;
  }
}

// stencil of point pidx of a cell's closure (0..7 interior, 8..31 face, 32..55 edge
// points), collapsed as its blocks need it, into the cell's shared record
__device__ __forceinline__ void bx_build(const LevelDesc& Lf, const double* eps_f, const double* ahat_f,
                                         const double* aniso_f, const int (&C3)[3], int pidx, double* cell) {
  int l[3], cat, ax = 0;
  double* out;
  if (pidx < 8) {
    l[0] = 1 + (pidx & 1);
    l[1] = 1 + ((pidx >> 1) & 1);
    l[2] = 1 + (pidx >> 2);
    cat = 0;
    out = cell + kBoxIntOff + 27 * pidx;
  } else if (pidx < 32) {
    const int fi = pidx - 8, f = fi >> 2, q = fi & 3, n = f >> 1;
    l[n] = 3 * (f & 1);
    l[bx_other(n, 0)] = 1 + (q & 1);
    l[bx_other(n, 1)] = 1 + (q >> 1);
    cat = 1;
    ax = n;
    out = cell + kBoxFaceOff + 9 * fi;
  } else {
    const int li = pidx - 32, edge = li >> 1, a = edge >> 2;
    l[a] = 1 + (li & 1);
    l[bx_other(a, 0)] = 3 * ((edge >> 1) & 1);
    l[bx_other(a, 1)] = 3 * (edge & 1);
    cat = 2;
    ax = a;
    out = cell + kBoxLineOff + 3 * li;
  }
  const int x[3] = {C3[0] + l[0], C3[1] + l[1], C3[2] + l[2]};
  const int64_t fs = slot_of<3>(Lf, x);
  double st[27];
  full_stencil<3>(Lf, eps_f, ahat_f, x, fs, st, aniso_f);
  if (cat == 0) {
#pragma unroll
    for (int k = 0; k < 27; ++k) out[k] = st[k];
  } else if (cat == 1) {  // over the normal axis; in-plane axes a < b: index ia + 3 ib
#pragma unroll
    for (int ib = 0; ib < 3; ++ib)
#pragma unroll
      for (int ia = 0; ia < 3; ++ia) {
        double s;
        if (ax == 0) s = (st[0 + 3 * ia + 9 * ib] + st[1 + 3 * ia + 9 * ib]) + st[2 + 3 * ia + 9 * ib];
        else if (ax == 1) s = (st[ia + 0 + 9 * ib] + st[ia + 3 + 9 * ib]) + st[ia + 6 + 9 * ib];
        else s = (st[ia + 3 * ib + 0] + st[ia + 3 * ib + 9]) + st[ia + 3 * ib + 18];
        out[ia + 3 * ib] = s;
      }
  } else {  // over the two axes other than ax
#pragma unroll
    for (int ia = 0; ia < 3; ++ia) {
      double s = 0.0;
#pragma unroll
      for (int v = 0; v < 9; ++v) {
        const int i = v % 3, j = v / 3;
        s += ax == 0 ? st[ia + 3 * i + 9 * j] : (ax == 1 ? st[i + 3 * ia + 9 * j] : st[i + 3 * j + 9 * ia]);
      }
      out[ia] = s;
    }
  }
}

// one CTA of 8 x kBoxCells threads: eight threads per coarse cell (the cell of coarse slot
// cs is the one with lower corner at cs's vertex); output P_hat = P - P_dlin on 125 planes
__global__ void __launch_bounds__(8 * kBoxCells) k_boxmg3c(LevelDesc Lc, LevelDesc Lf, const double* eps_f,
                                                          const double* ahat_f, double* phat_c, int* status,
                                                          const double* aniso_f) {
  constexpr int N5 = 125;
  __shared__ double sbuf[kBoxCells * kBoxPerCell];
  const int g = threadIdx.x >> 3, eid = threadIdx.x & 7;
  const int64_t cs = blockIdx.x * static_cast<int64_t>(kBoxCells) + g;
  double* cell = sbuf + g * kBoxPerCell;
  int Cc[3] = {0, 0, 0};
  const bool valid = cs < Lc.n_slots && coords_of<3>(Lc, cs, Cc);
  // every slot's vertex is the lower corner of a cell (vertex n, the upper boundary, has
  // no slot; corners there are skipped as non-DoFs)
  const bool is_cell = valid;
  // a vertex that is no DoF carries zero planes (from the thread of its own slot)
  if (valid && eid == 0 && !is_dof(Lc.vflags[cs]))
    for (int k = 0; k < N5; ++k) phat_c[plane_index(Lc, cs, k, N5)] = 0.0;
  if (is_cell) {
    const int C3[3] = {3 * Cc[0], 3 * Cc[1], 3 * Cc[2]};
    for (int pidx = eid; pidx < 56; pidx += 8) bx_build(Lf, eps_f, ahat_f, aniso_f, C3, pidx, cell);
  }
  __syncthreads();
  if (!is_cell) return;
  const int e[3] = {eid & 1, (eid >> 1) & 1, eid >> 2};
  const int V[3] = {Cc[0] + e[0], Cc[1] + e[1], Cc[2] + e[2]};
  const int64_t vs = slot_of<3>(Lc, V);
  if (vs < 0 || !is_dof(Lc.vflags[vs])) return;
  const int sg[3] = {1 - 2 * e[0], 1 - 2 * e[1], 1 - 2 * e[2]};  // from V into the cell
  double p[27];
#pragma unroll
  for (int k = 0; k < 27; ++k) p[k] = 0.0;
  p[0] = 1.0;  // the c-point
  bool ok = bx_block<1>(cell, e, sg, p);
  ok = bx_block<2>(cell, e, sg, p) && ok;
  ok = bx_block<4>(cell, e, sg, p) && ok;
  ok = bx_block<3>(cell, e, sg, p) && ok;
  ok = bx_block<5>(cell, e, sg, p) && ok;
  ok = bx_block<6>(cell, e, sg, p) && ok;
  {
    // the interior block: once its rows are assembled the other entries are written, so
    // that only its 8 x 8 system stays live through the elimination
    double M[8][8], rhs[8];
    bx_assemble<7>(cell, e, sg, p, M, rhs);
    bx_write(Lc, vs, e, sg, p, false, phat_c);
    ok = bx_solve<8>(M, rhs) && ok;
#pragma unroll
    for (int j = 0; j < 8; ++j) p[bx_rpos(7, j, 0) + 3 * bx_rpos(7, j, 1) + 9 * bx_rpos(7, j, 2)] = rhs[j];
  }
  if (!ok) atomicExch(status, 1);
  bx_write(Lc, vs, e, sg, p, true, phat_c);
}

}  // namespace mg
