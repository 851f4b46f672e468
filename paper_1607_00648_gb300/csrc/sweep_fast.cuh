// Sweep kernels for the brick edges that carry the fine levels (2D: 27, 3D: 9),
// with every index fixed per thread and advanced incrementally along the last
// axis.  Same operations and results as sweep_item (in-situ stencil from the
// adjacent cells' coefficients, + stored delta on coarse levels, Jacobi / residual),
// with a fraction of its integer work: the generic kernel spends most of its issue
// slots on per-element index arithmetic, which bounds the FP32 sweeps.
#pragma once

#include "kernels.cuh"

namespace mg {

// 4-byte asynchronous global -> shared copy (cp.async); src_ok false writes zero
// (src-size 0) and reads nothing, so `g` only has to be a valid address
__device__ __forceinline__ void cp_async4(void* s, const void* g, bool src_ok) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(s));
  const int n = src_ok ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(g), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async8(void* s, const void* g, bool src_ok) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(s));
  const int n = src_ok ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(g), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// one element of type T (4 or 8 bytes)
template <typename T>
__device__ __forceinline__ void cp_async_el(T* s, const T* g, bool src_ok) {
  if constexpr (sizeof(T) == 8) cp_async8(s, g, src_ok);
  else cp_async4(s, g, src_ok);
}

// The 9-point bilinear stencil at one vertex from its 3x3 values and 4 cells
// (cells sw, se, nw, ne; values row-major m = y-1, 0 = y, p = y+1; l/r = x -+ 1).
template <typename T>
__device__ __forceinline__ void stencil2(T sw, T se, T nw, T ne, T um_l, T um, T um_r, T u0_l, T u0, T u0_r, T up_l,
                                         T up, T up_r, T& Au, T& D) {
  const T sW = sw + nw, sE = se + ne, sS = sw + se, sN = nw + ne;
  const T sC = sW + sE;
  T a1 = sW * u0_l;
  a1 = fma(sE, u0_r, a1);
  a1 = fma(sS, um, a1);
  a1 = fma(sN, up, a1);
  T a2 = sw * um_l;
  a2 = fma(se, um_r, a2);
  a2 = fma(nw, up_l, a2);
  a2 = fma(ne, up_r, a2);
  const T k0 = static_cast<T>(elem_k(2, 0)), k1 = static_cast<T>(elem_k(2, 1)), k2 = static_cast<T>(elem_k(2, 2));
  D = k0 * sC;
  Au = fma(D, u0, fma(k1, a1, k2 * a2));
}

// 2D, brick edge 27 (FP32): one CTA of 128 threads per (brick, slab of R rows).
// Lane l of warp g holds tile column x = l - 1 (x in [-1, 27]) and rows g, g + 4, ...
// of the slab with its halo.  The tile is filled by asynchronous copies (cp.async:
// no registers held, every load in flight at once), b and the flags of a thread's
// vertices are fetched into registers meanwhile; after one barrier each thread
// applies the stencil to its vertices from shared memory.
template <typename T, int AMODE, int OP, int R>
__device__ __forceinline__ double sweep2c_item(const SweepArgs<T>& a, int64_t brick, int slab) {
  constexpr int B = 27, Bu = B + 2, Be = B + 1, NR = (R + 3) / 4;
  __shared__ __align__(16) T su[(R + 2) * Bu];
  __shared__ __align__(16) T se[(R + 1) * Be];
  const LevelDesc& L = a.L;
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int64_t base = brick * L.S;
  const int z0 = slab * R;
  __syncthreads();  // the tile may still be read by a previous item of this CTA
  const int32_t* bn = L.brick_nbr + brick * 9;
  const int x = lane - 1;
  // this thread's vertices: rows zl = g + 4 k of the slab, column x in [0, 27)
  const bool vcol = x >= 0 && x < B;
  T bv[NR];
  uint8_t fv[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    const int zl = g + 4 * k;
    const bool on = vcol && zl < R;
    const int64_t slot = base + (z0 + zl) * B + x;
    fv[k] = on ? L.vflags[slot] : 0;
    bv[k] = (on && is_dof(fv[k])) ? a.b[slot] : T(0);
  }
  if (x <= B) {
    const int ox = x < 0 ? -1 : (x >= B ? 1 : 0);
    const int lx = x - ox * B;
    const int32_t nb_lo = bn[ox + 1], nb_mid = bn[ox + 4], nb_hi = bn[ox + 7];
    for (int zz = g; zz < R + 2; zz += 4) {
      const int y = z0 - 1 + zz;
      const int oy = y < 0 ? -1 : (y >= B ? 1 : 0);
      const int32_t nb = oy < 0 ? nb_lo : (oy > 0 ? nb_hi : nb_mid);
      const int64_t idx = nb >= 0 ? static_cast<int64_t>(nb) * L.S + (y - oy * B) * B + lx : 0;
      cp_async4(su + zz * Bu + lane, a.u + idx, nb >= 0);
      if (x < B && zz <= R) cp_async4(se + zz * Be + lane, a.eps + idx, nb >= 0);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  double part = 0.0;
  if (vcol) {
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int zl = g + 4 * k;
      if (zl >= R) break;
      const int64_t slot = base + (z0 + zl) * B + x;
      const uint8_t vf = fv[k];
      const T* uc = su + (zl + 1) * Bu + lane;  // tile column of x is lane
      const T* ec = se + (zl + 1) * Be + lane;  // cell with lower corner (x, y)
      T res = T(0);
      // iota vertices keep their value in the Jacobi part of a block step (Sect. 4.2)
      const bool keep = OP == kJacobi && a.block && x % 3 != 0 && (z0 + zl) % 3 != 0;
      if constexpr (OP == kJacobi || OP == kJacobiNorm) {
        if ((vf & MG_V_HANGING) || keep) res = uc[0];  // hanging values come from the coarser level (Sect. 3)
      }
      if (is_dof(vf) && !keep) {
        const T um_l = uc[-Bu - 1], um = uc[-Bu], um_r = uc[-Bu + 1];
        const T u0_l = uc[-1], u0 = uc[0], u0_r = uc[1];
        const T up_l = uc[Bu - 1], up = uc[Bu], up_r = uc[Bu + 1];
        T Au, D;
        stencil2<T>(ec[-Be - 1], ec[-Be], ec[-1], ec[0], um_l, um, um_r, u0_l, u0, u0_r, up_l, up, up_r, Au, D);
        const uint64_t akey = AMODE != 0 ? delta_row<AMODE>(a.ascale, slot) : 0;
        if (AMODE != 0 && delta_row_live<AMODE>(akey)) {
          const T nbv[9] = {um_l, um, um_r, u0_l, u0, u0_r, up_l, up, up_r};
          const int sl = (z0 + zl) * B + x;
#pragma unroll
          for (int q = 0; q < 9; ++q) {
            const T d = load_delta<AMODE, T>(a.ahat, a.ascale, (brick * 9 + q) * L.S + sl, slot, q, akey,
                                             a_lo_off<AMODE>(L, 9));
            Au = fma(d, nbv[q], Au);
            if (q == 4) D += d;
          }
        }
        const T r = bv[k] - Au;
        if constexpr (OP == kJacobi || OP == kJacobiNorm) {
          res = fma(a.omega * r, recip_nr(D), u0);
          if constexpr (OP == kJacobiNorm) part += static_cast<double>(r) * static_cast<double>(r);
        } else {
          res = r;
          part += static_cast<double>(r) * static_cast<double>(r);
        }
      }
      a.out[slot] = res;
    }
  }
  return part;
}

template <typename T, int AMODE, int OP, int R>
__global__ void __launch_bounds__(128) k_sweep2c(SweepArgs<T> a) {
  pdl_enter();
  const double part = sweep2c_item<T, AMODE, OP, R>(a, blockIdx.x, blockIdx.y);
  if constexpr (OP == kResidual) {
    if (a.partial) store_partial_and_finish(part, a.partial, a.counter, a.norm2);
  }
}

// 16-byte asynchronous global -> shared copy; both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16(void* s, const void* g) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(s));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}

// 2D, brick edge 27, FP32: staging by 16-byte copies and column marching.  One CTA of
// NW warps per (brick, slab of R rows).  The slab's rows are one contiguous range of
// the brick (slots are lexicographic), so u and eps are copied into linear tiles
// (row stride 27) by 16-byte cp.async; the tile starts at an offset that puts every
// 16-byte-aligned global element on a 16-byte-aligned shared address, and the few
// elements before the first aligned one are the row below's last ones, i.e. correct
// halo values.  The halo rows y0 - 1, y0 + R and the halo columns x = -1, 27 (and the
// column of cells x = -1) come by 4-byte copies from this brick or its neighbours.
// Lane l < 27 owns column x = l; warp w marches up a band of R / NW rows, carrying the
// values of the rows below and the cells below in registers, so each vertex reads three
// values and two cell coefficients from shared memory.
template <int AMODE, int OP, int R>
__device__ __forceinline__ double sweep2v_item(const SweepArgs<float>& a, int64_t brick, int slab) {
  constexpr int B = 27, NW = R >= 3 ? 3 : 1, RB = R / NW;
  constexpr int LIN = (R + 2) * B + 4;  // rows -1 .. R, + alignment slack
  __shared__ __align__(16) float lu[LIN];
  __shared__ __align__(16) float le[LIN];
  __shared__ float hlu[R + 2], hru[R + 2], hle[R + 1];
  const LevelDesc& L = a.L;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int t = threadIdx.x, nt = NW * 32;
  const int64_t base = brick * L.S;
  const int z0 = slab * R;
  __syncthreads();  // the tiles may still be read by a previous item of this CTA
  const int32_t* bn = L.brick_nbr + brick * 9;
  // tile index of global brick element g: o + B + (g - z0 B), 16-byte aligned where g is
  const int o = (((B * z0 - B) % 4) + 4) % 4;
  const int gs = z0 * B, ge = (z0 + R) * B;
  const int a0 = gs & ~3, a1 = ge & ~3;
  float* tu = lu + o + B - gs;  // tu[g]: value of brick element g (rows z0 - 1 .. z0 + R)
  float* te = le + o + B - gs;
  const float* gu = a.u + base;
  const float* geps = a.eps + base;
  for (int g = a0 + 4 * t; g < a1; g += 4 * nt) {
    cp_async16(tu + g, gu + g);
    cp_async16(te + g, geps + g);
  }
  for (int g = a1 + t; g < ge; g += nt) {
    cp_async4(tu + g, gu + g, true);
    cp_async4(te + g, geps + g, true);
  }
  // halo row below (row z0 - 1; its last gs - a0 elements came with the aligned copy)
  // and above (row z0 + R), vertex values; cells of the row below
  {
    const int nb_lo = z0 > 0 ? static_cast<int>(brick) : bn[1];
    const int ylo = z0 > 0 ? z0 - 1 : B - 1;
    const int nlo = B - (gs - a0);
    const int nb_hi = z0 + R < B ? static_cast<int>(brick) : bn[7];
    const int yhi = z0 + R < B ? z0 + R : 0;
    for (int i = t; i < 2 * B; i += nt) {
      const bool lo = i < B;
      const int x = lo ? i : i - B;
      if (lo && x >= nlo) continue;
      const int32_t nb = lo ? nb_lo : nb_hi;
      const int64_t idx = nb >= 0 ? static_cast<int64_t>(nb) * L.S + (lo ? ylo : yhi) * B + x : 0;
      float* dst = lo ? tu + gs - B + x : tu + ge + x;
      cp_async4(dst, a.u + idx, nb >= 0);
      if (lo) cp_async4(te + gs - B + x, a.eps + idx, nb >= 0);
    }
  }
  // halo columns x = -1 (values and cells) and x = 27 (values), rows z0 - 1 .. z0 + R
  for (int i = t; i < 2 * (R + 2); i += nt) {
    const bool left = i < R + 2;
    const int yl = (left ? i : i - (R + 2)) - 1;
    const int y = z0 + yl;
    const int oy = y < 0 ? -1 : (y >= B ? 1 : 0);
    const int32_t nb = bn[(left ? 0 : 2) + 3 * (oy + 1)];
    const int64_t idx = nb >= 0 ? static_cast<int64_t>(nb) * L.S + (y - oy * B) * B + (left ? B - 1 : 0) : 0;
    cp_async4(left ? hlu + yl + 1 : hru + yl + 1, a.u + idx, nb >= 0);
    if (left && yl < R) cp_async4(hle + yl + 1, a.eps + idx, nb >= 0);
  }
  // b and flags of this thread's vertices, fetched while the tiles stream in
  const int x = lane;
  const bool vl = x < B;
  const int yb = w * RB;
  float bv[RB];
  uint8_t fv[RB];
#pragma unroll
  for (int k = 0; k < RB; ++k) {
    const int64_t slot = base + (z0 + yb + k) * B + x;
    fv[k] = vl ? L.vflags[slot] : 0;
    bv[k] = (vl && is_dof(fv[k])) ? a.b[slot] : 0.0f;
  }
  cp_async_wait_all();
  __syncthreads();
  double part = 0.0;
  if (!vl) return part;
  // per-lane column pointers (row stride B in the linear tiles, 1 in the halo columns)
  const float* pc = tu + gs + (yb - 1) * B + x;  // column x, row yb - 1
  const float* pl = x > 0 ? pc - 1 : hlu + yb;
  const float* pr = x < B - 1 ? pc + 1 : hru + yb;
  const int sl = x > 0 ? B : 1, sr = x < B - 1 ? B : 1;
  const float* ec = te + gs + (yb - 1) * B + x;  // cell column x, row yb - 1
  const float* el = x > 0 ? ec - 1 : hle + yb;
  float um_l = pl[0], um = pc[0], um_r = pr[0];
  float u0_l = pl[sl], u0 = pc[B], u0_r = pr[sr];
  float em_l = el[0], em = ec[0];
  const float k0 = static_cast<float>(elem_k(2, 0)), k1 = static_cast<float>(elem_k(2, 1)),
              k2 = static_cast<float>(elem_k(2, 2));
#pragma unroll
  for (int k = 0; k < RB; ++k) {
    const float up_l = pl[(k + 2) * sl], upc = pc[(k + 2) * B], up_r = pr[(k + 2) * sr];
    const float e0_l = el[(k + 1) * sl], e0 = ec[(k + 1) * B];
    const float sW = em_l + e0_l, sE = em + e0, sS = em_l + em, sN = e0_l + e0;
    float a1 = sW * u0_l;
    a1 = fmaf(sE, u0_r, a1);
    a1 = fmaf(sS, um, a1);
    a1 = fmaf(sN, upc, a1);
    float a2 = em_l * um_l;
    a2 = fmaf(em, um_r, a2);
    a2 = fmaf(e0_l, up_l, a2);
    a2 = fmaf(e0, up_r, a2);
    float D = k0 * (sW + sE);
    float Au = fmaf(D, u0, fmaf(k1, a1, k2 * a2));
    const int yl = yb + k;
    const int64_t slot = base + (z0 + yl) * B + x;
    const uint8_t vf = fv[k];
    float res = 0.0f;
    // iota vertices keep their value in the Jacobi part of a block step (Sect. 4.2);
    // hanging values come from the coarser level (Sect. 3)
    const bool keep = OP == kJacobi && a.block && x % 3 != 0 && (z0 + yl) % 3 != 0;
    if constexpr (OP == kJacobi) {
      if ((vf & MG_V_HANGING) || keep) res = u0;
    }
    if (is_dof(vf) && !keep) {
      const uint64_t akey = AMODE != 0 ? delta_row<AMODE>(a.ascale, slot) : 0;
      if (AMODE != 0 && delta_row_live<AMODE>(akey)) {
        const float nbv[9] = {um_l, um, um_r, u0_l, u0, u0_r, up_l, upc, up_r};
        const int sl2 = (z0 + yl) * B + x;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          const float d = load_delta<AMODE, float>(a.ahat, a.ascale, (brick * 9 + q) * L.S + sl2, slot, q, akey,
                                                   a_lo_off<AMODE>(L, 9));
          Au = fmaf(d, nbv[q], Au);
          if (q == 4) D += d;
        }
      }
      const float r = bv[k] - Au;
      if constexpr (OP == kJacobi) {
        res = fmaf(a.omega * r, recip_nr(D), u0);
      } else {
        res = r;
        part += static_cast<double>(r) * static_cast<double>(r);
      }
    }
    a.out[slot] = res;
    um_l = u0_l; um = u0; um_r = u0_r;
    u0_l = up_l; u0 = upc; u0_r = up_r;
    em_l = e0_l; em = e0;
  }
  return part;
}

template <int AMODE, int OP, int R>
__global__ void __launch_bounds__(96) k_sweep2v(SweepArgs<float> a) {
  pdl_enter();
  const double part = sweep2v_item<AMODE, OP, R>(a, blockIdx.x, blockIdx.y);
  if constexpr (OP == kResidual) {
    if (a.partial) store_partial_and_finish(part, a.partial, a.counter, a.norm2);
  }
}

// 2D, brick edge 27, FP64.  GB300 issues about two FP64 instructions per clock and SM,
// so the FP64 units, not memory, bound these sweeps; this kernel is shaped to issue as
// few FP64 instructions per vertex as the element-wise stencil allows.  One CTA of NW
// warps per (brick, slab of R rows); lane l holds tile column x = l - 1 and warp w
// marches up its band of R / NW rows with the values and cell coefficients of the row
// below carried in registers.  With the Sect. 4 element matrix (edge neighbour
// k1 = -1/6, opposite corner k2 = -1/3 = 2 k1, each times the coefficient of the cell
// the two vertices share):
//   off_v / k1 = sW u_W + sE u_E + sS u_S + sN u_N
//                + 2 (e_sw u_sw + e_se u_se + e_nw u_nw + e_ne u_ne),
// where sE = e_se + e_ne is the column's vertical pair of cells (one add), sW the same
// pair of column x - 1 (a shuffle from the neighbouring lane), sN = e_nw + e_ne (one
// add) and sS the row below's sN (carried).  Jacobi: u' = (1 - omega) u + (omega / D)
// (b - off) with omega / D from the setup; residual: r = b - off - D u, D = 2/3 (sW + sE).
// FP64 instructions per vertex: 14 (Jacobi), 16 (residual and its square); coarse
// levels add one fma per stored delta entry.
template <int AMODE, int OP, int R>
__device__ __forceinline__ double sweep2f_item(const SweepArgs<double>& a, int64_t brick, int slab) {
  constexpr int B = 27, Bu = B + 2, Be = B + 1;
  constexpr int NW = R >= 3 ? 3 : 1, RB = R / NW;
  __shared__ __align__(16) double su[(R + 2) * Bu];
  __shared__ __align__(16) double se[(R + 1) * Be];
  const LevelDesc& L = a.L;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = brick * L.S;
  const int z0 = slab * R;
  __syncthreads();  // the tile may still be read by a previous item of this CTA
  const int32_t* bn = L.brick_nbr + brick * 9;
  const int x = lane - 1;
  const bool vl = x >= 0 && x < B;  // lanes 1..27: vertex columns 0..26
  const bool cl = lane <= B;        // lanes 0..27: cell columns -1..26
  const int yb = w * RB;            // first row of this warp's band (slab-relative)
  double bv[RB], dv[RB];
  uint8_t fv[RB];
#pragma unroll
  for (int k = 0; k < RB; ++k) {
    const int64_t slot = base + (z0 + yb + k) * B + x;
    fv[k] = vl ? L.vflags[slot] : 0;
    const bool on = vl && is_dof(fv[k]);
    bv[k] = on ? a.b[slot] : 0.0;
    dv[k] = (OP != kResidual && on) ? a.dinv[slot] : 0.0;
  }
  if (x <= B) {
    const int ox = x < 0 ? -1 : (x >= B ? 1 : 0);
    const int lx = x - ox * B;
    const int32_t nb_lo = bn[ox + 1], nb_mid = bn[ox + 4], nb_hi = bn[ox + 7];
    for (int zz = w; zz < R + 2; zz += NW) {
      const int y = z0 - 1 + zz;
      const int oy = y < 0 ? -1 : (y >= B ? 1 : 0);
      const int32_t nb = oy < 0 ? nb_lo : (oy > 0 ? nb_hi : nb_mid);
      const int64_t idx = nb >= 0 ? static_cast<int64_t>(nb) * L.S + (y - oy * B) * B + lx : 0;
      cp_async8(su + zz * Bu + lane, a.u + idx, nb >= 0);
      if (x < B && zz <= R) cp_async8(se + zz * Be + lane, a.eps + idx, nb >= 0);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const double om1 = 1.0 - a.omega;
  const double* ut = su + yb * Bu + lane;  // vertex row yb - 1, column x
  const double* et = se + yb * Be + lane;  // cell row yb - 1, cell column x
  double um_l = vl ? ut[-1] : 0.0, um = vl ? ut[0] : 0.0, um_r = vl ? ut[1] : 0.0;
  double u0_l = vl ? ut[Bu - 1] : 0.0, u0 = vl ? ut[Bu] : 0.0, u0_r = vl ? ut[Bu + 1] : 0.0;
  double em = cl ? et[0] : 0.0, em_l = vl ? et[-1] : 0.0;
  double sS = em_l + em;
  double part = 0.0;
#pragma unroll
  for (int k = 0; k < RB; ++k) {
    const double* up = ut + (k + 2) * Bu;  // vertex row yb + k + 1
    const double* ep = et + (k + 1) * Be;  // cell row yb + k
    const double up_l = vl ? up[-1] : 0.0, upc = vl ? up[0] : 0.0, up_r = vl ? up[1] : 0.0;
    const double e0 = cl ? ep[0] : 0.0, e0_l = vl ? ep[-1] : 0.0;
    const double sE = em + e0;
    const double sW = __shfl_up_sync(0xffffffffu, sE, 1);
    const double sN = e0_l + e0;
    double acc = em_l * um_l;
    acc = fma(em, um_r, acc);
    acc = fma(e0_l, up_l, acc);
    acc = fma(e0, up_r, acc);
    acc = acc + acc;
    acc = fma(sW, u0_l, acc);
    acc = fma(sE, u0_r, acc);
    acc = fma(sS, um, acc);
    acc = fma(sN, upc, acc);
    const int yl = yb + k;
    const int64_t slot = base + (z0 + yl) * B + x;
    const uint8_t vf = fv[k];
    double res = 0.0;
    // iota vertices keep their value in the Jacobi part of a block step (Sect. 4.2);
    // hanging values come from the coarser level (Sect. 3)
    const bool keep = OP == kJacobi && a.block && x % 3 != 0 && (z0 + yl) % 3 != 0;
    if constexpr (OP != kResidual) {
      if ((vf & MG_V_HANGING) || keep) res = u0;
    }
    if (vl && is_dof(vf) && !keep) {
      double t = fma(1.0 / 6.0, acc, bv[k]);  // b - off, off = k1 acc
      double dc = 0.0;
      if constexpr (AMODE != 0) {
        const double nbv[9] = {um_l, um, um_r, u0_l, u0, u0_r, up_l, upc, up_r};
        const int64_t sl = (z0 + yl) * B + x;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          if (q == 4) {
            if constexpr (OP != kJacobi) dc = load_delta<AMODE, double>(a.ahat, a.ascale, (brick * 9 + q) * L.S + sl, slot);
          } else {
            t = fma(-load_delta<AMODE, double>(a.ahat, a.ascale, (brick * 9 + q) * L.S + sl, slot), nbv[q], t);
          }
        }
      }
      if constexpr (OP == kJacobiNorm) {
        // the Jacobi update and, beside it, the residual b - A u of its input
        res = fma(dv[k], t, om1 * u0);
        const double r = fma(-fma(2.0 / 3.0, sW + sE, dc), u0, t);
        part = fma(r, r, part);
      } else if constexpr (OP == kJacobi) {
        res = fma(dv[k], t, om1 * u0);
      } else {
        const double D = fma(2.0 / 3.0, sW + sE, dc);
        const double r = fma(-D, u0, t);
        res = r;
        part = fma(r, r, part);
      }
    }
    if (vl) a.out[slot] = res;
    um_l = u0_l; um = u0; um_r = u0_r;
    u0_l = up_l; u0 = upc; u0_r = up_r;
    em = e0; em_l = e0_l;
    sS = sN;
  }
  return part;
}

template <int AMODE, int OP, int R>
__global__ void __launch_bounds__(96) k_sweep2f(SweepArgs<double> a) {
  pdl_enter();
  const double part = sweep2f_item<AMODE, OP, R>(a, blockIdx.x, blockIdx.y);
  if constexpr (OP == kResidual || OP == kJacobiNorm) {
    if (a.partial) store_partial_and_finish(part, a.partial, a.counter, a.norm2);
  }
}

// 3D, brick edge 9: one CTA of 128 threads per (brick, slab of R planes).  Thread t <
// 121 loads tile column (x, y) in [-1, 9]^2 of u (and of the cell coefficients) for
// every plane of the slab and its halo; thread t < 100 forms the per-cell corner
// sums q_c = eps_c S_c of its cell column with a rolling plane sum; thread t < 81
// marches its vertex column up the slab with the cells below / above and the values
// below / at the vertex carried in registers.  Vertex formula as in sweep_item:
//   (A u)_v = h/12 (5 sC u_v - sum_c q_c + sum_axis nbr n  S_n u_n).
template <typename T, int AMODE, int OP, int R>
__device__ __forceinline__ double sweep3c_item(const SweepArgs<T>& a, int64_t brick, int slab,
                                               unsigned char* smem_raw) {
  constexpr int B = 9, Bu = 11, Be = 10, UPL = Bu * Bu, EPL = Be * Be, PL = B * B, N3 = 27;
  const LevelDesc& L = a.L;
  const int z0 = slab * R;
  const int64_t base = brick * L.S;
  __syncthreads();  // the tile may still be read by a previous item of this CTA
  const int32_t* bn = L.brick_nbr + brick * N3;
  T* su = reinterpret_cast<T*>(smem_raw);
  T* se = su + UPL * (R + 2);
  T* sq = se + EPL * (R + 1);
  const int t = threadIdx.x;
  // b and flags of this thread's vertex column, fetched while the tile streams in
  T bv[R];
  uint8_t fv[R];
#pragma unroll
  for (int zl = 0; zl < R; ++zl) {
    const int64_t slot = base + (z0 + zl) * PL + t;
    fv[zl] = t < PL ? L.vflags[slot] : 0;
    bv[zl] = (t < PL && is_dof(fv[zl])) ? a.b[slot] : T(0);
  }
  if (t < UPL) {
    const int x = t % Bu - 1, y = t / Bu - 1;
    const int ox = x < 0 ? -1 : (x >= B ? 1 : 0), oy = y < 0 ? -1 : (y >= B ? 1 : 0);
    const int li = (y - oy * B) * B + (x - ox * B);
    const int nbase = (ox + 1) + 3 * (oy + 1);
    const int32_t nb_lo = bn[nbase], nb_mid = bn[nbase + 9], nb_hi = bn[nbase + 18];
    const bool cell = x < B && y < B;
    const int ce = (y + 1) * Be + (x + 1);
#pragma unroll
    for (int zz = 0; zz < R + 2; ++zz) {
      const int z = z0 - 1 + zz;
      const int oz = z < 0 ? -1 : (z >= B ? 1 : 0);
      const int32_t nb = oz < 0 ? nb_lo : (oz > 0 ? nb_hi : nb_mid);
      const int64_t idx = nb >= 0 ? static_cast<int64_t>(nb) * L.S + (z - oz * B) * PL + li : 0;
      cp_async_el(su + zz * UPL + t, a.u + idx, nb >= 0);
      if (cell && zz <= R) cp_async_el(se + zz * EPL + ce, a.eps + idx, nb >= 0);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (t < EPL) {
    const T* c0 = su + (t / Be) * Bu + (t % Be);  // lowest corner of cell column t
    T plo = (c0[0] + c0[1]) + (c0[Bu] + c0[Bu + 1]);
#pragma unroll
    for (int zz = 0; zz <= R; ++zz) {
      const T* c1 = c0 + (zz + 1) * UPL;
      const T phi = (c1[0] + c1[1]) + (c1[Bu] + c1[Bu + 1]);
      const T ev = se[zz * EPL + t];
      sq[zz * EPL + t] = ev != T(0) ? ev * (plo + phi) : T(0);  // absent cells cost no arithmetic
      plo = phi;
    }
  }
  __syncthreads();
  double part = 0.0;
  if (t < PL) {
    const int x = t % B, y = t / B;
    const int cu = (y + 1) * Bu + (x + 1), ce = (y + 1) * Be + (x + 1);
    const T hscale = static_cast<T>(L.h);
    // cells below the first vertex (lower corner z0 - 1): e at (x, y), (x-1, y), (x, y-1),
    // (x-1, y-1); the plane sums of their e and q are carried to the next vertex up
    T eb0 = se[ce], eb1 = se[ce - 1], eb2 = se[ce - Be], eb3 = se[ce - Be - 1];
    T szm = (eb0 + eb1) + (eb2 + eb3);
    T qsb = (sq[ce] + sq[ce - 1]) + (sq[ce - Be] + sq[ce - Be - 1]);
    T ub = su[cu], u0 = su[UPL + cu];
    const T om1 = T(1) - a.omega;
#pragma unroll
    for (int zl = 0; zl < R; ++zl) {
      const T* uc = su + (zl + 1) * UPL + cu;
      const T ua = uc[UPL];
      const T* ea = se + (zl + 1) * EPL + ce;
      const T* qa = sq + (zl + 1) * EPL + ce;
      const T ea0 = ea[0], ea1 = ea[-1], ea2 = ea[-Be], ea3 = ea[-Be - 1];
      const T szp = (ea0 + ea1) + (ea2 + ea3);
      const T qsa = (qa[0] + qa[-1]) + (qa[-Be] + qa[-Be - 1]);
      const int s = (z0 + zl) * PL + t;
      const int64_t slot = base + s;
      const uint8_t vf = fv[zl];
      T res = T(0);
      const bool keep = OP == kJacobi && a.block && x % 3 != 0 && y % 3 != 0 && (z0 + zl) % 3 != 0;
      if constexpr (OP == kJacobi || OP == kJacobiNorm) {
        if ((vf & MG_V_HANGING) || keep) res = u0;
      }
      if (is_dof(vf) && !keep) {
        // cell e<bx><by><bz> has lower corner v - (bx, by, bz): a = above (bz 0), b = below
        const T p00 = ea0 + eb0, p10 = ea1 + eb1, p01 = ea2 + eb2, p11 = ea3 + eb3;
        const T sxp = p00 + p01, sxm = p10 + p11, syp = p00 + p10, sym = p01 + p11;
        const T sC = sxp + sxm;
        const T Q = qsa + qsb;
        T s1 = sxp * uc[1];
        s1 = fma(sxm, uc[-1], s1);
        s1 = fma(syp, uc[Bu], s1);
        s1 = fma(sym, uc[-Bu], s1);
        s1 = fma(szp, ua, s1);
        s1 = fma(szm, ub, s1);
        const uint64_t akey = AMODE != 0 ? delta_row<AMODE>(a.ascale, slot) : 0;
        if constexpr (std::is_same<T, double>::value && (OP == kJacobi || OP == kJacobiNorm)) {
          // FP64 Jacobi with omega / D from the setup: off = A u - D u
          //   = h/12 (sC u_v + sum_axis nbr S_n u_n - sum_c q_c)   (D = h/3 sC)
          T t2 = fma(-(hscale * static_cast<T>(1.0 / 12.0)), fma(sC, u0, s1 - Q), bv[zl]);
          T dc = T(0);
          if (AMODE != 0 && delta_row_live<AMODE>(akey)) {
#pragma unroll
            for (int k = 0; k < N3; ++k) {
              if (k == N3 / 2) {
                if constexpr (OP == kJacobiNorm) dc = load_delta<AMODE, T>(a.ahat, a.ascale, (brick * N3 + k) * L.S + s, slot, k, akey);
                continue;
              }
              const int off = (k % 3 - 1) + Bu * ((k / 3) % 3 - 1) + UPL * (k / 9 - 1);
              t2 = fma(-load_delta<AMODE, T>(a.ahat, a.ascale, (brick * N3 + k) * L.S + s, slot, k, akey),
                       uc[off], t2);
            }
          }
          res = fma(a.dinv[slot], t2, om1 * u0);
          if constexpr (OP == kJacobiNorm) {  // and the residual b - A u = t2 - D u of its input
            const T r = fma(-fma(sC, hscale * static_cast<T>(1.0 / 3.0), dc), u0, t2);
            part = fma(static_cast<double>(r), static_cast<double>(r), part);
          }
        } else {
          T Au = fma(T(5) * sC, u0, s1 - Q) * (hscale * static_cast<T>(1.0 / 12.0));
          T D = sC * (hscale * static_cast<T>(1.0 / 3.0));
          if (AMODE != 0 && delta_row_live<AMODE>(akey)) {
#pragma unroll
            for (int k = 0; k < N3; ++k) {
              const int off = (k % 3 - 1) + Bu * ((k / 3) % 3 - 1) + UPL * (k / 9 - 1);
              const T d = load_delta<AMODE, T>(a.ahat, a.ascale, (brick * N3 + k) * L.S + s, slot, k, akey,
                                               a_lo_off<AMODE>(L, N3));
              Au = fma(d, uc[off], Au);
              if (k == N3 / 2) D += d;
            }
          }
          const T r = bv[zl] - Au;
          if constexpr (OP == kJacobi || OP == kJacobiNorm) {
            res = fma(a.omega * r, recip_nr(D), u0);
            if constexpr (OP == kJacobiNorm) part += static_cast<double>(r) * static_cast<double>(r);
          } else {
            res = r;
            part += static_cast<double>(r) * static_cast<double>(r);
          }
        }
      }
      a.out[slot] = res;
      eb0 = ea0; eb1 = ea1; eb2 = ea2; eb3 = ea3;
      szm = szp;
      qsb = qsa;
      ub = u0;
      u0 = ua;
    }
  }
  return part;
}

template <typename T, int AMODE, int OP, int R>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? 4 : 8) k_sweep3c(SweepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_enter();
  const double part = sweep3c_item<T, AMODE, OP, R>(a, blockIdx.x, blockIdx.y, smem_raw);
  if constexpr (OP == kResidual || OP == kJacobiNorm) {
    if (a.partial) store_partial_and_finish(part, a.partial, a.counter, a.norm2);
  }
}

// FP32 column kernels for a runtime slab depth (batched sweeps: items of one launch
// may come from levels with different slabs)
template <int DIM, typename T, int AMODE, int OP>
__device__ __forceinline__ double sweep_col_item(const SweepArgs<T>& a, int64_t brick, int slab,
                                                 unsigned char* smem_raw) {
  if constexpr (DIM == 2) {
    switch (a.R) {
      case 1: return sweep2c_item<T, AMODE, OP, 1>(a, brick, slab);
      case 3: return sweep2c_item<T, AMODE, OP, 3>(a, brick, slab);
      case 9: return sweep2c_item<T, AMODE, OP, 9>(a, brick, slab);
      default: return sweep2c_item<T, AMODE, OP, 27>(a, brick, slab);
    }
  } else {
    switch (a.R) {
      case 1: return sweep3c_item<T, AMODE, OP, 1>(a, brick, slab, smem_raw);
      case 3: return sweep3c_item<T, AMODE, OP, 3>(a, brick, slab, smem_raw);
      default: return sweep3c_item<T, AMODE, OP, 9>(a, brick, slab, smem_raw);
    }
  }
}

}  // namespace mg
