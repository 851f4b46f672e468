// Two damped Jacobi sweeps in one launch (2D levels of brick edge 27 and 9: the FP32
// cycles of the mixed path, the coarse levels of FP64 cycles, lockstep FP32 batches).
// These levels are L2-resident, so a sweep costs its launch and the dependency on its
// predecessor (a round trip through L2), not bandwidth; smoothing with nu = 2 therefore
// pays that latency twice per level and side.  Here one CTA per (brick, slab of R rows)
// stages u with a two-vertex halo and the cell coefficients with a two-cell halo, forms
// the first sweep on the slab and a one-vertex ring around it in shared memory (the
// ring's b, flags and stored deltas come from the neighbouring bricks), and the second
// sweep of the slab from it.  Every vertex update is the arithmetic of the single-sweep
// kernel it replaces (brick edge 27, FP32: sweep2c_item's stencil2, the deltas in entry
// order, u + omega r / D; FP64: sweep2f_item's; brick edge 9: the generic sweep_item's),
// so the result is bit for bit that of two separate sweeps.  Levels with hanging
// vertices, block smoothing and the anisotropy pass keep separate sweeps.
#pragma once

#include "sweep_fast.cuh"

namespace mg {

// one damped Jacobi update of vertex (x, y) (global brick-local coordinates may lie in a
// neighbouring brick) from the values around position c of a shared tile with row
// stride ws and the cells around position ce of a cell tile with row stride wc
template <typename T, int AMODE>
__device__ __forceinline__ T pair_update(const SweepArgs<T>& a, const T* c, int ws, const T* ce, int wc,
                                         int64_t slot, int64_t plane_base, uint8_t vf, T bv) {
  const T u0 = c[0];
  if (!is_dof(vf)) return (vf & MG_V_HANGING) ? u0 : T(0);
  const T um_l = c[-ws - 1], um = c[-ws], um_r = c[-ws + 1];
  const T u0_l = c[-1], u0_r = c[1];
  const T up_l = c[ws - 1], up = c[ws], up_r = c[ws + 1];
  T Au, D;
  stencil2<T>(ce[-wc - 1], ce[-wc], ce[-1], ce[0], um_l, um, um_r, u0_l, u0, u0_r, up_l, up, up_r, Au, D);
  const uint64_t akey = AMODE != 0 ? delta_row<AMODE>(a.ascale, slot) : 0;
  if (AMODE != 0 && delta_row_live<AMODE>(akey)) {
    const T nbv[9] = {um_l, um, um_r, u0_l, u0, u0_r, up_l, up, up_r};
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const T d = load_delta<AMODE, T>(a.ahat, a.ascale, plane_base + static_cast<int64_t>(q) * a.L.S, slot, q, akey,
                                       a_lo_off<AMODE>(a.L, 9));
      Au = fma(d, nbv[q], Au);
      if (q == 4) D += d;
    }
  }
  const T r = bv - Au;
  return fma(a.omega * r, recip_nr(D), u0);
}

// FP64 hierarchies: the operations of sweep2f_item in its order (edge pair sums of cell
// coefficients, corners doubled, b + acc / 6 minus the stored deltas, then omega / D from
// the setup), so that a pair equals two k_sweep2f sweeps bit for bit
template <int AMODE>
__device__ __forceinline__ double pair_update_f64(const SweepArgs<double>& a, const double* c, int ws,
                                                  const double* ce, int wc, int64_t slot, int64_t plane_base,
                                                  uint8_t vf, double bv) {
  const double u0 = c[0];
  if (!is_dof(vf)) return (vf & MG_V_HANGING) ? u0 : 0.0;
  const double um_l = c[-ws - 1], um = c[-ws], um_r = c[-ws + 1];
  const double u0_l = c[-1], u0_r = c[1];
  const double up_l = c[ws - 1], upc = c[ws], up_r = c[ws + 1];
  // cells: em_l = (x-1, y-1), em = (x, y-1), e0_l = (x-1, y), e0 = (x, y)
  const double em_l = ce[-wc - 1], em = ce[-wc], e0_l = ce[-1], e0 = ce[0];
  const double sE = em + e0, sW = em_l + e0_l, sN = e0_l + e0, sS = em_l + em;
  double acc = em_l * um_l;
  acc = fma(em, um_r, acc);
  acc = fma(e0_l, up_l, acc);
  acc = fma(e0, up_r, acc);
  acc = acc + acc;
  acc = fma(sW, u0_l, acc);
  acc = fma(sE, u0_r, acc);
  acc = fma(sS, um, acc);
  acc = fma(sN, upc, acc);
  double t = fma(1.0 / 6.0, acc, bv);
  if constexpr (AMODE != 0) {
    const double nbv[9] = {um_l, um, um_r, u0_l, u0, u0_r, up_l, upc, up_r};
#pragma unroll
    for (int q = 0; q < 9; ++q)
      if (q != 4) t = fma(-load_delta<AMODE, double>(a.ahat, a.ascale, plane_base + q * a.L.S, slot), nbv[q], t);
  }
  return fma(a.dinv[slot], t, (1.0 - a.omega) * u0);
}

// brick edge 9 (2D level 2): the operations of the generic sweep_item in its order
// (off-diagonal part and diagonal apart, the deltas into them, then the update), with
// omega / D from the setup where the hierarchy stores it (FP64)
template <typename T, int AMODE>
__device__ __forceinline__ T pair_update_gen(const SweepArgs<T>& a, const T* c, int ws, const T* ce, int wc,
                                             int64_t slot, int64_t plane_base, uint8_t vf, T bv) {
  const T u0 = c[0];
  if (!is_dof(vf)) return (vf & MG_V_HANGING) ? u0 : T(0);
  const T e_sw = ce[-wc - 1], e_se = ce[-wc], e_nw = ce[-1], e_ne = ce[0];
  const T sW = e_sw + e_nw, sE = e_se + e_ne, sS = e_sw + e_se, sN = e_nw + e_ne;
  const T sC = sW + sE;
  T a1 = sW * c[-1];
  a1 = fma(sE, c[1], a1);
  a1 = fma(sS, c[-ws], a1);
  a1 = fma(sN, c[ws], a1);
  T a2 = e_sw * c[-ws - 1];
  a2 = fma(e_se, c[-ws + 1], a2);
  a2 = fma(e_nw, c[ws - 1], a2);
  a2 = fma(e_ne, c[ws + 1], a2);
  const T k0 = static_cast<T>(elem_k(2, 0)), k1 = static_cast<T>(elem_k(2, 1)), k2 = static_cast<T>(elem_k(2, 2));
  T D = k0 * sC;
  T off = fma(k1, a1, k2 * a2);
  const uint64_t akey = AMODE != 0 ? delta_row<AMODE>(a.ascale, slot) : 0;
  if (AMODE != 0 && delta_row_live<AMODE>(akey)) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const T d = load_delta<AMODE, T>(a.ahat, a.ascale, plane_base + static_cast<int64_t>(k) * a.L.S, slot, k, akey,
                                       a_lo_off<AMODE>(a.L, 9));
      if (k == 4)
        D += d;
      else
        off = fma(d, c[(k % 3 - 1) + ws * (k / 3 - 1)], off);
    }
  }
  if (a.dinv) return fma(a.dinv[slot], bv - off, (T(1) - a.omega) * u0);
  const T r = bv - fma(D, u0, off);
  return fma(a.omega * r, recip_nr(D), u0);
}

template <typename T, int AMODE, int R, int B = 27>
__device__ __forceinline__ void sweep_pair_item(const SweepArgs<T>& a, int64_t brick, int slab) {
  constexpr int WU = B + 4, HU = R + 4;  // u: columns -2 .. B + 1, rows z0 - 2 .. z0 + R + 1
  constexpr int WE = B + 3, HE = R + 3;  // cells: lower corners -2 .. B, z0 - 2 .. z0 + R
  constexpr int W1 = B + 2, H1 = R + 2;  // first sweep: columns -1 .. B, rows z0 - 1 .. z0 + R
  __shared__ __align__(16) T su[HU * WU];
  __shared__ __align__(16) T se[HE * WE];
  __shared__ __align__(16) T s1[H1 * W1];
  const LevelDesc& L = a.L;
  const int32_t* bn = L.brick_nbr + brick * 9;
  const int z0 = slab * R;
  // brick and local index of brick-relative position (x, y), x, y in [-B, 2B); -1 outside
  auto locate = [&](int x, int y, int64_t& nbl, int& li) {
    const int ox = x < 0 ? -1 : (x >= B ? 1 : 0), oy = y < 0 ? -1 : (y >= B ? 1 : 0);
    const int32_t nb = bn[(ox + 1) + 3 * (oy + 1)];
    nbl = nb;
    li = (y - oy * B) * B + (x - ox * B);
  };
  for (int i = threadIdx.x; i < HU * WU; i += blockDim.x) {
    const int x = i % WU - 2, y = z0 - 2 + i / WU;
    int64_t nb;
    int li;
    locate(x, y, nb, li);
    cp_async_el(su + i, a.u + (nb >= 0 ? nb * L.S + li : 0), nb >= 0);
    if (i % WU < WE && i / WU < HE)
      cp_async_el(se + (i / WU) * WE + i % WU, a.eps + (nb >= 0 ? nb * L.S + li : 0), nb >= 0);
  }
  cp_async_wait_all();
  __syncthreads();
  // first sweep on the slab and its ring
  for (int i = threadIdx.x; i < H1 * W1; i += blockDim.x) {
    const int cx = i % W1, cy = i / W1;
    const int x = cx - 1, y = z0 - 1 + cy;
    int64_t nb;
    int li;
    locate(x, y, nb, li);
    T v = T(0);
    if (nb >= 0) {
      const int64_t slot = nb * L.S + li;
      const uint8_t vf = L.vflags[slot];
      const T bv = is_dof(vf) ? a.b[slot] : T(0);
      if constexpr (B != 27)
        v = pair_update_gen<T, AMODE>(a, su + (cy + 1) * WU + cx + 1, WU, se + (cy + 1) * WE + cx + 1, WE, slot,
                                      nb * 9 * L.S + li, vf, bv);
      else if constexpr (std::is_same<T, double>::value)
        v = pair_update_f64<AMODE>(a, su + (cy + 1) * WU + cx + 1, WU, se + (cy + 1) * WE + cx + 1, WE, slot,
                                   nb * 9 * L.S + li, vf, bv);
      else
        v = pair_update<T, AMODE>(a, su + (cy + 1) * WU + cx + 1, WU, se + (cy + 1) * WE + cx + 1, WE, slot,
                                  nb * 9 * L.S + li, vf, bv);
    }
    s1[i] = v;
  }
  __syncthreads();
  // second sweep on the slab
  const int64_t base = brick * L.S;
  for (int i = threadIdx.x; i < R * B; i += blockDim.x) {
    const int x = i % B, yl = i / B;
    const int li = (z0 + yl) * B + x;
    const int64_t slot = base + li;
    const uint8_t vf = L.vflags[slot];
    const T bv = is_dof(vf) ? a.b[slot] : T(0);
    if constexpr (B != 27)
      a.out[slot] = pair_update_gen<T, AMODE>(a, s1 + (yl + 1) * W1 + x + 1, W1, se + (yl + 2) * WE + x + 2, WE, slot,
                                              brick * 9 * L.S + li, vf, bv);
    else if constexpr (std::is_same<T, double>::value)
      a.out[slot] = pair_update_f64<AMODE>(a, s1 + (yl + 1) * W1 + x + 1, W1, se + (yl + 2) * WE + x + 2, WE, slot,
                                           brick * 9 * L.S + li, vf, bv);
    else
      a.out[slot] = pair_update<T, AMODE>(a, s1 + (yl + 1) * W1 + x + 1, W1, se + (yl + 2) * WE + x + 2, WE, slot,
                                           brick * 9 * L.S + li, vf, bv);
  }
}

template <typename T, int AMODE, int R, int B = 27>
__global__ void __launch_bounds__(256) k_sweep_pair(SweepArgs<T> a) {
  pdl_enter();
  sweep_pair_item<T, AMODE, R, B>(a, blockIdx.x, blockIdx.y);
}

}  // namespace mg
