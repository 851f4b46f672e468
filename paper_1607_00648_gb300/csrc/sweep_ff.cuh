// Finest-level FP64 sweeps in float-float arithmetic.  GB300's FP64 units deliver about
// 1/64 of its FP32 rate (measured ~1.05 TFLOP/s by mg_probe_fp64_fma), so the FP64
// sweeps of sweep_fast.cuh are bound by the FP64 pipe at ~14 (2D) and ~33 (3D) FP64
// instructions per vertex.  Here the same vertex formulas run on the FP32 units: a value
// is the unevaluated sum h + l of two binary32 numbers (47-49 significant bits instead of
// 53), built from the error-free transformations
//   TwoSum      s + e = a + b exactly        (Knuth, TAOCP vol. 2, Sect. 4.2.2, Thm. B)
//   TwoProduct  p + e = a b exactly, e = fma(a, b, -p)
// and sums of products carry their rounding errors in a second accumulator, as the
// compensated dot product of Ogita, Rump & Oishi ("Accurate sum and dot product", SIAM J.
// Sci. Comput. 26, 2005).  Inputs and outputs stay binary64: u and b are split into pairs
// from their bit patterns (integer instructions), the cell coefficients and omega / D come
// pre-split from the setup, and each result is joined back with one FP64 addition.
//
// Accuracy: a split u or b is exact to 2^-48 relative; every product and sum keeps its
// error below ~2^-47 of the magnitudes involved, so a sweep's result differs from the
// exact one by a few 2^-47 of the sum of the absolute terms (FP64: a few 2^-53).
// Range: binary32 exponents, i.e. nonzero |values| in [2^-103, 2^128): smaller ones
// are flushed to zero, larger ones (and NaN, Inf) become NaN, which the solvers report
// as a non-finite residual.
#pragma once

#include "sweep_fast.cuh"

namespace mg {

struct ff2 {
  float h, l;
};

// pairs travel in binary64 containers: low word = h, high word = l (plain register moves)
__device__ __forceinline__ ff2 ff_unpack(double v) {
  return {__int_as_float(__double2loint(v)), __int_as_float(__double2hiint(v))};
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float ap = __fsub_rn(s, b);
  const float bp = __fsub_rn(s, ap);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// x + y, unnormalised (|l| stays ~2^-23 of |h| + the parts' magnitudes)
__device__ __forceinline__ ff2 ff_add(ff2 x, ff2 y) {
  float s, e;
  two_sum(x.h, y.h, s, e);
  return {s, __fadd_rn(e, __fadd_rn(x.l, y.l))};
}

// x y as an unnormalised pair: the rounded product of the high parts and, beside it, its
// exact rounding error plus the two cross terms (x.l y.l, below 2^-46 of |x y|, is dropped)
__device__ __forceinline__ ff2 ff_mul(ff2 x, ff2 y) {
  const float p = __fmul_rn(x.h, y.h);
  float q = fmaf(x.h, y.h, -p);
  q = fmaf(x.h, y.l, q);
  q = fmaf(x.l, y.h, q);
  return {p, q};
}

// sum of products: s is the running rounded sum of the products' high parts, c collects
// every rounding error (of the products and of the additions into s)
struct FfAcc {
  float s, c;
  __device__ __forceinline__ void first(ff2 x, ff2 y) {
    const ff2 p = ff_mul(x, y);
    s = p.h;
    c = p.l;
  }
  __device__ __forceinline__ void add(ff2 x, ff2 y) {
    const ff2 p = ff_mul(x, y);
    float e;
    two_sum(s, p.h, s, e);
    c = __fadd_rn(c, __fadd_rn(e, p.l));
  }
  __device__ __forceinline__ ff2 get() const { return {s, c}; }
};

// binary64 -> pair from the bit pattern, rounded to nearest twice: h = the value rounded
// to 24 significant bits (2^28 added to the 64-bit pattern, half-way cases away from zero;
// a carry into the exponent field gives the next binade), l = the remainder d - h, an
// integer of at most 29 bits in units of d's last place, converted to binary32 and scaled
// by d's exponent; |d - (h + l)| <= max(2^-48 |d|, 2^-126) (l is flushed to zero below 2^-126)
__device__ __forceinline__ ff2 ff_from_double(double d) {
  const uint32_t hw = static_cast<uint32_t>(__double2hiint(d)), lw = static_cast<uint32_t>(__double2loint(d));
  const uint32_t s = hw & 0x80000000u, e = (hw >> 20) & 0x7ffu;
  if (e < 920u) return {__uint_as_float(s), 0.0f};  // |d| < 2^-103 and zero
  if (e > 1149u) return {__uint_as_float(0x7fc00000u), 0.0f};  // beyond binary32 range, Inf, NaN
  const uint64_t rb = ((static_cast<uint64_t>(hw) << 32) | lw) + (1ull << 28);
  const uint32_t rhw = static_cast<uint32_t>(rb >> 32), rlw = static_cast<uint32_t>(rb);
  const uint32_t hb = s | ((((rhw >> 20) & 0x7ffu) - 896u) << 23) | ((rhw & 0xfffffu) << 3) | (rlw >> 29);
  const int32_t rem = static_cast<int32_t>((lw + (1u << 28)) & 0x1fffffffu) - (1 << 28);
  const uint32_t fb = __float_as_uint(__int2float_rn(rem));
  const int le = static_cast<int>((fb >> 23) & 0xffu) + static_cast<int>(e) - 1075;
  const float l = (rem == 0 || le < 1) ? 0.0f : __uint_as_float((fb + ((e - 1075u) << 23)) ^ s);
  return {__uint_as_float(hb), l};
}

// binary32 -> binary64 exactly from the bit pattern (subnormal floats -> signed zero)
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t b = __float_as_uint(f), s = b & 0x80000000u, e = (b >> 23) & 0xffu;
  uint32_t hw, lw;
  if (e == 0u) {
    hw = s;
    lw = 0u;
  } else if (e == 0xffu) {
    hw = s | 0x7ff00000u | ((b & 0x7fffffu) ? 0x80000u : 0u);
    lw = 0u;
  } else {
    hw = s | (((b & 0x7fffffffu) >> 3) + (896u << 20));
    lw = b << 29;
  }
  return __hiloint2double(static_cast<int>(hw), static_cast<int>(lw));
}

// h + l rounded to binary64: the one FP64 instruction of a vertex update
__device__ __forceinline__ double ff_to_double(ff2 x) { return f2d_bits(x.h) + f2d_bits(x.l); }

// a binary64 constant as a pair (host or device; the low part by exact FP64 subtraction)
__host__ __device__ constexpr float ff_hi(double c) { return static_cast<float>(c); }
__host__ __device__ constexpr float ff_lo(double c) { return static_cast<float>(c - static_cast<double>(static_cast<float>(c))); }

// 2D, brick edge 27, finest level (no stored deltas): the operations of sweep2f_item
// (column marching, pair sums of cell coefficients shared through the warp) in pairs.
//   Jacobi:   u' = (omega / D) (b - off u) + (1 - omega) u,  off u = -(1/6) acc
//   residual: r = b - A u = b + (1/6) acc - D u,  D = (2/3) (sW + sE)
// with acc = 2 sum_corners e_c u_c + sum_edges (e_c1 + e_c2) u_e (bilinear element).
template <int OP, int R>
__device__ __forceinline__ double sweep2x_item(const SweepArgs<double>& a, int64_t brick, int slab) {
  constexpr int B = 27, Bu = B + 2, Be = B + 1;
  constexpr int NW = R >= 3 ? 3 : 1, RB = R / NW;
  __shared__ __align__(16) double su[(R + 2) * Bu];  // u staged as binary64, then split in place
  __shared__ __align__(16) double se[(R + 1) * Be];  // pre-split cell coefficients
  const LevelDesc& L = a.L;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = brick * L.S;
  const int z0 = slab * R;
  __syncthreads();  // the tile may still be read by a previous item of this CTA
  const int32_t* bn = L.brick_nbr + brick * 9;
  const int x = lane - 1;
  const bool vl = x >= 0 && x < B;  // lanes 1..27: vertex columns 0..26
  const bool cl = lane <= B;        // lanes 0..27: cell columns -1..26
  const int yb = w * RB;
  double bv[RB], dv[RB];
  uint8_t fv[RB];
#pragma unroll
  for (int k = 0; k < RB; ++k) {
    const int64_t slot = base + (z0 + yb + k) * B + x;
    fv[k] = vl ? L.vflags[slot] : 0;
    const bool on = vl && is_dof(fv[k]);
    bv[k] = on ? a.b[slot] : 0.0;
    dv[k] = (OP != kResidual && on) ? a.dinv_pair[slot] : 0.0;
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
      if (x < B && zz <= R) cp_async8(se + zz * Be + lane, a.eps_pair + idx, nb >= 0);
    }
    cp_async_wait_all();
    for (int zz = w; zz < R + 2; zz += NW) {  // split this thread's own staged values
      const ff2 p = ff_from_double(su[zz * Bu + lane]);
      su[zz * Bu + lane] = __hiloint2double(__float_as_int(p.l), __float_as_int(p.h));
    }
  }
  __syncthreads();
  const ff2 om1 = ff_from_double(1.0 - a.omega);
  constexpr float k6h = ff_hi(1.0 / 6.0), k6l = ff_lo(1.0 / 6.0);
  constexpr float k23h = ff_hi(2.0 / 3.0), k23l = ff_lo(2.0 / 3.0);
  const ff2 z{0.0f, 0.0f};
  const double* ut = su + yb * Bu + lane;  // vertex row yb - 1, column x
  const double* et = se + yb * Be + lane;  // cell row yb - 1, cell column x
  ff2 um_l = vl ? ff_unpack(ut[-1]) : z, um = vl ? ff_unpack(ut[0]) : z, um_r = vl ? ff_unpack(ut[1]) : z;
  ff2 u0_l = vl ? ff_unpack(ut[Bu - 1]) : z, u0 = vl ? ff_unpack(ut[Bu]) : z, u0_r = vl ? ff_unpack(ut[Bu + 1]) : z;
  ff2 em = cl ? ff_unpack(et[0]) : z, em_l = vl ? ff_unpack(et[-1]) : z;
  ff2 sS = ff_add(em_l, em);
  double part = 0.0;
#pragma unroll
  for (int k = 0; k < RB; ++k) {
    const double* up = ut + (k + 2) * Bu;
    const double* ep = et + (k + 1) * Be;
    const ff2 up_l = vl ? ff_unpack(up[-1]) : z, upc = vl ? ff_unpack(up[0]) : z, up_r = vl ? ff_unpack(up[1]) : z;
    const ff2 e0 = cl ? ff_unpack(ep[0]) : z, e0_l = vl ? ff_unpack(ep[-1]) : z;
    const ff2 sE = ff_add(em, e0);
    const ff2 sW{__shfl_up_sync(0xffffffffu, sE.h, 1), __shfl_up_sync(0xffffffffu, sE.l, 1)};
    const ff2 sN = ff_add(e0_l, e0);
    const int yl = yb + k;
    const int64_t slot = base + (z0 + yl) * B + x;
    const uint8_t vf = fv[k];
    double res = 0.0;
    if constexpr (OP != kResidual) {
      if (vf & MG_V_HANGING) res = a.u[slot];  // hanging values come from the coarser level (Sect. 3)
    }
    if (vl && is_dof(vf)) {
      FfAcc acc;
      acc.first(em_l, um_l);
      acc.add(em, um_r);
      acc.add(e0_l, up_l);
      acc.add(e0, up_r);
      acc.s = acc.s * 2.0f;  // exact
      acc.c = acc.c * 2.0f;
      acc.add(sW, u0_l);
      acc.add(sE, u0_r);
      acc.add(sS, um);
      acc.add(sN, upc);
      // t = b + acc / 6
      const ff2 b2 = ff_from_double(bv[k]);
      const ff2 q6 = ff_mul(acc.get(), ff2{k6h, k6l});
      ff2 t;
      {
        float s, e;
        two_sum(b2.h, q6.h, s, e);
        t = {s, __fadd_rn(e, __fadd_rn(b2.l, q6.l))};
      }
      if constexpr (OP != kResidual) {
        const ff2 p1 = ff_mul(ff_unpack(dv[k]), t);
        const ff2 p2 = ff_mul(om1, u0);
        res = ff_to_double(ff_add(p1, p2));
        if constexpr (OP == kJacobiNorm) {  // and the residual b - A u of its input
          const ff2 D = ff_mul(ff_add(sW, sE), ff2{k23h, k23l});
          const ff2 Du = ff_mul(D, u0);
          const double r = ff_to_double(ff_add(t, ff2{-Du.h, -Du.l}));
          part = fma(r, r, part);
        }
      } else {
        const ff2 D = ff_mul(ff_add(sW, sE), ff2{k23h, k23l});
        const ff2 Du = ff_mul(D, u0);
        const double r = ff_to_double(ff_add(t, ff2{-Du.h, -Du.l}));
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

template <int OP, int R>
__global__ void __launch_bounds__(96) k_sweep2x(SweepArgs<double> a) {
  pdl_enter();
  const double part = sweep2x_item<OP, R>(a, blockIdx.x, blockIdx.y);
  if constexpr (OP == kResidual || OP == kJacobiNorm) {
    if (a.partial) store_partial_and_finish(part, a.partial, a.counter, a.norm2);
  }
}

// 3D, brick edge 9, finest level: the operations of sweep3c_item in pairs.  Per cell c the
// corner sum q_c = eps_c S_c (S_c = sum of u over the cell's 8 corners), per vertex v
//   (A u)_v = h/12 (5 sC u_v - sum_c q_c + sum_axis nbr S_n u_n)
//   Jacobi:   u' = (omega / D) (b - (A u - D u)) + (1 - omega) u,  D = h/3 sC
//   residual: r = b - A u
template <int OP, int R>
__device__ __forceinline__ double sweep3x_item(const SweepArgs<double>& a, int64_t brick, int slab,
                                               unsigned char* smem_raw) {
  constexpr int B = 9, Bu = 11, Be = 10, UPL = Bu * Bu, EPL = Be * Be, PL = B * B, N3 = 27;
  const LevelDesc& L = a.L;
  const int z0 = slab * R;
  const int64_t base = brick * L.S;
  __syncthreads();  // the tile may still be read by a previous item of this CTA
  const int32_t* bn = L.brick_nbr + brick * N3;
  double* su = reinterpret_cast<double*>(smem_raw);  // u staged as binary64, then split in place
  double* se = su + UPL * (R + 2);                   // pre-split cell coefficients
  double* sq = se + EPL * (R + 1);                   // cell corner sums q_c (pairs)
  const int t = threadIdx.x;
  double bv[R], dv[R];
  uint8_t fv[R];
#pragma unroll
  for (int zl = 0; zl < R; ++zl) {
    const int64_t slot = base + (z0 + zl) * PL + t;
    fv[zl] = t < PL ? L.vflags[slot] : 0;
    const bool on = t < PL && is_dof(fv[zl]);
    bv[zl] = on ? a.b[slot] : 0.0;
    dv[zl] = (OP != kResidual && on) ? a.dinv_pair[slot] : 0.0;
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
      cp_async8(su + zz * UPL + t, a.u + idx, nb >= 0);
      if (cell && zz <= R) cp_async8(se + zz * EPL + ce, a.eps_pair + idx, nb >= 0);
    }
    cp_async_wait_all();
#pragma unroll
    for (int zz = 0; zz < R + 2; ++zz) {  // split this thread's own staged values
      const ff2 p = ff_from_double(su[zz * UPL + t]);
      su[zz * UPL + t] = __hiloint2double(__float_as_int(p.l), __float_as_int(p.h));
    }
  }
  __syncthreads();
  const ff2 z{0.0f, 0.0f};
  if (t < EPL) {
    const double* c0 = su + (t / Be) * Bu + (t % Be);  // lowest corner of cell column t
    ff2 plo = ff_add(ff_add(ff_unpack(c0[0]), ff_unpack(c0[1])), ff_add(ff_unpack(c0[Bu]), ff_unpack(c0[Bu + 1])));
#pragma unroll
    for (int zz = 0; zz <= R; ++zz) {
      const double* c1 = c0 + (zz + 1) * UPL;
      const ff2 phi =
          ff_add(ff_add(ff_unpack(c1[0]), ff_unpack(c1[1])), ff_add(ff_unpack(c1[Bu]), ff_unpack(c1[Bu + 1])));
      const ff2 ev = ff_unpack(se[zz * EPL + t]);
      const ff2 q = ev.h != 0.0f ? ff_mul(ev, ff_add(plo, phi)) : z;  // absent cells cost no arithmetic
      sq[zz * EPL + t] = __hiloint2double(__float_as_int(q.l), __float_as_int(q.h));
      plo = phi;
    }
  }
  __syncthreads();
  double part = 0.0;
  if (t < PL) {
    const int x = t % B, y = t / B;
    const int cu = (y + 1) * Bu + (x + 1), ce = (y + 1) * Be + (x + 1);
    const ff2 hk = ff_from_double(L.h * (1.0 / 12.0));
    const ff2 om1 = ff_from_double(1.0 - a.omega);
    ff2 eb0 = ff_unpack(se[ce]), eb1 = ff_unpack(se[ce - 1]), eb2 = ff_unpack(se[ce - Be]),
        eb3 = ff_unpack(se[ce - Be - 1]);
    ff2 szm = ff_add(ff_add(eb0, eb1), ff_add(eb2, eb3));
    ff2 qsb = ff_add(ff_add(ff_unpack(sq[ce]), ff_unpack(sq[ce - 1])),
                     ff_add(ff_unpack(sq[ce - Be]), ff_unpack(sq[ce - Be - 1])));
    ff2 ub = ff_unpack(su[cu]), u0 = ff_unpack(su[UPL + cu]);
#pragma unroll
    for (int zl = 0; zl < R; ++zl) {
      const double* uc = su + (zl + 1) * UPL + cu;
      const ff2 ua = ff_unpack(uc[UPL]);
      const double* ea = se + (zl + 1) * EPL + ce;
      const double* qa = sq + (zl + 1) * EPL + ce;
      const ff2 ea0 = ff_unpack(ea[0]), ea1 = ff_unpack(ea[-1]), ea2 = ff_unpack(ea[-Be]),
                ea3 = ff_unpack(ea[-Be - 1]);
      const ff2 szp = ff_add(ff_add(ea0, ea1), ff_add(ea2, ea3));
      const ff2 qsa = ff_add(ff_add(ff_unpack(qa[0]), ff_unpack(qa[-1])), ff_add(ff_unpack(qa[-Be]),
                                                                                 ff_unpack(qa[-Be - 1])));
      const int64_t slot = base + (z0 + zl) * PL + t;
      const uint8_t vf = fv[zl];
      double res = 0.0;
      if constexpr (OP != kResidual) {
        if (vf & MG_V_HANGING) res = a.u[slot];  // hanging values come from the coarser level (Sect. 3)
      }
      if (is_dof(vf)) {
        // cell e<bx><by><bz> has lower corner v - (bx, by, bz): a = above (bz 0), b = below
        const ff2 p00 = ff_add(ea0, eb0), p10 = ff_add(ea1, eb1), p01 = ff_add(ea2, eb2), p11 = ff_add(ea3, eb3);
        const ff2 sxp = ff_add(p00, p01), sxm = ff_add(p10, p11), syp = ff_add(p00, p10), sym = ff_add(p01, p11);
        const ff2 sC = ff_add(sxp, sxm);
        const ff2 Q = ff_add(qsa, qsb);
        FfAcc acc;
        acc.first(sxp, ff_unpack(uc[1]));
        acc.add(sxm, ff_unpack(uc[-1]));
        acc.add(syp, ff_unpack(uc[Bu]));
        acc.add(sym, ff_unpack(uc[-Bu]));
        acc.add(szp, ua);
        acc.add(szm, ub);
        // Jacobi: sC u_v (off-diagonal part: A u - D u); residual: 5 sC u_v (A u)
        acc.add(OP != kResidual ? sC : ff_mul(sC, ff2{5.0f, 0.0f}), u0);
        {
          float s, e;
          two_sum(acc.s, -Q.h, s, e);
          acc.s = s;
          acc.c = __fadd_rn(acc.c, __fsub_rn(e, Q.l));
        }
        const ff2 hq = ff_mul(acc.get(), hk);
        const ff2 b2 = ff_from_double(bv[zl]);
        ff2 t2;
        {
          float s, e;
          two_sum(b2.h, -hq.h, s, e);
          t2 = {s, __fadd_rn(e, __fsub_rn(b2.l, hq.l))};
        }
        if constexpr (OP != kResidual) {
          res = ff_to_double(ff_add(ff_mul(ff_unpack(dv[zl]), t2), ff_mul(om1, u0)));
          if constexpr (OP == kJacobiNorm) {  // and the residual t2 - D u, D = h/3 sC = 4 (h/12) sC
            const ff2 du = ff_mul(ff_mul(sC, hk), u0);
            const double r = ff_to_double(ff_add(t2, ff2{-4.0f * du.h, -4.0f * du.l}));
            part = fma(r, r, part);
          }
        } else {
          const double r = ff_to_double(t2);
          res = r;
          part = fma(r, r, part);
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

template <int OP, int R>
__global__ void __launch_bounds__(128, 4) k_sweep3x(SweepArgs<double> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_enter();
  const double part = sweep3x_item<OP, R>(a, blockIdx.x, blockIdx.y, smem_raw);
  if constexpr (OP == kResidual || OP == kJacobiNorm) {
    if (a.partial) store_partial_and_finish(part, a.partial, a.counter, a.norm2);
  }
}

}  // namespace mg
