// Hot-path kernels: in-situ stencil sweeps (A2-A4), restriction (A5), prolongation
// (A6), hanging interpolation (A7) and reductions, templated on dimension,
// arithmetic type, delta storage and the (compile-time) brick edge.
#pragma once

#include <type_traits>

#include "device.cuh"

namespace mg {

enum SweepOp { kJacobi = 0, kResidual = 1, kJacobiNorm = 2 };  // kJacobiNorm: Jacobi + sum of r^2

template <typename T>
struct SweepArgs {
  LevelDesc L;
  const T* u;
  const T* b;
  T* out;
  const T* eps;         // cell coefficients (cell slots)
  const void* ahat;     // A_hat planes (3^d per vertex) or nullptr
  const void* ascale;   // per-vertex aux of A_hat: FP32 scales (16-bit codes) or bpa records
  T omega;
  double* partial;      // per-CTA partial sums of r^2 (residual op), nullable
  unsigned* counter;    // completion counter for the fused final sum, nullable
  double* norm2;        // fused final sum of r^2 (written by the last CTA), nullable
  int R;                // slab thickness along the last axis (divides B)
  const T* dinv;        // Jacobi: omega / diag(A) per vertex (setup), nullable
  int block;            // Jacobi of a block step (Sect. 4.2): iota vertices keep their value
  // float-float sweeps of the finest FP64 level (sweep_ff.cuh): the cell coefficients and
  // omega / diag(A) pre-split into (h, l) float pairs, each in a binary64 container (low
  // word h); nullptr: FP64 arithmetic
  const double* eps_pair;
  const double* dinv_pair;
};

// iota vertex of brick slot s (local coordinates; bricks start at multiples of 3): no
// coordinate a multiple of 3, i.e. inside a cell of the next coarser level
template <int DIM>
__device__ __forceinline__ bool iota_local(int s, int B) {
  const int x = s % B, y = (s / B) % B;
  if constexpr (DIM == 2) return x % 3 != 0 && y % 3 != 0;
  return x % 3 != 0 && y % 3 != 0 && (s / (B * B)) % 3 != 0;
}

// Deterministic CTA reduction of one double per thread; thread 0 returns the sum.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double warp_sums[kBlock / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_sums[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) s += warp_sums[w];
  }
  return s;
}

// Stores this CTA's partial sum; the last CTA to finish (counter ticket) adds all
// partials in index order, so the result does not depend on scheduling.
__device__ __forceinline__ void store_partial_and_finish(double v, double* partial, unsigned* counter,
                                                         double* norm2) {
  const unsigned nblocks = gridDim.x * gridDim.y;
  const unsigned bid = blockIdx.x * gridDim.y + blockIdx.y;
  const double s = block_sum(v);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partial[bid] = s;
    last = false;
    if (counter) {
      __threadfence();
      last = atomicAdd(counter, 1u) == nblocks - 1;
    }
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (unsigned i = threadIdx.x; i < nblocks; i += blockDim.x) t += static_cast<volatile double*>(partial)[i];
  const double tot = block_sum(t);
  if (threadIdx.x == 0) {
    norm2[0] = tot;
    *counter = 0u;  // ready for the next launch (graph replays included)
  }
}

// 1/D by Newton-Raphson from an FP32 seed (x_{k+1} = x_k (2 - D x_k), quadratic
// convergence: 2^-22 -> 2^-44 -> 2^-88, i.e. correctly rounded up to the last bit
// or two), cheaper than an FP64 division on GB300's scarce FP64 units.
__device__ __forceinline__ double recip_nr(double D) {
  const double a = fabs(D);
  if (!(a > 1e-30 && a < 1e30)) return 1.0 / D;
  double y = static_cast<double>(__fdividef(1.0f, static_cast<float>(D)));
  double e = fma(-D, y, 1.0);
  y = fma(y, e, y);
  e = fma(-D, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ float recip_nr(float D) { return 1.0f / D; }

// One CTA per (brick, slab of R rows / planes along the last axis).  The slab's
// vertex values with a one-vertex halo and the coefficients of all cells touching
// it are staged in shared memory; each DoF vertex then rebuilds its 3^d stencil
// from the 2^d adjacent cells (element-wise split of Sect. 4, summed per Hamming
// class), adds the stored delta A_hat on coarse levels (Sect. 5), and applies
// either the damped Jacobi update (Alg. 1) or the residual b - A u.
template <int DIM, typename T, int AMODE, int OP, int B>
__device__ __forceinline__ double sweep_item(const SweepArgs<T>& a, int64_t brick, int slab,
                                             unsigned char* smem_raw) {
  constexpr int N3 = cpow(3, DIM);
  constexpr int Bu = B + 2, Be = B + 1;
  constexpr int PLANE = DIM == 2 ? B : B * B;      // vertices per row / plane
  constexpr int UPL = DIM == 2 ? Bu : Bu * Bu;     // tile entries per row / plane (u)
  constexpr int EPL = DIM == 2 ? Be : Be * Be;     // (eps)
  const LevelDesc& L = a.L;
  const int R = a.R;
  const int z0 = slab * R;
  T* su = reinterpret_cast<T*>(smem_raw);
  T* se = su + UPL * (R + 2);
  const int64_t base = brick * L.S;
  __syncthreads();  // the tile may still be read by a previous item of this CTA
  const int32_t* bn = L.brick_nbr + brick * N3;
  const int nt = blockDim.x;

  // interior of the slab: contiguous slots of this brick (vertex values and the
  // coefficients of the cells they own).  A whole brick starts on a 16-byte
  // boundary (slots_per_brick is a multiple of 32), so it is read with 16-byte
  // vector loads; slabs of a split brick use scalar loads.
  const int nin = R * PLANE;
  auto put = [&](int s, T uv, T ev) {
    const int x = s % B;
    const int y = DIM == 2 ? s / B : (s / B) % B;
    const int zl = s / PLANE - z0;
    const int tu = DIM == 2 ? (zl + 1) * Bu + (x + 1) : ((zl + 1) * Bu + (y + 1)) * Bu + (x + 1);
    const int te = DIM == 2 ? (zl + 1) * Be + (x + 1) : ((zl + 1) * Be + (y + 1)) * Be + (x + 1);
    su[tu] = uv;
    se[te] = ev;
  };
  constexpr int VEC = 16 / sizeof(T);
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const bool vec_ok = R == B && ((reinterpret_cast<uintptr_t>(a.u) | reinterpret_cast<uintptr_t>(a.eps)) & 15) == 0;
  if (vec_ok) {
    const V* up = reinterpret_cast<const V*>(a.u + base);
    const V* ep = reinterpret_cast<const V*>(a.eps + base);
    const int nvec = (nin + VEC - 1) / VEC;
#pragma unroll 2
    for (int j = threadIdx.x; j < nvec; j += nt) {
      const V uv = up[j];  // plain loads: coherent with writes of earlier work in the same launch
      const V ev = ep[j];
      const T* uu = reinterpret_cast<const T*>(&uv);
      const T* ee = reinterpret_cast<const T*>(&ev);
#pragma unroll
      for (int c = 0; c < VEC; ++c)
        if (j * VEC + c < nin) put(j * VEC + c, uu[c], ee[c]);
    }
  } else {
    for (int i = threadIdx.x; i < nin; i += nt) put(z0 * PLANE + i, a.u[base + z0 * PLANE + i], a.eps[base + z0 * PLANE + i]);
  }
  // halo vertices (tile positions outside the slab interior)
  auto load_halo = [&](int t, int x, int y, int z) {
    const int ox = x < 0 ? -1 : (x >= B ? 1 : 0);
    const int oy = DIM == 2 ? 0 : (y < 0 ? -1 : (y >= B ? 1 : 0));
    const int oz = z < 0 ? -1 : (z >= B ? 1 : 0);
    const int nidx = DIM == 2 ? (ox + 1) + 3 * (oz + 1) : (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
    const int32_t nb = bn[nidx];
    const int lx = x - ox * B, ly = y - oy * B, lz = z - oz * B;
    const int li = DIM == 2 ? lz * B + lx : (lz * B + ly) * B + lx;
    su[t] = nb >= 0 ? a.u[static_cast<int64_t>(nb) * L.S + li] : T(0);
  };
  if constexpr (DIM == 2) {
    // two halo rows of B + 2 and two halo columns of R
    const int nh = 2 * Bu + 2 * R;
    for (int i = threadIdx.x; i < nh; i += nt) {
      int x, zl;
      if (i < 2 * Bu) {
        x = i % Bu - 1;
        zl = i < Bu ? -1 : R;
      } else {
        const int j = i - 2 * Bu;
        x = j < R ? -1 : B;
        zl = j % R;
      }
      load_halo((zl + 1) * Bu + (x + 1), x, 0, zl + z0);
    }
  } else {
    const int nu = UPL * (R + 2);
    for (int t = threadIdx.x; t < nu; t += nt) {
      const int x = t % Bu - 1;
      const int y = (t / Bu) % Bu - 1;
      const int z = t / UPL - 1 + z0;
      if (x >= 0 && x < B && y >= 0 && y < B && z >= z0 && z < z0 + R) continue;
      load_halo(t, x, y, z);
    }
  }
  // halo cells: local cell coordinate -1 on some axis (x, y, or the slab's z0 - 1)
  const int ne = EPL * (R + 1);
  for (int t = threadIdx.x; t < ne; t += nt) {
    const int x = t % Be - 1;
    const int y = DIM == 2 ? 0 : (t / Be) % Be - 1;
    const int z = t / EPL - 1 + z0;
    if (x >= 0 && (DIM == 2 || y >= 0) && z >= z0) continue;
    const int ox = x < 0 ? -1 : 0;
    const int oy = DIM == 2 ? 0 : (y < 0 ? -1 : 0);
    const int oz = z < 0 ? -1 : 0;
    const int nidx = DIM == 2 ? (ox + 1) + 3 * (oz + 1) : (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1);
    const int32_t nb = bn[nidx];
    const int lx = x - ox * B, ly = y - oy * B, lz = z - oz * B;
    const int li = DIM == 2 ? lz * B + lx : (lz * B + ly) * B + lx;
    se[t] = nb >= 0 ? a.eps[static_cast<int64_t>(nb) * L.S + li] : T(0);
  }
  __syncthreads();
  const T hscale = DIM == 3 ? static_cast<T>(L.h) : T(1);
  double part = 0.0;
  for (int i = threadIdx.x; i < nin; i += nt) {
    const int s = z0 * PLANE + i;
    const int64_t slot = base + s;
    T res = T(0);
    const uint8_t vf = L.vflags[slot];
    const bool keep = OP == kJacobi && a.block && iota_local<DIM>(s, B);
    if constexpr (OP == kJacobi || OP == kJacobiNorm) {
      // hanging vertices keep their value: it is the coarser level's interpolant
      // (Sect. 3, rule 2), refreshed by the composite cycle, not a smoother unknown;
      // so do iota vertices in the Jacobi part of a block step (Sect. 4.2)
      if ((vf & MG_V_HANGING) || keep) res = a.u[slot];
    }
    if (is_dof(vf) && !keep) {
      const int x = s % B;
      const int y = DIM == 2 ? 0 : (s / B) % B;
      const int zl = s / PLANE - z0;
      const int cu = DIM == 2 ? (zl + 1) * Bu + (x + 1) : ((zl + 1) * Bu + (y + 1)) * Bu + (x + 1);
      const int ce = DIM == 2 ? (zl + 1) * Be + (x + 1) : ((zl + 1) * Be + (y + 1)) * Be + (x + 1);
      T off, D;  // off-diagonal part of (A u)_v and the diagonal of A at v
      if constexpr (DIM == 2) {
        // explicit 2D form: cells sw, se, nw, ne; pair sums of the cells shared with
        // each edge neighbour; corners see one cell
        const T e_sw = se[ce - Be - 1], e_se = se[ce - Be], e_nw = se[ce - 1], e_ne = se[ce];
        const T sW = e_sw + e_nw, sE = e_se + e_ne, sS = e_sw + e_se, sN = e_nw + e_ne;
        const T sC = sW + sE;
        const T* uc = su + cu;
        T a1 = sW * uc[-1];
        a1 = fma(sE, uc[1], a1);
        a1 = fma(sS, uc[-Bu], a1);
        a1 = fma(sN, uc[Bu], a1);
        T a2 = e_sw * uc[-Bu - 1];
        a2 = fma(e_se, uc[-Bu + 1], a2);
        a2 = fma(e_nw, uc[Bu - 1], a2);
        a2 = fma(e_ne, uc[Bu + 1], a2);
        const T k0 = static_cast<T>(elem_k(2, 0)), k1 = static_cast<T>(elem_k(2, 1)), k2 = static_cast<T>(elem_k(2, 2));
        D = k0 * sC;
        off = fma(k1, a1, k2 * a2);
      } else {
        T acc[DIM + 1];
#pragma unroll
        for (int c = 0; c <= DIM; ++c) acc[c] = T(0);
        T es_centre = T(0);
#pragma unroll
        for (int k = 0; k < N3; ++k) {
          int o[DIM];
          int ham = 0, kk = k;
#pragma unroll
          for (int q = 0; q < DIM; ++q) {
            o[q] = kk % 3 - 1;
            kk /= 3;
            ham += o[q] != 0;
          }
          if (elem_k(DIM, ham) == 0.0) continue;
          T es = T(0);
#pragma unroll
          for (int e = 0; e < (1 << DIM); ++e) {
            bool ok = true;
            int cidx = ce, m = 1;
#pragma unroll
            for (int q = 0; q < DIM; ++q) {
              const int eq = (e >> q) & 1;
              const int tq = eq + o[q];
              ok = ok && tq >= 0 && tq <= 1;
              cidx -= eq * m;
              m *= Be;
            }
            if (ok) es += se[cidx];
          }
          int uidx = cu, m = 1;
#pragma unroll
          for (int q = 0; q < DIM; ++q) {
            uidx += o[q] * m;
            m *= Bu;
          }
          acc[ham] = fma(es, su[uidx], acc[ham]);
          if (ham == 0) es_centre = es;
        }
        off = T(0);
#pragma unroll
        for (int c = 1; c <= DIM; ++c)
          if (elem_k(DIM, c) != 0.0) off = fma(static_cast<T>(elem_k(DIM, c)), acc[c], off);
        off *= hscale;
        D = static_cast<T>(elem_k(DIM, 0)) * es_centre * hscale;
      }
      const uint64_t akey = AMODE != 0 ? delta_row<AMODE>(a.ascale, slot) : 0;
      if (AMODE != 0 && delta_row_live<AMODE>(akey)) {
#pragma unroll
        for (int k = 0; k < N3; ++k) {
          int uidx = cu, m = 1, kk = k;
#pragma unroll
          for (int q = 0; q < DIM; ++q) {
            uidx += (kk % 3 - 1) * m;
            kk /= 3;
            m *= Bu;
          }
          const T d = load_delta<AMODE, T>(a.ahat, a.ascale, (brick * N3 + k) * L.S + s, slot, k, akey,
                                           a_lo_off<AMODE>(L, N3));
          if (k == N3 / 2)
            D += d;
          else
            off = fma(d, su[uidx], off);
        }
      }
      const T uv = su[cu];
      if (OP == kJacobi && a.dinv) {
        // u + omega (b - D u - off) / D = (1 - omega) u + (omega / D) (b - off), with
        // omega / D from the setup: no division here (FP64 units are the bound)
        res = fma(a.dinv[slot], a.b[slot] - off, (T(1) - a.omega) * uv);
      } else {
        const T r = a.b[slot] - fma(D, uv, off);
        if constexpr (OP == kJacobi || OP == kJacobiNorm) {
          res = fma(a.omega * r, recip_nr(D), uv);
          if constexpr (OP == kJacobiNorm) part += static_cast<double>(r) * static_cast<double>(r);
        } else {
          res = r;
          part += static_cast<double>(r) * static_cast<double>(r);
        }
      }
    }
    a.out[slot] = res;
  }
  return part;
}

// Gauss-Seidel sweeps of a block Jacobi step (Sect. 4.2): one thread per 3^d patch (a
// cell of the next coarser level; (B/3)^d of them per brick).  The thread loads the
// 4^d vertex values and 3^d cell coefficients of its patch into registers, then
// updates the 2^d iota vertices x = c + (1 or 2)^d in lexicographic order,
// u_v += (b_v - (A u)_v) / A_vv with the current values, `sweeps` times, and writes
// them back.  Patches share no iota vertex and no iota vertex neighbours another
// patch's, so the in-place updates of different threads never meet.
template <int DIM, typename T, int AMODE>
__global__ void __launch_bounds__(DIM == 2 ? 256 : 64) k_patch_gs(SweepArgs<T> a, int sweeps) {
  constexpr int N3 = cpow(3, DIM), N4 = cpow(4, DIM), NI = 1 << DIM;
  const LevelDesc& L = a.L;
  const int pb = L.B / 3;  // patches per brick axis
  const int pp = DIM == 2 ? pb * pb : pb * pb * pb;
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= static_cast<int64_t>(L.n_bricks) * pp) return;
  const int64_t brick = t / pp;
  int p = static_cast<int>(t - brick * pp);
  int cl[DIM];  // brick-local corner of the patch (a multiple of 3, at most B - 3)
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    cl[i] = 3 * (p % pb);
    p /= pb;
  }
  // slot of corner + d, d in {0..3}^d: the same brick, or for a local coordinate of B
  // the next brick along that axis (brick neighbour table, -1 beyond the domain)
  const int32_t* bn = L.brick_nbr + brick * N3;
  auto slot_at = [&](const int* d) -> int64_t {
    int bidx = 0, m3 = 1;
    int64_t li = 0, mb = 1;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      int l = cl[i] + d[i];
      const int o = l >= L.B ? 1 : 0;
      l -= o * L.B;
      bidx += (o + 1) * m3;
      m3 *= 3;
      li += l * mb;
      mb *= L.B;
    }
    const int32_t nb = bn[bidx];
    return nb < 0 ? -1 : static_cast<int64_t>(nb) * L.S + li;
  };
  T* u = a.out;  // the iterate, updated in place (a.u aliases it)
  T ul[N4];      // vertex values at corner + {0..3}^d
  T el[N3];      // cell coefficients of the patch's cells corner + {0..2}^d
#pragma unroll
  for (int q = 0; q < N4; ++q) {
    int d[DIM], qq = q;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      d[i] = qq % 4;
      qq /= 4;
    }
    const int64_t w = slot_at(d);
    ul[q] = w >= 0 ? u[w] : T(0);
  }
#pragma unroll
  for (int q = 0; q < N3; ++q) {
    int d[DIM], qq = q;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      d[i] = qq % 3;
      qq /= 3;
    }
    el[q] = a.eps[slot_at(d)];  // inside the patch's own brick
  }
  int64_t vs[NI];
  T bv[NI];
#pragma unroll
  for (int j = 0; j < NI; ++j) {
    int d[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) d[i] = 1 + ((j >> i) & 1);
    const int64_t v = slot_at(d);
    vs[j] = (v >= 0 && is_dof(L.vflags[v])) ? v : -1;
    bv[j] = vs[j] >= 0 ? a.b[v] : T(0);
  }
  const T scale = DIM == 3 ? static_cast<T>(L.h) : T(1);
  for (int sw = 0; sw < sweeps; ++sw) {
#pragma unroll
    for (int j = 0; j < NI; ++j) {
      if (vs[j] < 0) continue;
      int q[DIM];  // local position of the vertex, in {1,2}^d
#pragma unroll
      for (int i = 0; i < DIM; ++i) q[i] = 1 + ((j >> i) & 1);
      const uint64_t key = AMODE != 0 ? delta_row<AMODE>(a.ascale, vs[j]) : 0;
      T au = T(0), diag = T(0);
#pragma unroll
      for (int k = 0; k < N3; ++k) {
        int o[DIM], kk = k, ham = 0, un = 0, m4 = 1;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          o[i] = kk % 3 - 1;
          kk /= 3;
          ham += o[i] != 0;
          un += (q[i] + o[i]) * m4;
          m4 *= 4;
        }
        T es = T(0);  // cells holding both the vertex and its neighbour x + o
#pragma unroll
        for (int e = 0; e < NI; ++e) {
          bool ok = true;
          int cl = 0, m3 = 1;
#pragma unroll
          for (int i = 0; i < DIM; ++i) {
            const int ei = (e >> i) & 1;
            ok = ok && ei + o[i] >= 0 && ei + o[i] <= 1;
            cl += (q[i] - ei) * m3;
            m3 *= 3;
          }
          if (ok) es += el[cl];
        }
        T st = static_cast<T>(elem_k(DIM, ham)) * es * scale;
        if constexpr (AMODE != 0)
          st += load_delta<AMODE, T>(a.ahat, a.ascale, plane_index(L, vs[j], k, N3), vs[j], k, key,
                                     a_lo_off<AMODE>(L, N3));
        if (k == N3 / 2) diag = st;
        au = fma(st, ul[un], au);
      }
      int ui = 0, m4 = 1;
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        ui += q[i] * m4;
        m4 *= 4;
      }
      ul[ui] += (bv[j] - au) / diag;
    }
  }
#pragma unroll
  for (int j = 0; j < NI; ++j) {
    if (vs[j] < 0) continue;
    int ui = 0, m4 = 1;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      ui += (1 + ((j >> i) & 1)) * m4;
      m4 *= 4;
    }
    u[vs[j]] = ul[ui];
  }
}

template <int DIM, typename T, int AMODE, int OP, int B>
__global__ void __launch_bounds__(kBlock) k_sweep(SweepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_enter();
  const double part = sweep_item<DIM, T, AMODE, OP, B>(a, blockIdx.x, blockIdx.y, smem_raw);
  if constexpr (OP == kResidual) {
    if (a.partial) store_partial_and_finish(part, a.partial, a.counter, a.norm2);
  }
}

// CTAs along x of a sweep launch (times B / R slabs along y): one brick per CTA
template <typename T>
inline int64_t sweep_ctas_x(int, int, T, int64_t n_bricks) {
  return n_bricks;
}

// slab depth R (a divisor of B) of a sweep launch: enough CTAs to fill the GPU
template <typename T>
inline int sweep_slab(int, int B, int64_t n_bricks) {
  int R = B;
  while (R > 1 && n_bricks * (B / R) < 4 * 152) R /= 3;
  return R;
}

// shared memory of one sweep item: the u tile with its halo and the cell
// coefficients (cell_sums: the 3D column kernel also keeps per-cell corner sums)
template <int DIM, typename T>
inline size_t sweep_tile_bytes(int B, int R, bool cell_sums = false) {
  const size_t upl = DIM == 2 ? B + 2 : (B + 2) * (B + 2);
  const size_t epl = DIM == 2 ? B + 1 : (B + 1) * (B + 1);
  return (upl * (R + 2) + epl * (R + 1) * (cell_sums ? 2 : 1)) * sizeof(T);
}

// slot of integer position x on a level with compile-time brick edge B
template <int DIM, int B>
__device__ __forceinline__ int64_t slot_of_b(const LevelDesc& L, const int* x) {
  int64_t ri = 0, li = 0;
#pragma unroll
  for (int i = DIM - 1; i >= 0; --i) {
    if (x[i] < 0 || x[i] >= L.n) return -1;
    ri = ri * L.nb_axis + x[i] / B;
    li = li * B + x[i] % B;
  }
  const int32_t rank = L.brick_rank[ri];
  return rank < 0 ? -1 : static_cast<int64_t>(rank) * L.S + li;
}

template <int DIM, int B>
__device__ __forceinline__ bool coords_of_b(const LevelDesc& L, int64_t slot, int* x) {
  constexpr int VOL = DIM == 2 ? B * B : B * B * B;
  const int64_t b = slot / L.S;
  int k = static_cast<int>(slot - b * L.S);
  if (k >= VOL) return false;
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    x[i] = L.brick_roots[b * DIM + i] * B + k % B;
    k /= B;
  }
  return true;
}

// b_c(V) = sum_o P(V,o) r_f(3V + o): restriction with R = P^T (Sect. 4.4).
// One thread per coarse slot; zero on non-DoF coarse slots.  The 5^d loop is fully
// unrolled so the d-linear weights are compile-time constants.
template <int DIM, typename T, int PMODE, int BC, int BF>
__device__ __forceinline__ void restrict_one(const LevelDesc& Lc, const LevelDesc& Lf, const T* rf, T* bc,
                                             const void* phat, const void* pscale, int64_t cs) {
  constexpr int N5 = cpow(5, DIM);
  int X[DIM];
  if (!coords_of_b<DIM, BC>(Lc, cs, X) || !is_dof(Lc.vflags[cs])) {
    bc[cs] = T(0);
    return;
  }
  const int64_t cb = cs / Lc.S, cl = cs - cb * Lc.S;
  const uint64_t pkey = PMODE != 0 ? delta_row<PMODE>(pscale, cs) : 0;
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < N5; ++k) {
    int o[DIM], y[DIM];
    int kk = k;
    double w = 1.0;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      o[i] = kk % 5 - 2;
      kk /= 5;
      y[i] = 3 * X[i] + o[i];
      w *= wlin1(o[i]);
    }
    const int64_t fs = slot_of_b<DIM, BF>(Lf, y);
    if (fs < 0) continue;
    T p = static_cast<T>(w);
    if constexpr (PMODE != 0) p += load_delta<PMODE, T>(phat, pscale, (cb * N5 + k) * Lc.S + cl, cs, k, pkey);
    acc = fma(p, rf[fs], acc);
  }
  bc[cs] = acc;
}

// d-linear weight of 5^d offset index k (offset o_i = digit_i(k) - 2), prod (3 - |o_i|) / 3
template <int DIM, typename T>
__device__ __forceinline__ T dlin_weight(int k) {
  double w = 1.0;
  for (int i = 0; i < DIM; ++i) {
    w *= wlin1(k % 5 - 2);
    k /= 5;
  }
  return static_cast<T>(w);
}

// Restriction kernel: the 5^d taps of a coarse vertex are split over kRestrictWarps
// warps.  Lane i of every warp serves coarse slot 32*blockIdx + i (so P_hat planes
// and fine values are read coalesced across a warp), warp j sums taps j, j + 8, ...,
// and the warps' partial sums are added in warp order (deterministic).  With a slot
// list (composite grid: the refined coarse DoFs) lane i serves list[32*blockIdx + i]
// and other coarse slots are not written.  zero_c (nullable): a coarse vector set to
// zero at every slot served (the coarse correction's initial guess), so the cycle
// needs no separate memset.
constexpr int kRestrictWarps = 8;

template <int DIM, typename T, int PMODE, int BC, int BF>
__global__ void __launch_bounds__(32 * kRestrictWarps)
    k_restrict(LevelDesc Lc, LevelDesc Lf, const T* rf, T* bc, const void* phat, const void* pscale,
               const int32_t* list, int64_t n_list, T* zero_c) {
  constexpr int N5 = cpow(5, DIM);
  __shared__ T part[kRestrictWarps][32];
  __shared__ T wtab[N5];  // d-linear weights by tap, formed once per CTA (FP64 units are scarce)
  for (int k = threadIdx.x; k < N5; k += blockDim.x) wtab[k] = dlin_weight<DIM, T>(k);
  __syncthreads();
  pdl_enter();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = blockIdx.x * 32LL + lane;
  const int64_t cs = list ? (i < n_list ? list[i] : -1) : (i < Lc.n_slots ? i : -1);
  int X[DIM];
  const bool dof = cs >= 0 && coords_of_b<DIM, BC>(Lc, cs, X) && is_dof(Lc.vflags[cs]);
  T acc = T(0);
  if (dof) {
    const int64_t cb = cs / Lc.S, cl = cs - cb * Lc.S;
    const uint64_t pkey = PMODE != 0 ? delta_row<PMODE>(pscale, cs) : 0;
    for (int k = warp; k < N5; k += kRestrictWarps) {
      int y[DIM];
      int kk = k;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        y[a] = 3 * X[a] + kk % 5 - 2;
        kk /= 5;
      }
      const int64_t fs = slot_of_b<DIM, BF>(Lf, y);
      if (fs < 0) continue;
      T p = wtab[k];
      if constexpr (PMODE != 0)
        p += load_delta<PMODE, T>(phat, pscale, (cb * N5 + k) * Lc.S + cl, cs, k, pkey);
      acc = fma(p, rf[fs], acc);
    }
  }
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && cs >= 0) {
    T t = part[0][lane];
#pragma unroll
    for (int j = 1; j < kRestrictWarps; ++j) t += part[j][lane];
    bc[cs] = dof ? t : T(0);
    if (zero_c) zero_c[cs] = T(0);
  }
}

// u_f(v) += sum over coarse parents V of P(V, v - 3V) e_c(V) (coarse-grid
// correction of Alg. 1).  One thread per fine slot; non-DoF slots untouched.
template <int DIM, typename T, int PMODE, int BC, int BF>
__device__ __forceinline__ void prolong_one(const LevelDesc& Lc, const LevelDesc& Lf, const T* ec, T* uf,
                                            const void* phat, const void* pscale, int64_t fs,
                                            const T* wtab = nullptr) {
  constexpr int N5 = cpow(5, DIM);
  int x[DIM];
  if (!coords_of_b<DIM, BF>(Lf, fs, x) || !is_dof(Lf.vflags[fs])) return;
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
    int k = 0, m = 1;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      const int ei = (e >> i) & 1;
      if (ei >= cnt[i]) ok = false;
      X[i] = lo[i] + ei;
      o[i] = x[i] - 3 * X[i];
      k += (o[i] + 2) * m;
      m *= 5;
    }
    if (!ok) continue;
    const int64_t cs = slot_of_b<DIM, BC>(Lc, X);
    if (cs < 0 || !is_dof(Lc.vflags[cs])) continue;
    T p = wtab ? wtab[k] : dlin_weight<DIM, T>(k);
    if constexpr (PMODE != 0) {
      const int64_t cb = cs / Lc.S;
      p += load_delta<PMODE, T>(phat, pscale, (cb * N5 + k) * Lc.S + (cs - cb * Lc.S), cs, k,
                                delta_row<PMODE>(pscale, cs));
    }
    acc = fma(p, ec[cs], acc);
  }
  uf[fs] += acc;
}

// (list: fine DoF slots to serve, thread i -> list[i]; nullptr: every fine slot)
template <int DIM, typename T, int PMODE, int BC, int BF>
__global__ void __launch_bounds__(kBlock) k_prolong(LevelDesc Lc, LevelDesc Lf, const T* ec, T* uf,
                                                      const void* phat, const void* pscale,
                                                      const int32_t* list, int64_t n_list) {
  constexpr int N5 = cpow(5, DIM);
  __shared__ T wtab[N5];  // d-linear weights by offset, formed once per CTA
  for (int k = threadIdx.x; k < N5; k += blockDim.x) wtab[k] = dlin_weight<DIM, T>(k);
  __syncthreads();
  pdl_enter();
  const int64_t i = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  if (list) {
    if (i < n_list) prolong_one<DIM, T, PMODE, BC, BF>(Lc, Lf, ec, uf, phat, pscale, list[i], wtab);
  } else if (i < Lf.n_slots) {
    prolong_one<DIM, T, PMODE, BC, BF>(Lc, Lf, ec, uf, phat, pscale, i, wtab);
  }
}

// u_f on HANGING slots = d-linear interpolant of the coarser level (Sect. 3, rule 2)
// (list: the hanging slots, thread i -> list[i]; nullptr: every slot, flag-checked)
template <int DIM, typename T>
__global__ void __launch_bounds__(kBlock) k_hanging(LevelDesc Lf, const int32_t* hang_idx, const double* hang_w,
                                                      const T* uc, T* uf, const int32_t* list, int64_t n_list) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(kBlock) + threadIdx.x;
  int64_t fs;
  if (list) {
    if (i >= n_list) return;
    fs = list[i];
  } else {
    if (i >= Lf.n_slots || !(Lf.vflags[i] & MG_V_HANGING)) return;
    fs = i;
  }
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

// ---- host-side launchers (instantiated per dimension / type in k2d_*.cu, k3d_*.cu) ----

// slab thickness: the largest divisor R of B giving at least `target` CTAs (or 1)
inline int pick_slab(int B, int64_t n_bricks, int64_t target) {
  int R = B;
  while (R > 1 && n_bricks * (B / R) < target) R /= 3;
  return R;
}

template <int DIM, typename T>
void launch_sweep(SweepArgs<T> a, int op, int amode, cudaStream_t s);

// two damped Jacobi sweeps a.u -> a.out in one launch (sweep_pair.cuh): 2D FP32 levels
// of brick edge 27 or 9; amode 0, 2 or 3
void launch_sweep_pair_2d_f32(SweepArgs<float> a, int amode, cudaStream_t s);
// the same for FP64 hierarchies (coarse levels: amode 0 or 1, omega / diag(A) in a.dinv)
void launch_sweep_pair_2d_f64(SweepArgs<double> a, int amode, cudaStream_t s);

// Gauss-Seidel part of a block Jacobi step (Sect. 4.2) on a.u in place
template <int DIM, typename T>
void launch_patch_gs(SweepArgs<T> a, int amode, int sweeps, cudaStream_t s);

// list / n_list: the coarse (restriction) or fine (prolongation) slots to serve;
// nullptr serves every slot of the target level
template <int DIM, typename T>
void launch_transfer(const LevelDesc& Lc, const LevelDesc& Lf, bool restrict_op, int pmode, const T* in, T* out,
                     const void* phat, const void* pscale, cudaStream_t s, const int32_t* list = nullptr,
                     int64_t n_list = 0, T* zero_c = nullptr);

}  // namespace mg
