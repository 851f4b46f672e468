// Galerkin coarse operator A_c = P^T A P in 3D in two stages (Sect. 4.3), so that every
// fine stencil and every product A(f, g) P(g, W) is formed once:
//   stage 1 (k_rap3_ap, per fine vertex f):  AP(f, W) = sum_g A(f, g) P(g, W)
//   stage 2 (k_rap3_pt, per coarse vertex V): A_c(V, W) = sum_f P(f, V) AP(f, W)
// and A_hat(V, W) = A_c(V, W) - A_redisc(V, W) as in k_rap.  The single-kernel form
// recomputes every fine stencil and product for each of the ~4.6 coarse vertices whose
// prolongation support holds the fine vertex (~71,000 FP64 instructions per coarse
// vertex); here a coarse vertex costs 27 x (~91 stencil + 250 product) + 1,331 + 125.
//
// AP lives in a scratch array in a class-major compact layout.  A fine vertex f = 3 V_f + d
// (V_f the nearest coarse vertex, d in {-1, 0, 1}^3) reaches the coarse vertices
// W = V_f + o with |d_i - 3 o_i| <= 3 per axis: o_i in {-1, 0, 1} for d_i = 0, {0, 1}
// for d_i = 1, {-1, 0} for d_i = -1.  Fine vertices of one class c = (x mod 3) +
// 3 (y mod 3) + 9 (z mod 3) (local brick coordinates; bricks start at multiples of 9)
// share d and so their count cnt[c] = prod_i n_i of entries; per class, per fine brick
// b, per position p of the class in the brick (27), the cnt[c] entries follow in o order
// (x fastest).  A warp of stage 1 covers fine vertices of one class (identical loop trip
// counts, no divergence) and writes consecutive entries.
#pragma once

#include "device.cuh"

namespace mg {

constexpr int kApPerBrick = 343 * 27;  // sum over classes of cnt[c] (= 7^3) x 27 positions
// stage-1 threads run group by group: the 27 classes of kApGroup consecutive fine bricks
// (Peano order) in consecutive CTAs, so the coarse P and the fine coefficients they read
// stay in L2 while every class passes over them (class by class over the whole level,
// each of the 27 passes re-read the coarse level's P from DRAM)
constexpr int kApGroup = 32;
__host__ __device__ constexpr int64_t ap_threads(int64_t n_bricks) {
  return (n_bricks + kApGroup - 1) / kApGroup * (27 * 27 * kApGroup);
}

// per-axis admissible coarse offsets of a fine vertex with local coordinate x (mod 3)
__host__ __device__ constexpr int ap_nofs(int xm3) { return xm3 == 0 ? 3 : 2; }
__host__ __device__ constexpr int ap_omin(int xm3) { return xm3 == 1 ? 0 : -1; }
__host__ __device__ constexpr int ap_d(int xm3) { return xm3 == 0 ? 0 : (xm3 == 1 ? 1 : -1); }

// entries of the classes before class c, per brick position
__host__ __device__ constexpr int ap_class_prefix(int c) {
  int s = 0;
  for (int k = 0; k < c; ++k) s += ap_nofs(k % 3) * ap_nofs((k / 3) % 3) * ap_nofs(k / 9);
  return s;
}

// stage 1: one thread per (class, fine brick, position); the fine level has brick edge 9
template <int PMODE>
__global__ void __launch_bounds__(128) k_rap3_ap(LevelDesc Lc, LevelDesc Lf, const double* eps_f,
                                                  const double* ahat_f, const double* phat_c, double* ap,
                                                  const double* aniso_f) {
  constexpr int N3 = 27, N5 = 125;
  __shared__ double plin[N5];
  __shared__ double sst[128][N3];  // this thread's fine stencil (zero towards non-DoFs)
  for (int k = threadIdx.x; k < N5; k += blockDim.x)
    plin[k] = wlin1(k % 5 - 2) * wlin1((k / 5) % 5 - 2) * wlin1(k / 25 - 2);
  const int64_t per_class = Lf.n_bricks * 27;
  const int64_t gid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  // gid -> (group, class, (brick, position) within the group); a warp covers 32
  // consecutive (brick, position) pairs of one class (27 kApGroup is a multiple of 32)
  constexpr int64_t kGsz = 27 * kApGroup;
  const int64_t grp = gid / (27 * kGsz);
  const int64_t rem = gid - grp * (27 * kGsz);
  const int cg = static_cast<int>(rem / kGsz);
  const int64_t rg = grp * kGsz + (rem - cg * kGsz);
  const bool live = rg < per_class;
  const int c = live ? cg : 0;
  const int64_t r = live ? rg : 0;
  const int64_t b = r / 27;
  const int p = static_cast<int>(r - b * 27);
  const int cm[3] = {c % 3, (c / 3) % 3, c / 9};
  const int lx[3] = {3 * (p % 3) + cm[0], 3 * ((p / 3) % 3) + cm[1], 3 * (p / 9) + cm[2]};
  const int n_o[3] = {ap_nofs(cm[0]), ap_nofs(cm[1]), ap_nofs(cm[2])};
  const int cnt = n_o[0] * n_o[1] * n_o[2];
  double* out = ap + (Lf.n_bricks * 27) * ap_class_prefix(c) + r * cnt;
  int f[3], d[3], Vf[3];
  bool fdof = false;
  int64_t fs = -1;
  if (live) {
    fs = b * Lf.S + (lx[2] * 9 + lx[1]) * 9 + lx[0];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      f[i] = Lf.brick_roots[b * 3 + i] * 9 + lx[i];
      d[i] = ap_d(cm[i]);
      Vf[i] = (f[i] - d[i]) / 3;
    }
    fdof = f[0] < Lf.n && f[1] < Lf.n && f[2] < Lf.n && is_dof(Lf.vflags[fs]);
  }
  double* st = sst[threadIdx.x];
  if (fdof) {
    double s[N3];
    full_stencil<3>(Lf, eps_f, ahat_f, f, fs, s, aniso_f);
#pragma unroll
    for (int e = 0; e < N3; ++e) {
      const int g[3] = {f[0] + e % 3 - 1, f[1] + (e / 3) % 3 - 1, f[2] + e / 9 - 1};
      const int64_t gs = slot_of<3>(Lf, g);
      st[e] = (gs >= 0 && is_dof(Lf.vflags[gs])) ? s[e] : 0.0;
    }
  }
  __syncthreads();
  if (!live) return;
  for (int j = 0; j < cnt; ++j) {
    const int o[3] = {ap_omin(cm[0]) + j % n_o[0], ap_omin(cm[1]) + (j / n_o[0]) % n_o[1],
                      ap_omin(cm[2]) + j / (n_o[0] * n_o[1])};
    double acc = 0.0;
    if (fdof) {
      const int W[3] = {Vf[0] + o[0], Vf[1] + o[1], Vf[2] + o[2]};
      const int64_t ws = slot_of<3>(Lc, W);
      if (ws >= 0 && is_dof(Lc.vflags[ws])) {
        // eps per axis with |d + eps - 3 o| <= 2; P(g, W) at offset g - 3W = d + eps - 3 o
        int lo[3], hi[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          lo[i] = max(-1, 3 * o[i] - 2 - d[i]);
          hi[i] = min(1, 3 * o[i] + 2 - d[i]);
        }
        const int64_t pb = PMODE == 1 ? plane_index(Lc, ws, 0, N5) : 0;
        for (int ez = lo[2]; ez <= hi[2]; ++ez)
          for (int ey = lo[1]; ey <= hi[1]; ++ey)
            for (int ex = lo[0]; ex <= hi[0]; ++ex) {
              const int e = (ex + 1) + 3 * (ey + 1) + 9 * (ez + 1);
              const int k = (d[0] + ex - 3 * o[0] + 2) + 5 * (d[1] + ey - 3 * o[1] + 2) +
                            25 * (d[2] + ez - 3 * o[2] + 2);
              acc = fma(st[e], plin[k], acc);
              if constexpr (PMODE == 1) acc = fma(st[e], phat_c[pb + static_cast<int64_t>(k) * Lc.S], acc);
            }
      }
    }
    out[j] = acc;  // zero for non-DoF f or W: stage 2 reads every entry it may need
  }
}

// stage 2: a CTA of 27 warps over 32 consecutive coarse slots; warp w handles the coarse
// neighbour offset o' = (w mod 3 - 1, (w / 3) mod 3 - 1, w / 9 - 1) of all 32, lane = slot
constexpr int kRapPtSlots = 32;
constexpr size_t rap3_pt_smem() { return (sizeof(double) + sizeof(int64_t)) * kRapPtSlots * 125; }

__device__ __forceinline__ double redisc_entry3(const LevelDesc& L, const double* eps, const int* V, const int* o) {
  double es = 0.0;
  int ham = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) ham += o[i] != 0;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    bool ok = true;
    int c[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int t = ((e >> i) & 1) + o[i];
      ok = ok && t >= 0 && t <= 1;
      c[i] = V[i] - ((e >> i) & 1);
    }
    if (!ok) continue;
    const int64_t cs = slot_of<3>(L, c);
    if (cs >= 0) es += eps[cs];
  }
  return (elem_k(3, ham) * L.h) * es;  // as full_stencil
}

template <int PMODE>
__global__ void __launch_bounds__(27 * 32) k_rap3_pt(LevelDesc Lc, LevelDesc Lf, const double* eps_c,
                                                      const double* phat_c, const double* ap, double* ahat_c) {
  constexpr int N5 = 125;
  // dynamic shared memory (rap3_pt_smem bytes): P(f, V) at f = 3V + d (zero where f is no
  // DoF), and the AP index of (f, W = V) with its strides along o'_y, o'_z in bits 48..63
  extern __shared__ __align__(16) unsigned char smem_pt[];
  auto sP = reinterpret_cast<double(*)[N5]>(smem_pt);
  auto sE = reinterpret_cast<int64_t(*)[N5]>(smem_pt + sizeof(double) * kRapPtSlots * N5);
  const int64_t cs0 = blockIdx.x * static_cast<int64_t>(kRapPtSlots);
  const int64_t per_class = Lf.n_bricks * 27;
  for (int idx = threadIdx.x; idx < kRapPtSlots * N5; idx += blockDim.x) {
    const int v = idx / N5, k = idx % N5;
    const int64_t cs = cs0 + v;
    double P = 0.0;
    int64_t E = 0;
    int V[3];
    if (cs < Lc.n_slots && coords_of<3>(Lc, cs, V) && is_dof(Lc.vflags[cs])) {
      const int dd[3] = {k % 5 - 2, (k / 5) % 5 - 2, k / 25 - 2};
      const int f[3] = {3 * V[0] + dd[0], 3 * V[1] + dd[1], 3 * V[2] + dd[2]};
      const int64_t fs = slot_of<3>(Lf, f);
      if (fs >= 0 && is_dof(Lf.vflags[fs])) {
        P = p_entry_d<3, PMODE>(Lc, phat_c, cs, dd);
        const int64_t b = fs / Lf.S;
        const int loc = static_cast<int>(fs - b * Lf.S);
        const int lx[3] = {loc % 9, (loc / 9) % 9, loc / 81};
        const int cm[3] = {lx[0] % 3, lx[1] % 3, lx[2] % 3};
        const int c = cm[0] + 3 * cm[1] + 9 * cm[2];
        const int p = lx[0] / 3 + 3 * (lx[1] / 3) + 9 * (lx[2] / 3);
        const int n_o[3] = {ap_nofs(cm[0]), ap_nofs(cm[1]), ap_nofs(cm[2])};
        // o' = 0 is o = -delta relative to f's nearest coarse vertex (delta_i = +-1 where
        // |d_i| = 2): entry index j_i = -delta_i - o_min
        int j0[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) j0[i] = -((dd[i] >= 2) - (dd[i] <= -2)) - ap_omin(cm[i]);
        E = per_class * ap_class_prefix(c) + (b * 27 + p) * (n_o[0] * n_o[1] * n_o[2]) +
            (j0[2] * n_o[1] + j0[1]) * n_o[0] + j0[0];
        E |= (static_cast<int64_t>(n_o[0]) << 48) | (static_cast<int64_t>(n_o[0] * n_o[1]) << 56);
      }
    }
    sP[v][k] = P;
    sE[v][k] = E;
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, v = threadIdx.x & 31;
  const int op[3] = {w % 3 - 1, (w / 3) % 3 - 1, w / 9 - 1};
  const int64_t cs = cs0 + v;
  int V[3];
  if (cs >= Lc.n_slots || !coords_of<3>(Lc, cs, V)) return;
  double out = 0.0;
  const int W[3] = {V[0] + op[0], V[1] + op[1], V[2] + op[2]};
  const int64_t ws = slot_of<3>(Lc, W);
  if (is_dof(Lc.vflags[cs]) && ws >= 0 && is_dof(Lc.vflags[ws])) {
    // fine offsets d with |d_i - 3 o'_i| <= 3 (5 values for o'_i = 0, 3 otherwise)
    int lo[3], hi[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      lo[i] = max(-2, 3 * op[i] - 3);
      hi[i] = min(2, 3 * op[i] + 3);
    }
    double acc = 0.0;
    for (int dz = lo[2]; dz <= hi[2]; ++dz)
      for (int dy = lo[1]; dy <= hi[1]; ++dy)
        for (int dx = lo[0]; dx <= hi[0]; ++dx) {
          const int k = (dx + 2) + 5 * (dy + 2) + 25 * (dz + 2);
          const double P = sP[v][k];
          if (P != 0.0) {
            const int64_t E = sE[v][k];
            const int sy = static_cast<int>((E >> 48) & 0xff), sz = static_cast<int>(E >> 56);
            acc = fma(P, ap[(E & 0xffffffffffffll) + op[2] * sz + op[1] * sy + op[0]], acc);
          }
        }
    out = acc - redisc_entry3(Lc, eps_c, V, op);
  }
  ahat_c[plane_index(Lc, cs, w, 27)] = out;
}

}  // namespace mg
