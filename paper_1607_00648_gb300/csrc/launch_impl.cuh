// Host launchers of the hot-path kernels, instantiated per (dimension, type) in
// k2d_f64.cu, k2d_f32.cu, k3d_f64.cu, k3d_f32.cu so they compile in parallel.
#pragma once

#include <type_traits>

#include "kernels.cuh"
#include "sweep_fast.cuh"
#include "sweep_ff.cuh"

namespace mg {

template <int DIM, typename T, int B>
static void sweep_b(SweepArgs<T> a, int op, int amode, cudaStream_t s) {
  constexpr int PLANE = DIM == 2 ? B : B * B;
  const int R = a.R;
  const size_t smem = sweep_tile_bytes<DIM, T>(B, R);
  if constexpr (std::is_same<T, float>::value && ((DIM == 2 && B == 27) || (DIM == 3 && B == 9))) {
    // FP32 (issue- and latency-bound): column-marching kernels with the slab depth
    // as a template parameter so every plane's loads are issued together
    const dim3 grid(static_cast<unsigned>(sweep_ctas_x(DIM, B, T(0), a.L.n_bricks)), static_cast<unsigned>(B / R));
    const size_t sm = DIM == 2 ? 0 : sweep_tile_bytes<DIM, T>(B, R, true);
    // 2D: the 16-byte-staged column-marching kernel where the level's vectors exceed L2
    // (2D level 7 and finer: 2.64 -> 3.84 TB/s on level 7); on L2-resident levels the
    // row-interleaved kernel is faster (its warps are independent: 4.9 against 8.8 us on
    // level 6).  16-byte staging needs u and eps 16-byte aligned (user vectors may be
    // offset views).
    const bool v16 = a.L.n_bricks >= 2048 &&
                     ((reinterpret_cast<uintptr_t>(a.u) | reinterpret_cast<uintptr_t>(a.eps)) & 15) == 0;
#define MG_SWR(AM, OP, RR)                                                                \
  do {                                                                                    \
    if constexpr (DIM == 2) {                                                             \
      if (v16) launch_pdl(k_sweep2v<AM, OP, RR>, grid, RR >= 3 ? 96 : 32, 0, s, a);        \
      else launch_pdl(k_sweep2c<T, AM, OP, RR>, grid, 128, 0, s, a);                      \
    } else {                                                                              \
      launch_pdl(k_sweep3c<T, AM, OP, (RR > 9 ? 9 : RR)>, grid, 128, sm, s, a);           \
    }                                                                                     \
  } while (0)
#define MG_SW(AM, OP)                                                    \
  do {                                                                   \
    if (R == 1) MG_SWR(AM, OP, 1);                                       \
    else if (R == 3) MG_SWR(AM, OP, 3);                                  \
    else if (R == 9) MG_SWR(AM, OP, 9);                                  \
    else MG_SWR(AM, OP, 27);                                             \
  } while (0)
    if (op == kJacobi) {
      if (amode == 2) MG_SW(2, kJacobi); else if (amode == 3) MG_SW(3, kJacobi);
      else if (amode == 4) MG_SW(4, kJacobi); else MG_SW(0, kJacobi);
    } else {
      if (amode == 2) MG_SW(2, kResidual); else if (amode == 3) MG_SW(3, kResidual);
      else if (amode == 4) MG_SW(4, kResidual); else MG_SW(0, kResidual);
    }
#undef MG_SW
#undef MG_SWR
  } else if (std::is_same<T, double>::value && ((DIM == 2 && B == 27) || (DIM == 3 && B == 9)) &&
             (op == kResidual || a.dinv != nullptr)) {
    // FP64 (FP64-unit bound): column-marching kernels that issue the fewest FP64
    // instructions per vertex; Jacobi takes omega / diag(A) from the setup
    if constexpr (std::is_same<T, double>::value && ((DIM == 2 && B == 27) || (DIM == 3 && B == 9))) {
      const dim3 grid(static_cast<unsigned>(a.L.n_bricks), static_cast<unsigned>(B / R));
      // float-float arithmetic on the finest level when the setup split its coefficients
      const bool ff = a.eps_pair != nullptr && amode == 0 && !a.block;
#define MG_SWR(AM, OP, RR)                                                                                  \
  do {                                                                                                      \
    if constexpr (DIM == 2) {                                                                               \
      if (AM == 0 && ff) launch_pdl(k_sweep2x<OP, RR>, grid, RR >= 3 ? 96 : 32, 0, s, a);                   \
      else launch_pdl(k_sweep2f<AM, OP, RR>, grid, RR >= 3 ? 96 : 32, 0, s, a);                             \
    } else if (AM == 0 && ff) {                                                                             \
      launch_pdl(k_sweep3x<OP, (RR > 9 ? 9 : RR)>, grid, 128, sweep_tile_bytes<DIM, T>(B, RR > 9 ? 9 : RR, true), s, a); \
    } else {                                                                                                \
      launch_pdl(k_sweep3c<T, AM, OP, (RR > 9 ? 9 : RR)>, grid, 128, sweep_tile_bytes<DIM, T>(B, RR > 9 ? 9 : RR, true), s, a); \
    }                                                                                                       \
  } while (0)
#define MG_SW(AM, OP)                                                    \
  do {                                                                   \
    if (R == 1) MG_SWR(AM, OP, 1);                                       \
    else if (R == 3) MG_SWR(AM, OP, 3);                                  \
    else if (R == 9) MG_SWR(AM, OP, 9);                                  \
    else MG_SWR(AM, OP, 27);                                             \
  } while (0)
      if (op == kJacobi) {
        if (amode == 1) MG_SW(1, kJacobi); else MG_SW(0, kJacobi);
      } else if (op == kJacobiNorm) {  // finest levels (no stored deltas) of the FP64 solve
        MG_SW(0, kJacobiNorm);
      } else {
        if (amode == 1) MG_SW(1, kResidual); else MG_SW(0, kResidual);
      }
#undef MG_SW
#undef MG_SWR
    }
  } else {
    const dim3 grid(static_cast<unsigned>(a.L.n_bricks), static_cast<unsigned>(B / R));
    int threads = ((R * PLANE + 31) / 32) * 32;
    if (threads > kBlock) threads = kBlock;
#define MG_SW(AM, OP) launch_pdl(k_sweep<DIM, T, AM, OP, B>, grid, threads, smem, s, a)
    if constexpr (std::is_same<T, double>::value) {
      if (op == kJacobi) {
        if (amode == 1) MG_SW(1, kJacobi); else MG_SW(0, kJacobi);
      } else {
        if (amode == 1) MG_SW(1, kResidual); else MG_SW(0, kResidual);
      }
    } else {
      if (op == kJacobi) {
        if (amode == 2) MG_SW(2, kJacobi); else if (amode == 3) MG_SW(3, kJacobi);
        else if (amode == 4) MG_SW(4, kJacobi); else MG_SW(0, kJacobi);
      } else {
        if (amode == 2) MG_SW(2, kResidual); else if (amode == 3) MG_SW(3, kResidual);
        else if (amode == 4) MG_SW(4, kResidual); else MG_SW(0, kResidual);
      }
    }
#undef MG_SW
  }
}

template <int DIM, typename T, int BC, int BF>
static void transfer_b(const LevelDesc& Lc, const LevelDesc& Lf, bool restrict_op, int pmode, const T* in, T* out,
                       const void* ph, const void* ps, cudaStream_t s, const int32_t* li, int64_t nl,
                       T* zc) {
  const int64_t nc = li ? nl : Lc.n_slots, nf = li ? nl : Lf.n_slots;
  const unsigned gc = static_cast<unsigned>((nc + 31) / 32);
  const unsigned gf = static_cast<unsigned>((nf + kBlock - 1) / kBlock);
  if ((restrict_op ? gc : gf) == 0) return;
#define MG_TR(PM)                                                                                   \
  do {                                                                                              \
    if (restrict_op)                                                                                \
      launch_pdl(k_restrict<DIM, T, PM, BC, BF>, gc, 32 * kRestrictWarps, 0, s, Lc, Lf, in, out, ph, ps, li, nl, zc); \
    else                                                                                            \
      launch_pdl(k_prolong<DIM, T, PM, BC, BF>, gf, kBlock, 0, s, Lc, Lf, in, out, ph, ps, li, nl);   \
  } while (0)
  if constexpr (std::is_same<T, double>::value) {
    if (pmode == 1) MG_TR(1); else MG_TR(0);
  } else {
    if (pmode == 2) MG_TR(2); else if (pmode == 3) MG_TR(3); else if (pmode == 4) MG_TR(4); else MG_TR(0);
  }
#undef MG_TR
}

template <int DIM, typename T>
static void patch_gs_b(SweepArgs<T> a, int amode, int sweeps, cudaStream_t s) {
  const int64_t pb = a.L.B / 3, pp = DIM == 2 ? pb * pb : pb * pb * pb;  // patches per brick
  constexpr int nt = DIM == 2 ? 256 : 64;
  const unsigned g = static_cast<unsigned>((a.L.n_bricks * pp + nt - 1) / nt);
  if (g == 0 || sweeps <= 0) return;
  if constexpr (std::is_same<T, double>::value) {
    if (amode == 1) k_patch_gs<DIM, T, 1><<<g, nt, 0, s>>>(a, sweeps);
    else k_patch_gs<DIM, T, 0><<<g, nt, 0, s>>>(a, sweeps);
  } else {
    if (amode == 2) k_patch_gs<DIM, T, 2><<<g, nt, 0, s>>>(a, sweeps);
    else if (amode == 3) k_patch_gs<DIM, T, 3><<<g, nt, 0, s>>>(a, sweeps);
    else if (amode == 4) k_patch_gs<DIM, T, 4><<<g, nt, 0, s>>>(a, sweeps);
    else k_patch_gs<DIM, T, 0><<<g, nt, 0, s>>>(a, sweeps);
  }
}

}  // namespace mg

#define MG_INSTANTIATE_LAUNCHERS(DIM, T)                                                                    \
  namespace mg {                                                                                            \
  template <>                                                                                               \
  void launch_sweep<DIM, T>(SweepArgs<T> a, int op, int amode, cudaStream_t s) {                             \
    switch (a.L.B) {                                                                                        \
      case 3: sweep_b<DIM, T, 3>(a, op, amode, s); break;                                                   \
      case 9: sweep_b<DIM, T, 9>(a, op, amode, s); break;                                                   \
      default: MG_SWEEP_27(DIM, T) break;                                                                   \
    }                                                                                                       \
  }                                                                                                         \
  template <>                                                                                               \
  void launch_patch_gs<DIM, T>(SweepArgs<T> a, int amode, int sweeps, cudaStream_t s) {                     \
    patch_gs_b<DIM, T>(a, amode, sweeps, s);                                                                \
  }                                                                                                         \
  template <>                                                                                               \
  void launch_transfer<DIM, T>(const LevelDesc& Lc, const LevelDesc& Lf, bool r, int pmode, const T* in,     \
                               T* out, const void* ph, const void* ps, cudaStream_t s, const int32_t* li,  \
                               int64_t nl, T* zc) {                                                         \
    if (Lc.B == 3 && Lf.B == 9) transfer_b<DIM, T, 3, 9>(Lc, Lf, r, pmode, in, out, ph, ps, s, li, nl, zc);  \
    else if (Lc.B == 9 && Lf.B == 9) transfer_b<DIM, T, 9, 9>(Lc, Lf, r, pmode, in, out, ph, ps, s, li, nl, zc); \
    else MG_TRANSFER_27(DIM, T)                                                                             \
  }                                                                                                         \
  }
