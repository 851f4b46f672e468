// Device-side level descriptors, stencil rebuild and delta decoding shared by the
// libmg CUDA translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "../../include/mg.h"

namespace mg {

constexpr int kBlock = 256;  // threads per CTA of the brick kernels

// Everything a kernel needs to address one level (passed by value).
struct LevelDesc {
  int dim, level, n, B, S, nb_axis;
  int64_t n_bricks, n_slots;
  double h;
  const int32_t* brick_nbr;    // n_bricks * 3^d
  const int32_t* brick_roots;  // n_bricks * d
  const int32_t* brick_rank;   // nb_axis^d
  const uint8_t* vflags;       // n_slots
};

__host__ __device__ constexpr int cpow(int b, int e) { return e == 0 ? 1 : b * cpow(b, e - 1); }

// Programmatic dependent launch: the kernels of a cycle are launched with programmatic
// stream serialization (launch_pdl), so the launch of a kernel is processed while its
// predecessor still runs and its CTAs start as soon as the predecessor's CTAs exit;
// pdl_enter makes each wait for the predecessor's results.  No kernel signals its
// dependents early (griddepcontrol.launch_dependents): CTAs of the next kernel that
// become resident early and wait beside a running FP64-bound sweep slowed it (2D level 6:
// a residual sweep 33 -> 22 us, an FP64 V-cycle 250 -> 231 us without the early signal).
// Without the launch attribute the wait is a no-op.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// FEM element matrix of -div(eps grad u) for d-linear elements on a unit cube, by
// Hamming distance of the two corners (Sect. 4): 2D 2/3, -1/6, -1/3; 3D 1/3, 0,
// -1/12, -1/12 (times h in 3D, applied by the caller).
__host__ __device__ constexpr double elem_k(int dim, int ham) {
  return dim == 2 ? (ham == 0 ? 2.0 / 3.0 : ham == 1 ? -1.0 / 6.0 : -1.0 / 3.0)
                  : (ham == 0 ? 1.0 / 3.0 : ham == 1 ? 0.0 : -1.0 / 12.0);
}

// d-linear interpolation weight (coarsening by three) at fine offset o in [-2,2]
__host__ __device__ constexpr double wlin1(int o) { return o == 0 ? 1.0 : (o == 1 || o == -1) ? 2.0 / 3.0 : 1.0 / 3.0; }

__device__ __forceinline__ bool is_dof(uint8_t f) {
  return (f & MG_V_EXISTS) && !(f & (MG_V_BOUNDARY | MG_V_HANGING));
}

template <int DIM>
__device__ __forceinline__ int brick_vol(int B) {
  return DIM == 2 ? B * B : B * B * B;
}

// slot of integer position x on level L, -1 outside [0,n)^d or without a brick
template <int DIM>
__device__ __forceinline__ int64_t slot_of(const LevelDesc& L, const int* x) {
  int64_t ri = 0, li = 0;
#pragma unroll
  for (int i = DIM - 1; i >= 0; --i) {
    if (x[i] < 0 || x[i] >= L.n) return -1;
    ri = ri * L.nb_axis + x[i] / L.B;
    li = li * L.B + x[i] % L.B;
  }
  const int32_t rank = L.brick_rank[ri];
  return rank < 0 ? -1 : static_cast<int64_t>(rank) * L.S + li;
}

// global coordinates of a slot; false on padding slots
template <int DIM>
__device__ __forceinline__ bool coords_of(const LevelDesc& L, int64_t slot, int* x) {
  const int64_t b = slot / L.S;
  int k = static_cast<int>(slot - b * L.S);
  if (k >= brick_vol<DIM>(L.B)) return false;
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    x[i] = L.brick_roots[b * DIM + i] * L.B + k % L.B;
    k /= L.B;
  }
  return true;
}

// index of plane k of a per-vertex multi-entry array (brick-major planes)
__device__ __forceinline__ int64_t plane_index(const LevelDesc& L, int64_t slot, int k, int K) {
  const int64_t b = slot / L.S;
  return (b * K + k) * L.S + (slot - b * L.S);
}

// ---- delta storage ---------------------------------------------------------
// DMODE 0: none, 1: FP64 values, 2: BF16 codes x FP32 scale, 3: FP16 codes x FP32 scale,
// 4: the bpa byte codec
__device__ __forceinline__ float bf16_bits_to_float(uint16_t q) {
  return __uint_as_float(static_cast<uint32_t>(q) << 16);
}
__device__ __forceinline__ float fp16_bits_to_float(uint16_t q) {
  __half_raw hr;
  hr.x = q;
  return __half2float(__half(hr));
}

// bpa codec (Sect. 5): an operator of a vertex is either dropped (bpa = 0) or stored
// entry by entry as bpa bytes: a signed exponent byte e, then bpa - 1 bytes of m
// little-endian, whose top bit is the sign and whose other M = 8 (bpa - 1) - 1 bits
// hold |m|; the value is (-1)^sign |m| 2^e.  rec = (byte offset << 4) | bpa locates the
// operator in its byte stream; entry k sits k * bpa bytes further.  The FP32 value is
// |m| rounded once to FP32 then scaled by 2^e (exact scaling), i.e. the FP32 rounding of
// the stored value wherever that is a normal number.
template <typename T>
__device__ __forceinline__ T bpa_decode(const uint8_t* bytes, uint64_t rec, int k) {
  const int bpa = static_cast<int>(rec & 15u);
  if (bpa == 0) return T(0);
  // the entry's bpa bytes from the (one or two) aligned 8-byte words holding them; the
  // stream is 8-byte aligned and its buffer a multiple of 8 bytes, so both words exist
  const uint64_t at = (rec >> 4) + static_cast<uint64_t>(k) * bpa;
  const uint64_t* w = reinterpret_cast<const uint64_t*>(bytes) + (at >> 3);
  const int sh = static_cast<int>(at & 7u) * 8;
  uint64_t v = w[0] >> sh;
  if (sh + 8 * bpa > 64) v |= w[1] << (64 - sh);
  const int e = static_cast<int>(static_cast<int8_t>(v & 0xffu));
  const uint64_t word = v >> 8;
  const int M = 8 * (bpa - 1) - 1;
  const uint64_t m = word & ((1ull << M) - 1ull);
  // 2^e built from its bit pattern (e in [-128, 127]: normal in FP64; in FP32 normal down
  // to -126, and 2^-127, 2^-128 are FP32 subnormals), so the product is the one rounding
  T x;
  if constexpr (std::is_same<T, double>::value) {
    x = __ull2double_rn(m) * __longlong_as_double(static_cast<long long>(e + 1023) << 52);
  } else {
    const float p2 = e >= -126 ? __int_as_float((e + 127) << 23) : __int_as_float(0x00400000 >> (-127 - e));
    x = __fmul_rn(__ull2float_rn(m), p2);
  }
  return ((word >> M) & 1u) ? -x : x;
}

// per-vertex key of a delta row: the bpa record (DMODE 4; a zero bpa marks a dropped
// operator whose entries all read as zero), the bit pattern of the FP32 scale (DMODE 2,
// 3: its sign bit is the promotion flag), else a non-zero constant
template <int DMODE>
__device__ __forceinline__ uint64_t delta_row(const void* aux, int64_t slot) {
  if constexpr (DMODE == 4) return static_cast<const uint64_t*>(aux)[slot];
  else if constexpr (DMODE == 2 || DMODE == 3) return __float_as_uint(static_cast<const float*>(aux)[slot]);
  else return 1;
}
template <int DMODE>
__device__ __forceinline__ bool delta_row_live(uint64_t key) {
  return DMODE != 4 || (key & 15u) != 0;
}

// delta entry k of the vertex in slot `slot`; idx = its position in the 16-bit or FP64
// planes; key = the vertex's delta_row.  DMODE 2, 3: the scale comes from the key.
// lo_off (DMODE 2, 3; 0 = no promotion): distance from the code planes to the planes of
// the low halves.  A promoted vertex (the sign bit of its scale set: its 16-bit codes
// could not reconstruct its diagonal, Sect. 5 cancellation) stores the FP32 bit pattern
// of delta / s as (code << 16 | low half); the value is then that FP32 number times |s|.
// DMODE 4 decodes from the stream p with the vertex's record.
template <int DMODE, typename T>
__device__ __forceinline__ T load_delta(const void* p, const void* aux, int64_t idx, int64_t slot, int k = 0,
                                        uint64_t key = 0, int64_t lo_off = 0) {
  if constexpr (DMODE == 1) {
    return static_cast<T>(static_cast<const double*>(p)[idx]);
  } else if constexpr (DMODE == 2 || DMODE == 3) {
    const float s = __uint_as_float(static_cast<uint32_t>(key));
    const uint16_t* q = static_cast<const uint16_t*>(p);
    if (lo_off != 0 && s < 0.0f)
      return static_cast<T>(__uint_as_float((static_cast<uint32_t>(q[idx]) << 16) | q[idx + lo_off]) * -s);
    return static_cast<T>((DMODE == 2 ? bf16_bits_to_float(q[idx]) : fp16_bits_to_float(q[idx])) * s);
  } else if constexpr (DMODE == 4) {
    return bpa_decode<T>(static_cast<const uint8_t*>(p), key, k);
  } else {
    return T(0);
  }
}

// distance to the low-half planes of A_hat codes on level L (16-bit modes; 0 otherwise)
template <int DMODE>
__device__ __forceinline__ int64_t a_lo_off(const LevelDesc& L, int K) {
  return (DMODE == 2 || DMODE == 3) ? L.n_slots * K : 0;
}

// P(V, o) = P_dlin(o) + P_hat_V(o) in FP64 (PMODE 0: d-linear only, 1: FP64 delta planes)
template <int DIM, int PMODE>
__device__ __forceinline__ double p_entry_d(const LevelDesc& Lc, const double* phat, int64_t cs, const int* o) {
  double w = 1.0;
  int k = 0, m = 1;
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    w *= wlin1(o[i]);
    k += (o[i] + 2) * m;
    m *= 5;
  }
  if constexpr (PMODE == 1) w += phat[plane_index(Lc, cs, k, cpow(5, DIM))];
  return w;
}

// ---- full stencil at an arbitrary vertex (setup kernels) -------------------
// st[k], k over offsets {-1,0,1}^d lexicographic (x fastest): rediscretised from
// the adjacent existing cells' eps (cell slot = lower-left vertex slot), plus the
// stored FP64 delta when ahat != nullptr.
// Anisotropy of a diagonal-tensor coefficient eps = diag(eps_i) (Sect. 7 `checkerboard`):
// with the per-cell mean e = mean_i eps_i and d_i = eps_i - e, the d-linear element
// matrix is e K + sum_i d_i K_i (K_i = int d_i phi_a d_i phi_b), and since sum_i d_i = 0
// the second term is, per pair of corners, 2D: -d_x / 2 for corners differing in x only,
// +d_x / 2 for those differing in y only, 0 otherwise; 3D (times h): -d_i / 6 for corners
// differing in axis i only, +d_k / 12 for corners differing in the two axes other than
// k, 0 otherwise (nothing on the diagonal).  Returned: the entry of one cell with per-axis
// deviations dv for neighbour offset o (o in {-1, 0, 1}^d, o != 0, inside the cell).
template <int DIM>
__device__ __forceinline__ double aniso_entry(const double* dv, const int* o, double h) {
  int nz = 0, k0 = -1, z = -1;
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    if (o[i] != 0) {
      ++nz;
      k0 = i;
    } else {
      z = i;
    }
  }
  if constexpr (DIM == 2) return nz == 1 ? (k0 == 0 ? -0.5 * dv[0] : 0.5 * dv[0]) : 0.0;
  if (nz == 1) return -h * dv[k0] / 6.0;
  if (nz == 2) return h * dv[z] / 12.0;
  return 0.0;
}

// aniso (nullable): per-axis deviations d_i of a diagonal-tensor coefficient on this level,
// axis-major (aniso[i * n_slots + cell slot]); eps then holds the per-cell mean.
template <int DIM>
__device__ void full_stencil(const LevelDesc& L, const double* eps, const double* ahat, const int* x,
                             int64_t slot, double* st, const double* aniso = nullptr) {
  constexpr int N3 = cpow(3, DIM);
  double ec[1 << DIM];
#pragma unroll
  for (int e = 0; e < (1 << DIM); ++e) {
    int c[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) c[i] = x[i] - ((e >> i) & 1);
    const int64_t cs = slot_of<DIM>(L, c);
    ec[e] = cs >= 0 ? eps[cs] : 0.0;
  }
  const double scale = DIM == 3 ? L.h : 1.0;
#pragma unroll
  for (int k = 0; k < N3; ++k) {
    int o[DIM];
    int ham = 0;
    int kk = k;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      o[i] = kk % 3 - 1;
      kk /= 3;
      ham += o[i] != 0;
    }
    // (elem_k scale) es: one multiply per entry; the 3D face entries have elem_k = 0
    // (trilinear element) and are exact zeros
    double es = 0.0;
    if (elem_k(DIM, ham) != 0.0) {
#pragma unroll
      for (int e = 0; e < (1 << DIM); ++e) {
        bool ok = true;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          const int t = ((e >> i) & 1) + o[i];
          ok = ok && t >= 0 && t <= 1;
        }
        if (ok) es += ec[e];
      }
    }
    st[k] = (elem_k(DIM, ham) * scale) * es;
    if (ahat && slot >= 0) st[k] += ahat[plane_index(L, slot, k, N3)];
    if (aniso && ham > 0) {
#pragma unroll
      for (int e = 0; e < (1 << DIM); ++e) {
        bool ok = true;
        int c[DIM];
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          const int t = ((e >> i) & 1) + o[i];
          ok = ok && t >= 0 && t <= 1;
          c[i] = x[i] - ((e >> i) & 1);
        }
        if (!ok) continue;
        const int64_t cs = slot_of<DIM>(L, c);
        if (cs < 0) continue;
        double dv[DIM];
#pragma unroll
        for (int i = 0; i < DIM; ++i) dv[i] = aniso[i * L.n_slots + cs];
        st[k] += aniso_entry<DIM>(dv, o, L.h);
      }
    }
  }
}

}  // namespace mg
