// Encoder of the bpa byte codec of the hierarchical deltas (Sect. 5): per vertex and
// operator the smallest bpa in {0, 2, ..., 8} whose f_bpa = m 2^e keeps every entry
// within eps_mf, then one byte stream per operator kind and level.  The decoder is
// bpa_decode in device.cuh.  Three launches: choose bpa per vertex, exclusive scan of
// the sizes bpa * K into records (offset << 4 | bpa), write the bytes.
#pragma once

#include "device.cuh"

namespace mg {

__device__ __forceinline__ double pow2d(int i) {  // 2^i for i in [-1022, 1023], exact
  return __longlong_as_double(static_cast<long long>(i + 1023) << 52);
}

// (e, |m|) of one entry at bpa >= 2 and its error | |m| 2^e - |x| | (the FP64 expression
// of the tolerance test); false if the exponent does not fit a signed byte.  The
// exponent is the smallest whose |m| = rint(|x| 2^-e) fits M = 8 (bpa - 1) - 1 bits,
// clamped below at -128.  Every scaling is by an exact power of two.
__device__ __forceinline__ bool bpa_entry(double x, int bpa, int* e_out, uint64_t* m_out, double* err) {
  const double a = fabs(x);
  if (a == 0.0) {
    *e_out = 0;
    *m_out = 0;
    *err = 0.0;
    return true;
  }
  const int M = 8 * (bpa - 1) - 1;
  int E;
  frexp(a, &E);  // a = f 2^E, f in [0.5, 1)
  int e = E - M;
  uint64_t m;
  if (e < -128) {
    // clamped exponent (a rounding carry from e = -129 lands on the same value)
    e = -128;
    m = static_cast<uint64_t>(rint(a * pow2d(64) * pow2d(64)));
  } else {
    m = static_cast<uint64_t>(rint(a * pow2d(-e)));
    if (m == (1ull << M)) {  // rounding carried into the next power of two
      m >>= 1;
      ++e;
    }
  }
  if (e > 127) return false;
  *e_out = e;
  *m_out = m;
  *err = fabs(__ull2double_rn(m) * pow2d(e) - a);
  return true;
}

// entries of operator `row` (K of them): rows layout x[row * K + k] or a level's planes
struct BpaSrc {
  const double* x;
  int K;
  bool planes;
  LevelDesc L;  // planes only
  __device__ __forceinline__ double at(int64_t row, int k) const {
    return planes ? x[plane_index(L, row, k, K)] : x[row * K + k];
  }
};

// One thread per entry: the entry's smallest bpa (0 if |x| <= eps_mf, else the first of
// 2..8 whose error is within eps_mf), merged into rec[row] (zeroed before) by atomicMax.
// The error of an entry never grows with bpa (the finer grid of m 2^e contains the
// coarser one, and FP64 rounding of the difference is monotone), so the row's smallest
// admissible bpa is the largest of its entries' smallest ones.
// *status <- code_nonfinite for a non-finite entry, code_unrep for an entry no bpa can store
__global__ void k_bpa_choose(BpaSrc src, int64_t n, double eps_mf, uint64_t* rec, int* status, int code_nonfinite,
                             int code_unrep) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= n * src.K) return;
  const int64_t row = t / src.K;
  const int k = static_cast<int>(t - row * src.K);
  const double v = src.at(row, k);
  if (!isfinite(v)) {
    if (status) atomicExch(status, code_nonfinite);
    return;
  }
  if (fabs(v) <= eps_mf) return;
  for (int b = 2; b <= 8; ++b) {
    int e;
    uint64_t m;
    double err;
    if (bpa_entry(v, b, &e, &m, &err) && err <= eps_mf) {
      atomicMax(reinterpret_cast<unsigned long long*>(rec + row), static_cast<unsigned long long>(b));
      return;
    }
  }
  if (status) atomicExch(status, code_unrep);
}

// one CTA: rec[i] (= bpa) -> (exclusive prefix of bpa * K) << 4 | bpa; *total = bytes
constexpr int kScanThreads = 1024, kScanItems = 4;
__global__ void __launch_bounds__(kScanThreads) k_bpa_scan(int64_t n, int K, uint64_t* rec, uint64_t* total) {
  __shared__ uint64_t wsum[32];
  __shared__ uint64_t carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += kScanThreads * kScanItems) {
    const int64_t i0 = base + static_cast<int64_t>(threadIdx.x) * kScanItems;
    uint64_t b[kScanItems], sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      b[j] = i0 + j < n ? rec[i0 + j] : 0;
      sum += b[j] * static_cast<uint64_t>(K);
    }
    uint64_t x = sum;  // inclusive scan over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      uint64_t t = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      wsum[lane] = t;
    }
    __syncthreads();
    uint64_t off = carry + (w > 0 ? wsum[w - 1] : 0) + x - sum;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      if (i0 + j < n) rec[i0 + j] = (off << 4) | b[j];
      off += b[j] * static_cast<uint64_t>(K);
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// one thread per entry: its bpa bytes at the row's offset + k * bpa
__global__ void k_bpa_write(BpaSrc src, int64_t n, const uint64_t* rec, uint8_t* bytes) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= n * src.K) return;
  const int64_t row = t / src.K;
  const int k = static_cast<int>(t - row * src.K);
  const uint64_t r = rec[row];
  const int bpa = static_cast<int>(r & 15u);
  if (bpa == 0) return;
  uint8_t* p = bytes + (r >> 4) + static_cast<int64_t>(k) * bpa;
  const double v = src.at(row, k);
  int e = 0;
  uint64_t m = 0;
  double err;
  if (!isfinite(v) || !bpa_entry(v, bpa, &e, &m, &err)) e = 0, m = 0;  // flagged in k_bpa_choose
  const int M = 8 * (bpa - 1) - 1;
  const uint64_t word = m | (static_cast<uint64_t>(v < 0.0) << M);
  p[0] = static_cast<uint8_t>(static_cast<int8_t>(e));
  for (int j = 1; j < bpa; ++j) p[j] = static_cast<uint8_t>(word >> (8 * (j - 1)));
}

template <typename T>
__global__ void k_bpa_decode(int64_t n, int K, const uint64_t* rec, const uint8_t* bytes, T* out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < K; ++k) out[i * K + k] = bpa_decode<T>(bytes, rec[i], k);
}

// enqueue the three encode launches; bytes must hold n * K * 8 (the worst case)
inline void bpa_encode_enqueue(const BpaSrc& src, int64_t n, double eps_mf, uint64_t* rec, uint8_t* bytes,
                               uint64_t* total, int* status, int code_nonfinite, int code_unrep, cudaStream_t s) {
  if (n <= 0) {
    cudaMemsetAsync(total, 0, sizeof(uint64_t), s);
    return;
  }
  const unsigned g = static_cast<unsigned>((n * src.K + 255) / 256);
  cudaMemsetAsync(rec, 0, static_cast<size_t>(n) * sizeof(uint64_t), s);
  k_bpa_choose<<<g, 256, 0, s>>>(src, n, eps_mf, rec, status, code_nonfinite, code_unrep);
  k_bpa_scan<<<1, kScanThreads, 0, s>>>(n, src.K, rec, total);
  k_bpa_write<<<g, 256, 0, s>>>(src, n, rec, bytes);
}

}  // namespace mg
