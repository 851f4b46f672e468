// FP64 FMA-rate probe: the denominator of the FP64 roofline of the sweep kernels.
// Every thread runs kChains independent chains of dependent fmas x <- x * a + c, so
// that enough fmas are in flight to keep the FP64 units busy; the chains' sum is
// written out so that no chain can be removed.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace mg {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_fma_chains_f64(int iters, double a, double c, double* sink) {
  double x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == 12345.678) sink[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}

}  // namespace mg

extern "C" mg_status mg_probe_fp64_fma(int64_t n_ctas, int32_t iters, double* sink, int64_t* flops, void* stream) {
  if (n_ctas < 1 || n_ctas > (1LL << 24) || iters < 1 || !sink || !flops) {
    mg::set_error("mg_probe_fp64_fma: n_ctas in 1..2^24, iters >= 1, sink and flops non-NULL");
    return MG_ERR_INVALID_ARG;
  }
  mg::k_fma_chains_f64<<<static_cast<unsigned>(n_ctas), mg::kProbeThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      iters, 1.0 - 1e-9, 1e-9, sink);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mg::set_error(std::string("mg_probe_fp64_fma: ") + cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  *flops = 2LL * mg::kChains * iters * mg::kProbeThreads * n_ctas;
  return MG_OK;
}
