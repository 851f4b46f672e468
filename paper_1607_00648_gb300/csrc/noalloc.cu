// Residual with its squared norm, for callers that must not allocate device memory.
//
// mg_residual keeps the per-CTA partial sums of the norm reduction in workspace
// that mg_hier_create allocated on the device.  This variant keeps them in a
// fixed file-scope device array instead, so a call performs no allocation of any
// kind and does not synchronise: the squared norm is written to a device double
// the caller provides.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "hier.h"
#include "kernels.cuh"

namespace mg {
namespace {

// One partial sum per CTA of the residual sweep (a brick, or a slab of a brick on
// small levels): 4096 entries (32 KiB) cover every level up to 2D level 6 and 3D
// level 4 (729 bricks each; smaller levels are split into at most 912 slabs).
constexpr int64_t kMaxBricks = 4096;
static __device__ __align__(256) double g_partials[kMaxBricks];

// Host code cannot use g_partials' name as a device address: it is a host-side
// stand-in.  The device address is looked up once per device with that device
// current and cached here.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_partials_dev[kMaxDevices] = {};

mg_status partials_on_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_error(std::string("mg_residual_norm_noalloc: no usable current device: ") + cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_partials_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess || !p) {
      set_error(std::string("mg_residual_norm_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return MG_ERR_CUDA;
    }
    g_partials_dev[dev] = static_cast<double*>(p);
  }
  *out = g_partials_dev[dev];
  return MG_OK;
}

__global__ void __launch_bounds__(kBlock) k_sum_partials(const double* partial, int64_t n, double* out) {
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kBlock) v += partial[i];
  __shared__ double warp_sums[kBlock / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) s += warp_sums[w];
    out[0] = s;
  }
}

constexpr int64_t kSweepTargetCtas = 4 * 152;

// launches the residual sweep with its per-CTA partial sums in `partial`; returns
// the number of partial sums written
int64_t launch_residual(const Hier& H, const DevLevel& D, bool coarse_delta, const double* u, const double* b,
                        double* r, double* partial, cudaStream_t s) {
  SweepArgs<double> a{};
  a.L = D.d;
  a.u = u;
  a.b = b;
  a.out = r;
  a.eps = D.eps;
  a.ahat = coarse_delta ? D.ahat : nullptr;
  a.partial = partial;
  // the default slab rule, not a depth chosen by mg_autotune: a tuned depth can need
  // more partial sums than the fixed array holds
  a.R = pick_slab(D.d.B, D.d.n_bricks, kSweepTargetCtas);
  if (H.dim == 2)
    launch_sweep<2, double>(a, kResidual, coarse_delta ? 1 : 0, s);
  else
    launch_sweep<3, double>(a, kResidual, coarse_delta ? 1 : 0, s);
  return sweep_ctas_x(H.dim, D.d.B, 0.0, D.d.n_bricks) * (D.d.B / a.R);
}

}  // namespace
}  // namespace mg

using namespace mg;

extern "C" mg_status mg_residual_norm_noalloc(mg_hier* h, int level, const double* u, const double* b, double* r,
                                              double* norm2, void* stream) {
  Hier* H = reinterpret_cast<Hier*>(h);
  if (!H || !H->ready) {
    set_error("mg_residual_norm_noalloc: NULL or not set-up hierarchy");
    return MG_ERR_INVALID_ARG;
  }
  if (level < H->c || level > H->L || !u || !b || !r || !norm2) {
    set_error("mg_residual_norm_noalloc: invalid level or NULL vector");
    return MG_ERR_INVALID_ARG;
  }
  if (H->tensor && level == H->L) {
    set_error("mg_residual_norm_noalloc: the finest level of a tensor-coefficient hierarchy; use mg_residual");
    return MG_ERR_UNSUPPORTED;
  }
  const DevLevel& D = H->lv[level];
  if (D.d.n_bricks > kMaxBricks) {
    set_error("mg_residual_norm_noalloc: level has " + std::to_string(D.d.n_bricks) +
              " bricks, more than the 4096 this allocation-free variant supports; use mg_residual");
    return MG_ERR_INVALID_ARG;
  }
  double* partial = nullptr;
  const mg_status st = partials_on_current_device(&partial);
  if (st != MG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool coarse_delta = level < H->top && H->galerkin;
  if (sweep_ctas_x(H->dim, D.d.B, 0.0, D.d.n_bricks) * (D.d.B / pick_slab(D.d.B, D.d.n_bricks, kSweepTargetCtas)) >
      kMaxBricks) {
    set_error("mg_residual_norm_noalloc: level needs more than 4096 partial sums; use mg_residual");
    return MG_ERR_INVALID_ARG;
  }
  const int64_t nparts = launch_residual(*H, D, coarse_delta, u, b, r, partial, s);
  k_sum_partials<<<1, kBlock, 0, s>>>(partial, nparts, norm2);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("mg_residual_norm_noalloc: launch failed: ") + cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  return MG_OK;
}
