// Persistent batch step, 3D (see batch_persist.cuh).
#include "batch_persist.cuh"

namespace mg {

template <>
cudaError_t bpersist_launch<3>(const QueueArgs& q, int amc64, int pm64, int amc32, int pm32, cudaStream_t s) {
  const size_t smem = bpersist_smem<3>();
  auto launch = [&](auto kernel) {
    // one wave of resident CTAs: they take the queue's entries until it is empty
    static int ctas = 0;
    if (ctas == 0) {
      int dev = 0, sms = 0, per_sm = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, smem);
      ctas = sms * (per_sm > 0 ? per_sm : 1);
    }
    kernel<<<ctas, 128, smem, s>>>(q);
    return cudaGetLastError();
  };
  if (amc64 == 1 && pm64 == 1 && amc32 == 2 && pm32 == 2) return launch(k_bpersist<3, 1, 1, 2, 2>);
  if (amc64 == 0 && pm64 == 0 && amc32 == 0 && pm32 == 0) return launch(k_bpersist<3, 0, 0, 0, 0>);
  return cudaErrorNotSupported;
}

}  // namespace mg
