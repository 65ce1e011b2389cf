// Host-side launchers of the numeric column kernels, one translation unit per
// value type so they compile in parallel.
#pragma once

#include "column.cuh"

// Launches the numeric pass for size bucket `bucket` over `count` listed
// columns (count known on the host).  The work counter in `a` must be zero.
cudaError_t launch_columns_f64(int bucket, int alg, const ColArgs& a, int count, cudaStream_t s);
cudaError_t launch_columns_c128(int bucket, int alg, const ColArgs& a, int count, cudaStream_t s);

// Shared launch helper: persistent grid sized by occupancy, the per-warp
// shared memory of WarpLayout.
template <class S, int KMAX, int MMAX, int ALG>
cudaError_t launch_warp_columns(const ColArgs& a, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  auto kern = column_warp_kernel<S, KMAX, MMAX, ALG>;
  const size_t per_warp = WarpLayout<S, KMAX, MMAX>::bytes();
  int wpb = (int)((96 * 1024) / per_warp);
  wpb = wpb < 1 ? 1 : (wpb > 8 ? 8 : wpb);
  const size_t smem = per_warp * wpb;
  static bool configured = false;  // one attribute call per instantiation and process
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
  if (per_sm < 1) per_sm = 1;
  int grid = ceil_div(count, wpb);
  if (grid > sms * per_sm) grid = sms * per_sm;
  kern<<<grid, wpb * 32, smem, s>>>(a);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}
