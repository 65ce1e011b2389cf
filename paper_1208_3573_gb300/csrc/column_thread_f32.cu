// One thread per column: the mixed-precision DIAF-S kernel for small real tiles.
#include "column_thread.cuh"
#include "launch.cuh"

namespace {
size_t g_thread_smem_configured = 0;
}

cudaError_t thread_columns_shape(int M, int K, int count_hint, ThreadShape* out) {
  *out = ThreadShape{};
  if (count_hint <= 0) return cudaSuccess;
  if (M < 1 || K < 1 || M > kThreadMMax || K > kThreadKMax) return cudaErrorInvalidValue;
  auto kern = column_thread_kernel<kThreadKMax>;
  const size_t smem = sizeof(float) * (size_t)thread_arena_floats(M, K) / 4 * 32 * kQuadWarps;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (g_thread_smem_configured < smem) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    g_thread_smem_configured = smem;
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kQuadWarps, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidValue;
  int grid = sms * per_sm;
  const int need = ceil_div(count_hint, kQuadCols * kQuadWarps);
  if (grid > need) grid = need;
  out->grid = grid;
  out->block = 32 * kQuadWarps;
  out->smem = smem;
  out->nquads = grid * kQuadWarps * kQuadCols;
  return cudaSuccess;
}

cudaError_t launch_columns_thread_f32(const ColArgs& a, const ThreadArgs& ta, const ThreadShape& sh, cudaStream_t s) {
  if (sh.grid <= 0) return cudaSuccess;
  column_thread_kernel<kThreadKMax><<<sh.grid, sh.block, sh.smem, s>>>(a, ta);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}
