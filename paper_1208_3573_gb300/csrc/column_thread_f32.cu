// One thread per column: the mixed-precision DIAF-S kernel for small real tiles.
#include "column_thread.cuh"
#include "launch.cuh"

namespace {
size_t g_thread_smem_configured = 0;

// The round-robin schedule of warp_jacobi: in round rnd, position p >= 1 holds
// column 1 + ((p - 1 + rnd) mod L), position 0 column 0, and positions p and
// qq - 1 - p pair up.
cudaError_t upload_pair_table() {
  static bool done = false;  // per process; the table is the same on every device
  static int dev_done = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (done && dev_done == dev) return cudaSuccess;
  uint8_t tab[kThreadKMax / 2][kPairRounds][kPairSlots] = {};
  for (int np = 1; np <= kThreadKMax / 2; ++np) {
    const int qq = 2 * np, L = qq - 1;
    for (int rnd = 0; rnd < L; ++rnd)
      for (int pr = 0; pr < np; ++pr) {
        int ea = pr - 1 + rnd, eb = qq - 2 - pr + rnd;
        ea = ((ea % L) + L) % L;
        eb = eb % L;
        int x = pr == 0 ? 0 : 1 + ea, y = 1 + eb;
        if (x > y) { const int t = x; x = y; y = t; }
        tab[np - 1][rnd][pr] = (uint8_t)((x << 4) | y);
      }
  }
  e = cudaMemcpyToSymbol(kPairTab, tab, sizeof(tab));
  if (e == cudaSuccess) { done = true; dev_done = dev; }
  return e;
}
}  // namespace

cudaError_t thread_columns_shape(int M, int K, int count_hint, ThreadShape* out) {
  *out = ThreadShape{};
  if (count_hint <= 0) return cudaSuccess;
  if (M < 1 || K < 1 || M > kThreadMMax || K > kThreadKMax) return cudaErrorInvalidValue;
  cudaError_t te = upload_pair_table();
  if (te != cudaSuccess) return te;
  auto kern = column_thread_kernel<kThreadKMax>;
  const size_t smem = thread_warp_smem(M, K) * kQuadWarps;
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
