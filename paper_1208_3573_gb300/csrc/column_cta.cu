// Size bucket 2: one CTA per column for large tiles (FP64 and complex128;
// mixed precision for real DIAF-S).
#include "column_cta_mixed.cuh"
#include "launch.cuh"

namespace {

template <class S, int ALG>
cudaError_t configure(int ldm, size_t* smem_out) {
  static int configured_for = -1;
  const size_t smem = CtaSmem<S>::bytes(ldm);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  if (configured_for < (int)smem) {
    cudaError_t e = cudaFuncSetAttribute(column_cta_kernel<S, ALG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured_for = (int)smem;
  }
  *smem_out = smem;
  return cudaSuccess;
}

template <class S, int ALG>
int grid_for(int ldm, int count) {
  size_t smem = 0;
  if (configure<S, ALG>(ldm, &smem) != cudaSuccess) return 0;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, column_cta_kernel<S, ALG>, kCtaThreads, smem);
  if (per_sm < 1) return 0;
  int grid = sms * per_sm;
  return count < grid ? count : grid;
}

template <class S, int ALG>
cudaError_t launch(const ColArgs& a, const CtaScratch& sc, int grid, cudaStream_t s) {
  size_t smem = 0;
  cudaError_t e = configure<S, ALG>(sc.ldm, &smem);
  if (e != cudaSuccess) return e;
  column_cta_kernel<S, ALG><<<grid, kCtaThreads, smem, s>>>(a, sc);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}

}  // namespace

int cta_columns_grid(int dtype, int alg, int ldm, int count) {
  if (count <= 0) return 0;
  if (dtype == DIAF_C128)
    return alg == DIAF_ALG_S ? grid_for<Cx<double>, DIAF_ALG_S>(ldm, count) : grid_for<Cx<double>, DIAF_ALG_Q>(ldm, count);
  return alg == DIAF_ALG_S ? grid_for<double, DIAF_ALG_S>(ldm, count) : grid_for<double, DIAF_ALG_Q>(ldm, count);
}

cudaError_t launch_columns_cta(int dtype, int alg, const ColArgs& a, const CtaScratch& sc, int grid, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  if (dtype == DIAF_C128)
    return alg == DIAF_ALG_S ? launch<Cx<double>, DIAF_ALG_S>(a, sc, grid, s) : launch<Cx<double>, DIAF_ALG_Q>(a, sc, grid, s);
  return alg == DIAF_ALG_S ? launch<double, DIAF_ALG_S>(a, sc, grid, s) : launch<double, DIAF_ALG_Q>(a, sc, grid, s);
}

static cudaError_t configure_mixed(int ldm, size_t* smem_out) {
  const size_t smem = CtaMixedSmem::bytes(ldm);
  if (smem > 227 * 1024) return cudaErrorNotSupported;
  static int configured_for = -1;
  if (configured_for < (int)smem) {
    cudaError_t e = cudaFuncSetAttribute(column_cta_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured_for = (int)smem;
  }
  *smem_out = smem;
  return cudaSuccess;
}

int cta_columns_grid_mixed(int dtype, int alg, int ldm, int count) {
  if (count <= 0 || dtype != DIAF_F64 || alg != DIAF_ALG_S) return 0;
  size_t smem = 0;
  if (configure_mixed(ldm, &smem) != cudaSuccess) return 0;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, column_cta_mixed_kernel, kCtaThreads, smem);
  if (per_sm < 1) return 0;
  const int grid = sms * per_sm;
  return count < grid ? count : grid;
}

cudaError_t launch_columns_cta_mixed(int dtype, int alg, const ColArgs& a, const CtaScratch& sc, int grid,
                                     cudaStream_t s) {
  if (dtype != DIAF_F64 || alg != DIAF_ALG_S) return cudaErrorNotSupported;
  if (grid <= 0) return cudaSuccess;
  size_t smem = 0;
  cudaError_t ce = configure_mixed(sc.ldm, &smem);
  if (ce != cudaSuccess) return ce;
  column_cta_mixed_kernel<<<grid, kCtaThreads, smem, s>>>(a, sc);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}
