// Host-side launchers of the numeric column kernels, one translation unit per
// value type and precision so they compile in parallel.
#pragma once

#include "column_cta.cuh"
#include "column_mixed.cuh"
#include "column_thread.cuh"

// Launches the numeric pass for size bucket `bucket` over the listed columns
// (count_hint: an upper bound of the device-side count, for grid sizing).
// The work counter in `a` must be zero.  cudaErrorNotSupported: no kernel for
// this bucket.
// wpb: warps per block (0 = the most warps resident per SM).
cudaError_t launch_columns_f64(int bucket, int alg, const ColArgs& a, int count_hint, int wpb, cudaStream_t s);
cudaError_t launch_columns_c128(int bucket, int alg, const ColArgs& a, int count_hint, int wpb, cudaStream_t s);
cudaError_t launch_columns_mixed_f32(int bucket, int alg, const ColArgs& a, int count_hint, int wpb, cudaStream_t s);
cudaError_t launch_columns_mixed_c64(int bucket, int alg, const ColArgs& a, int count_hint, int wpb, cudaStream_t s);

// Size bucket 2 (one CTA per column, FP64 / complex128): grid size for the
// scratch slabs (0 on error) and the launch itself.
int cta_columns_grid(int dtype, int alg, int ldm, int count);
cudaError_t launch_columns_cta(int dtype, int alg, const ColArgs& a, const CtaScratch& sc, int grid, cudaStream_t s);
// mixed precision for bucket 2 (real DIAF-S; cudaErrorNotSupported otherwise):
// hands columns back through a.fb_list / a.fb_count
cudaError_t launch_columns_cta_mixed(int dtype, int alg, const ColArgs& a, const CtaScratch& sc, int grid,
                                     cudaStream_t s);
// its persistent grid (resident CTAs, capped by count); 0 when not available
int cta_columns_grid_mixed(int dtype, int alg, int ldm, int count);

// Four lanes per column (size bucket 0, real DIAF-S, mixed precision): the
// launch shape for tiles of at most M rows and K columns (grid, block, shared
// memory, quads of the grid; grid 0 when count_hint is 0), and the launch.
// Columns it leaves go to ta.defer_list for the warp kernel.
struct ThreadShape {
  int grid = 0, block = 0, nquads = 0;
  size_t smem = 0;
};
cudaError_t thread_columns_shape(int M, int K, int count_hint, ThreadShape* out);
cudaError_t launch_columns_thread_f32(const ColArgs& a, const ThreadArgs& ta, const ThreadShape& sh, cudaStream_t s);

// Bytes of the mixed warp kernels' global tile scratch (ColArgs::tile_scratch)
// for this bucket's launch: one FP64 tile per warp of the persistent grid
// (0: no mixed kernel for the bucket, or nothing to do).
size_t mixed_tile_scratch_f32(int bucket, int alg, int count_hint, int wpb);
size_t mixed_tile_scratch_c64(int bucket, int alg, int count_hint, int wpb);

// Persistent grid sized by occupancy; `per_warp` bytes of shared memory per
// warp.  Sets *grid and *wpb (the block's warps); the launch below uses it.
template <class Kern>
cudaError_t persistent_warps_shape(Kern kern, size_t per_warp, size_t& configured, int count_hint, int wpb_req,
                                   int* grid_out, int* wpb_out) {
  *grid_out = 0;
  *wpb_out = 1;
  if (count_hint <= 0) return cudaSuccess;
  // warps per block: the most warps resident per SM (228 KB of shared memory,
  // 1 KB reserved per block), ties to the smaller block -- unless requested
  int wpb = 1, best = 0;
  for (int w = 1; w <= 8; ++w) {
    const size_t blk = per_warp * w + 1024;
    if (per_warp * w > 227 * 1024) break;
    const int resident = (int)((228 * 1024) / blk) * w;
    if (resident > best) { best = resident; wpb = w; }
  }
  if (wpb_req > 0 && per_warp * wpb_req <= 227 * 1024) wpb = wpb_req;
  const size_t smem = per_warp * wpb;
  if (configured < smem) {  // attribute raised once per instantiation and size
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
  if (per_sm < 1) per_sm = 1;
  int grid = ceil_div(count_hint, wpb);
  if (grid > sms * per_sm) grid = sms * per_sm;
  *grid_out = grid;
  *wpb_out = wpb;
  return cudaSuccess;
}

template <class Kern>
cudaError_t launch_persistent_warps(Kern kern, size_t per_warp, size_t& configured, const ColArgs& a, int count_hint,
                                    int wpb_req, cudaStream_t s) {
  int grid = 0, wpb = 1;
  cudaError_t e = persistent_warps_shape(kern, per_warp, configured, count_hint, wpb_req, &grid, &wpb);
  if (e != cudaSuccess || grid == 0) return e;
  kern<<<grid, wpb * 32, per_warp * wpb, s>>>(a);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <class S, int KMAX, int MMAX, int ALG>
cudaError_t launch_warp_columns(const ColArgs& a, int count_hint, int wpb, cudaStream_t s) {
  static size_t configured = 0;
  return launch_persistent_warps(column_warp_kernel<S, KMAX, MMAX, ALG>, WarpLayout<S, KMAX, MMAX>::bytes(),
                                 configured, a, count_hint, wpb, s);
}

template <class S, int KMAX, int MMAX, int ALG>
struct MixedLaunch {
  static inline size_t configured = 0;
  static constexpr auto kernel() {
    constexpr int cap = mixed_reg_cap<S, KMAX, ALG>();
    if constexpr (cap > 0) return column_mixed_kernel_cap<S, KMAX, MMAX, ALG, (cap > 0 ? cap : 255)>;
    else return column_mixed_kernel<S, KMAX, MMAX, ALG>;
  }
  static cudaError_t launch(const ColArgs& a, int count_hint, int wpb, cudaStream_t s) {
    if (!a.tile_scratch && count_hint > 0) return cudaErrorInvalidValue;
    return launch_persistent_warps(kernel(), MixedLayout<S, KMAX, MMAX, ALG>::bytes(),
                                   configured, a, count_hint, wpb, s);
  }
  static size_t scratch(int count_hint, int wpb_req) {
    int grid = 0, wpb = 1;
    if (persistent_warps_shape(kernel(), MixedLayout<S, KMAX, MMAX, ALG>::bytes(),
                               configured, count_hint, wpb_req, &grid, &wpb) != cudaSuccess)
      return 0;
    return (size_t)grid * wpb * MixedLayout<S, KMAX, MMAX, ALG>::tile_bytes();
  }
};

template <class S, int KMAX, int MMAX, int ALG>
cudaError_t launch_mixed_columns(const ColArgs& a, int count_hint, int wpb, cudaStream_t s) {
  return MixedLaunch<S, KMAX, MMAX, ALG>::launch(a, count_hint, wpb, s);
}
