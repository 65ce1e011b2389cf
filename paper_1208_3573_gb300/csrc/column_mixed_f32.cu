// Numeric column kernels, mixed precision (FP32 factorisations, FP64 tile and refinement), real values.
#include "launch.cuh"

cudaError_t launch_columns_mixed_f32(int bucket, int alg, const ColArgs& a, int count_hint, int wpb, cudaStream_t s) {
  if (alg == DIAF_ALG_S) {
    if (bucket == 0) return launch_mixed_columns<float, 16, 32, DIAF_ALG_S>(a, count_hint, wpb, s);
    if (bucket == 1) return launch_mixed_columns<float, 32, 64, DIAF_ALG_S>(a, count_hint, wpb, s);
  } else {
    if (bucket == 0) return launch_mixed_columns<float, 16, 32, DIAF_ALG_Q>(a, count_hint, wpb, s);
    if (bucket == 1) return launch_mixed_columns<float, 32, 64, DIAF_ALG_Q>(a, count_hint, wpb, s);
  }
  return cudaErrorNotSupported;
}

size_t mixed_tile_scratch_f32(int bucket, int alg, int count_hint, int wpb) {
  if (alg == DIAF_ALG_S) {
    if (bucket == 0) return MixedLaunch<float, 16, 32, DIAF_ALG_S>::scratch(count_hint, wpb);
    if (bucket == 1) return MixedLaunch<float, 32, 64, DIAF_ALG_S>::scratch(count_hint, wpb);
  } else {
    if (bucket == 0) return MixedLaunch<float, 16, 32, DIAF_ALG_Q>::scratch(count_hint, wpb);
    if (bucket == 1) return MixedLaunch<float, 32, 64, DIAF_ALG_Q>::scratch(count_hint, wpb);
  }
  return 0;
}
