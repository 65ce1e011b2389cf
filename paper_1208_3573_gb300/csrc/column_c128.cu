// Numeric column kernels, complex128 values.
#include "launch.cuh"

cudaError_t launch_columns_c128(int bucket, int alg, const ColArgs& a, int count, int wpb, cudaStream_t s) {
  if (alg == DIAF_ALG_S) {
    if (bucket == 0) return launch_warp_columns<Cx<double>, 16, 32, DIAF_ALG_S>(a, count, wpb, s);
    if (bucket == 1) return launch_warp_columns<Cx<double>, 32, 64, DIAF_ALG_S>(a, count, wpb, s);
  } else {
    if (bucket == 0) return launch_warp_columns<Cx<double>, 16, 32, DIAF_ALG_Q>(a, count, wpb, s);
    if (bucket == 1) return launch_warp_columns<Cx<double>, 32, 64, DIAF_ALG_Q>(a, count, wpb, s);
  }
  return cudaErrorNotSupported;
}
