// Row-oriented sparse operations for the solve phase.
#include "plan.cuh"
#include "sparse.cuh"

namespace {

__global__ void count_rows_kernel(int n, const int32_t* cp, const int32_t* ri, int32_t* cnt) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int p = cp[j]; p < cp[j + 1]; ++p) atomicAdd(&cnt[ri[p]], 1);
}

template <class S>
__global__ void fill_rows_kernel(int n, const int32_t* cp, const int32_t* ri, const S* v, const int32_t* rowptr,
                                 int32_t* cursor, int32_t* colidx, S* vals) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int p = cp[j]; p < cp[j + 1]; ++p) {
    int i = ri[p];
    int pos = rowptr[i] + atomicAdd(&cursor[i], 1);
    colidx[pos] = j;
    vals[pos] = v[p];
  }
}

// Rows are short: insertion sort by column makes the order deterministic.
template <class S>
__global__ void sort_rows_kernel(int n, const int32_t* rowptr, int32_t* colidx, S* vals) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = rowptr[i], b = rowptr[i + 1];
  for (int p = a + 1; p < b; ++p) {
    int c = colidx[p];
    S v = vals[p];
    int q = p - 1;
    while (q >= a && colidx[q] > c) {
      colidx[q + 1] = colidx[q];
      vals[q + 1] = vals[q];
      --q;
    }
    colidx[q + 1] = c;
    vals[q + 1] = v;
  }
}

template <class S>
cudaError_t csc_to_csr_t(int n, int64_t nnz, const int32_t* cp, const int32_t* ri, const S* v, int32_t* rowptr,
                         int32_t* colidx, S* vals, int32_t* work, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int32_t* cnt = work;
  int32_t* bs = work + n;
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n, s);
  count_rows_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, cp, ri, cnt);
  DIAF_COUNT_LAUNCH();
  exclusive_scan_i32(cnt, rowptr, n, bs, s);
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n, s);
  fill_rows_kernel<S><<<ceil_div(n, 256), 256, 0, s>>>(n, cp, ri, v, rowptr, cnt, colidx, vals);
  DIAF_COUNT_LAUNCH();
  sort_rows_kernel<S><<<ceil_div(n, 256), 256, 0, s>>>(n, rowptr, colidx, vals);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}

// y = M x with a group of G lanes per row.
template <class S, int G>
__global__ void spmv_kernel(int n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                            const S* __restrict__ vals, const S* __restrict__ x, S* __restrict__ y) {
  int gid = (blockIdx.x * blockDim.x + threadIdx.x);
  int row = gid / G, sub = gid % G;
  S acc = sc_zero<S>();
  if (row < n) {
    for (int p = rowptr[row] + sub; p < rowptr[row + 1]; p += G) acc += vals[p] * x[colidx[p]];
  }
  acc = group_sum<G>(acc);
  if (row < n && sub == 0) y[row] = acc;
}

template <class S>
__global__ void tri_check_kernel(int n, const int32_t* rowptr, const int32_t* colidx, const S* vals, uint32_t* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t f = 0;
  bool diag = false;
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
    int c = colidx[p];
    if (c < i) f |= 1u;
    if (c > i) f |= 2u;
    if (c == i && sc_abs2(vals[p]) > 0.0) diag = true;
  }
  if (!diag) f |= 4u;
  if (f) atomicOr(out, f);
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ Cx<double> ld_cg(const Cx<double>* p) {
  double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}

constexpr long long kSpinLimit = 1ll << 22;  // polls of one flag before giving up (~seconds)

template <class S>
__global__ void trsv_syncfree_kernel(int n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                     const S* __restrict__ vals, const S* __restrict__ x, S* t, uint32_t* ready,
                                     int32_t* counter, uint32_t gen, int upper, uint32_t* status) {
  const int lane = threadIdx.x & 31;
  while (true) {
    int tk = 0;
    if (lane == 0) tk = atomicAdd(counter, 1);
    tk = __shfl_sync(DIAF_FULL, tk, 0);
    if (tk >= n) return;
    const int i = upper ? (n - 1 - tk) : tk;
    S acc = sc_zero<S>();
    S diag = sc_zero<S>();
    bool timed_out = false;
    for (int p = rowptr[i] + lane; p < rowptr[i + 1]; p += DIAF_WARP) {
      int c = colidx[p];
      S v = vals[p];
      if (c == i) { diag = v; continue; }
      long long it = 0;
      while (ld_acquire(ready + c) != gen) {
        if (++it > kSpinLimit) { timed_out = true; break; }
        __nanosleep(64);
      }
      acc += v * ld_cg(t + c);
    }
    acc = warp_sum(acc);
    diag = warp_sum(diag);
    if (__any_sync(DIAF_FULL, timed_out) && lane == 0) atomicOr(status, DEV_ST_TIMEOUT);
    if (lane == 0) {
      S b = x[i] - acc;
      double d2 = sc_abs2(diag);
      S ti = (1.0 / d2) * (b * sc_conj(diag));
      t[i] = ti;
      __threadfence();
      st_release(ready + i, gen);
    }
    __syncwarp();
  }
}

constexpr int kLevelThreads = 1024;
constexpr int kLevelPtrSmem = 8192;  // level pointers kept in shared memory up to this many levels

template <class S>
__global__ void __launch_bounds__(kLevelThreads)
    trsv_levels_kernel(int nlev, const int32_t* __restrict__ lvlptr, const int32_t* __restrict__ order,
                       const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                       const S* __restrict__ vals, const S* __restrict__ dinv, const S* __restrict__ x, S* t) {
  __shared__ int32_t sptr[kLevelPtrSmem + 1];
  const bool in_smem = nlev <= kLevelPtrSmem;
  if (in_smem)
    for (int i = threadIdx.x; i <= nlev; i += blockDim.x) sptr[i] = lvlptr[i];
  __syncthreads();
  for (int lv = 0; lv < nlev; ++lv) {
    const int b = in_smem ? sptr[lv] : lvlptr[lv];
    const int e = in_smem ? sptr[lv + 1] : lvlptr[lv + 1];
    for (int idx = b + threadIdx.x; idx < e; idx += blockDim.x) {
      const int i = order[idx];
      S acc = x[i];
      for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        const int j = colidx[p];
        if (j != i) acc -= vals[p] * t[j];
      }
      t[i] = acc * dinv[i];
    }
    __syncthreads();
  }
}

template <class S>
__global__ void diag_inverse_kernel(int n, const int32_t* rowptr, const int32_t* colidx, const S* vals, S* dinv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  S d = sc_zero<S>();
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p)
    if (colidx[p] == i) d = vals[p];
  dinv[i] = (1.0 / sc_abs2(d)) * sc_conj(d);
}

}  // namespace

cudaError_t csr_trsv_levels(const Csr& V, bool cplx, int nlev, const int32_t* lvlptr, const int32_t* order,
                            const void* dinv, const void* x, void* t, cudaStream_t s) {
  if (V.n <= 0) return cudaSuccess;
  if (cplx)
    trsv_levels_kernel<Cx<double>><<<1, kLevelThreads, 0, s>>>(nlev, lvlptr, order, V.rowptr, V.colidx,
                                                              (const Cx<double>*)V.vals, (const Cx<double>*)dinv,
                                                              (const Cx<double>*)x, (Cx<double>*)t);
  else
    trsv_levels_kernel<double><<<1, kLevelThreads, 0, s>>>(nlev, lvlptr, order, V.rowptr, V.colidx,
                                                          (const double*)V.vals, (const double*)dinv,
                                                          (const double*)x, (double*)t);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t csr_diag_inverse(const Csr& V, bool cplx, void* dinv, cudaStream_t s) {
  if (V.n <= 0) return cudaSuccess;
  if (cplx)
    diag_inverse_kernel<Cx<double>><<<ceil_div(V.n, 256), 256, 0, s>>>(V.n, V.rowptr, V.colidx,
                                                                       (const Cx<double>*)V.vals, (Cx<double>*)dinv);
  else
    diag_inverse_kernel<double><<<ceil_div(V.n, 256), 256, 0, s>>>(V.n, V.rowptr, V.colidx, (const double*)V.vals,
                                                                   (double*)dinv);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t csc_to_csr(int n, int64_t nnz, const int32_t* cp, const int32_t* ri, const void* v, bool cplx,
                       int32_t* rowptr, int32_t* colidx, void* vals, int32_t* work, cudaStream_t s) {
  if (cplx)
    return csc_to_csr_t<Cx<double>>(n, nnz, cp, ri, (const Cx<double>*)v, rowptr, colidx, (Cx<double>*)vals, work, s);
  return csc_to_csr_t<double>(n, nnz, cp, ri, (const double*)v, rowptr, colidx, (double*)vals, work, s);
}

cudaError_t csr_spmv(const Csr& M, bool cplx, const void* x, void* y, cudaStream_t s) {
  if (M.n <= 0) return cudaSuccess;
  constexpr int G = 4;
  int threads = 256;
  int blocks = ceil_div(M.n * G, threads);
  if (cplx)
    spmv_kernel<Cx<double>, G><<<blocks, threads, 0, s>>>(M.n, M.rowptr, M.colidx, (const Cx<double>*)M.vals,
                                                          (const Cx<double>*)x, (Cx<double>*)y);
  else
    spmv_kernel<double, G><<<blocks, threads, 0, s>>>(M.n, M.rowptr, M.colidx, (const double*)M.vals,
                                                      (const double*)x, (double*)y);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t csr_triangle_check(const Csr& V, bool cplx, uint32_t* out, cudaStream_t s) {
  if (V.n <= 0) return cudaSuccess;
  if (cplx)
    tri_check_kernel<Cx<double>><<<ceil_div(V.n, 256), 256, 0, s>>>(V.n, V.rowptr, V.colidx,
                                                                     (const Cx<double>*)V.vals, out);
  else
    tri_check_kernel<double><<<ceil_div(V.n, 256), 256, 0, s>>>(V.n, V.rowptr, V.colidx, (const double*)V.vals, out);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t csr_trsv_syncfree(const Csr& V, bool cplx, bool upper, const void* x, void* t, uint32_t* ready,
                              int32_t* counter, uint32_t gen, uint32_t* status, cudaStream_t s) {
  if (V.n <= 0) return cudaSuccess;
  cudaMemsetAsync(counter, 0, sizeof(int32_t), s);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int threads = 256;
  int blocks = ceil_div(V.n, threads / 32);
  if (blocks > sms * 8) blocks = sms * 8;
  if (cplx)
    trsv_syncfree_kernel<Cx<double>><<<blocks, threads, 0, s>>>(V.n, V.rowptr, V.colidx, (const Cx<double>*)V.vals,
                                                                (const Cx<double>*)x, (Cx<double>*)t, ready, counter,
                                                                gen, upper ? 1 : 0, status);
  else
    trsv_syncfree_kernel<double><<<blocks, threads, 0, s>>>(V.n, V.rowptr, V.colidx, (const double*)V.vals,
                                                            (const double*)x, (double*)t, ready, counter, gen,
                                                            upper ? 1 : 0, status);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}
