// Sparsified powers (Sec. 4.1, Algorithm 1): the W pattern from the
// truncated Neumann series of A^-1 D with the diagonal initial subspace,
// S = -D^-1 (A - D) (so that A = D (I - S)).  One warp per column j:
//
//   s = t = e_j;  for level = 1..k: t = S t, drop t by count p_l, s = s + t;
//   optionally drop s by count to `keep` entries (diagonal included).
//
// Dropping by count keeps the p largest-modulus off-diagonal entries (ties
// to the lower row); the diagonal entry j is never dropped and does not use
// up the count.  Exact-zero sums are not stored (the diagonal of s always is).
// Every sum is formed in a fixed order -- the products S_ic t_c of a row are
// added in increasing c, multiplications and additions rounded separately --
// so the values, and the choices made on them, do not depend on scheduling.
// The sparse vectors live in shared memory as row-sorted lists of at most
// kSpCap entries; a column that needs more reports DIAF_EUNSUPPORTED.
#include <cstdint>

#include "factors.cuh"

namespace {

constexpr int kSpCap = 512;   // entries of a sparse vector / product list per warp
constexpr int kSpWarps = 2;   // warps per block

__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ Cx<double> mul_rn(Cx<double> a, Cx<double> b) {
  return {__dsub_rn(__dmul_rn(a.re, b.re), __dmul_rn(a.im, b.im)),
          __dadd_rn(__dmul_rn(a.re, b.im), __dmul_rn(a.im, b.re))};
}
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ Cx<double> add_rn(Cx<double> a, Cx<double> b) {
  return {__dadd_rn(a.re, b.re), __dadd_rn(a.im, b.im)};
}
__device__ __forceinline__ double neg(double a) { return -a; }
__device__ __forceinline__ Cx<double> neg(Cx<double> a) { return {-a.re, -a.im}; }
__device__ __forceinline__ bool is_zero_v(double a) { return a == 0.0; }
__device__ __forceinline__ bool is_zero_v(Cx<double> a) { return a.re == 0.0 && a.im == 0.0; }
// ordering key |v|^2, rounded step by step
__device__ __forceinline__ double key_of(double a) { return __dmul_rn(a, a); }
__device__ __forceinline__ double key_of(Cx<double> a) { return __dadd_rn(__dmul_rn(a.re, a.re), __dmul_rn(a.im, a.im)); }
__device__ __forceinline__ double recip(double d) { return 1.0 / d; }
__device__ __forceinline__ Cx<double> recip(Cx<double> d) {
  // 1/d = conj(d) / |d|^2 (only the exact structure matters for complex A)
  const double n2 = __dadd_rn(__dmul_rn(d.re, d.re), __dmul_rn(d.im, d.im));
  return {d.re / n2, -d.im / n2};
}

template <class S>
__global__ void diag_recip_kernel(int n, const int32_t* __restrict__ cp, const int32_t* __restrict__ ri,
                                  const S* __restrict__ v, S* __restrict__ dinv, uint32_t* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  S d = sc_zero<S>();
  bool found = false;
  for (int p = cp[i]; p < cp[i + 1]; ++p)
    if (ri[p] == i) { d = v[p]; found = true; }
  if (!found || is_zero_v(d)) atomicOr(status, DEV_ST_BAD_INPUT);
  dinv[i] = found ? recip(d) : sc_zero<S>();
}

template <class S>
struct SpWarp {
  int32_t tR[kSpCap];
  int32_t sR[kSpCap];
  uint64_t pK[kSpCap];
  int32_t keep[kSpCap];
  S tV[kSpCap];
  S sV[kSpCap];
  S pV[kSpCap];
};

// exclusive warp scan of x (lane order); returns the prefix, *total the sum
__device__ __forceinline__ int warp_excl_scan(int x, int lane, int* total) {
  int v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(DIAF_FULL, v, o);
    if (lane >= o) v += y;
  }
  *total = __shfl_sync(DIAF_FULL, v, 31);
  return v - x;
}

// bitonic sort of pK[0..np) ascending with payload pV (np padded with ~0)
template <class S>
__device__ void warp_sort_pairs(SpWarp<S>& w, int np, int lane) {
  int P = 1;
  while (P < np) P <<= 1;
  for (int i = np + lane; i < P; i += 32) { w.pK[i] = ~0ull; w.pV[i] = sc_zero<S>(); }
  __syncwarp();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = lane; i < P; i += 32) {
        const int jx = i ^ stride;
        if (jx > i) {
          const bool up = (i & size) == 0;
          const uint64_t a = w.pK[i], b = w.pK[jx];
          if ((a > b) == up) {
            w.pK[i] = b; w.pK[jx] = a;
            const S va = w.pV[i]; w.pV[i] = w.pV[jx]; w.pV[jx] = va;
          }
        }
      }
      __syncwarp();
    }
  }
}

// Sorted pairs (key = row << 32 | order) -> row-sorted list (R, V) of the
// sums over equal rows, added in key order; zero sums are dropped unless the
// row is `keep_row`.  Returns the list length.
template <class S>
__device__ int warp_segment_sums(SpWarp<S>& w, int np, int32_t* R, S* V, int keep_row, int lane) {
  int carry = 0;
  for (int base = 0; base < np; base += 32) {
    const int p = base + lane;
    bool head = false, nz = false;
    int row = -1;
    S acc = sc_zero<S>();
    if (p < np) {
      row = (int)(w.pK[p] >> 32);
      head = p == 0 || (int)(w.pK[p - 1] >> 32) != row;
      if (head) {
        acc = w.pV[p];
        for (int q = p + 1; q < np && (int)(w.pK[q] >> 32) == row; ++q) acc = add_rn(acc, w.pV[q]);
        nz = !is_zero_v(acc) || row == keep_row;
      }
    }
    const unsigned bal = __ballot_sync(DIAF_FULL, head && nz);
    if (head && nz) {
      const int pos = carry + __popc(bal & ((1u << lane) - 1u));
      R[pos] = row;
      V[pos] = acc;
    }
    carry += __popc(bal);
  }
  __syncwarp();
  return carry;
}

// Keeps in (R, V, n) the entry `diag` (if present) and the `count` largest
// keys among the others (ties to the lower row); order preserved.  count < 0:
// keep all.  Returns the new length.
template <class S>
__device__ int warp_drop_by_count(SpWarp<S>& w, int32_t* R, S* V, int n, int diag, int count, int lane) {
  if (count < 0) return n;
  for (int i = lane; i < n; i += 32) w.keep[i] = R[i] == diag ? 1 : 0;
  __syncwarp();
  int off = 0;
  for (int i = lane; i < n; i += 32) off += R[i] != diag;
  off = warp_sum(off);
  if (off > count) {
    for (int it = 0; it < count; ++it) {  // select the best remaining entry, count times
      double bk = -1.0;
      int br = INT_MAX, bi = -1;
      for (int i = lane; i < n; i += 32) {
        if (w.keep[i] || R[i] == diag) continue;
        const double kk = key_of(V[i]);
        if (kk > bk || (kk == bk && R[i] < br)) { bk = kk; br = R[i]; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ok = __shfl_xor_sync(DIAF_FULL, bk, o);
        const int orr = __shfl_xor_sync(DIAF_FULL, br, o);
        const int oi = __shfl_xor_sync(DIAF_FULL, bi, o);
        if (ok > bk || (ok == bk && orr < br)) { bk = ok; br = orr; bi = oi; }
      }
      if (lane == 0 && bi >= 0) w.keep[bi] = 1;
      __syncwarp();
    }
  } else {
    for (int i = lane; i < n; i += 32) w.keep[i] = 1;
    __syncwarp();
  }
  // stable compaction
  int carry = 0;
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    const bool k = i < n && w.keep[i];
    int32_t r = 0;
    S v = sc_zero<S>();
    if (k) { r = R[i]; v = V[i]; }
    const unsigned bal = __ballot_sync(DIAF_FULL, k);
    __syncwarp();
    if (k) {
      const int pos = carry + __popc(bal & ((1u << lane) - 1u));
      R[pos] = r;
      V[pos] = v;
    }
    carry += __popc(bal);
    __syncwarp();
  }
  return carry;
}

// One column: returns its entry count (>= 0) and leaves the rows in w.sR, or
// -1 when a list would exceed kSpCap.
template <class S>
__device__ int sparsified_column(const int32_t* __restrict__ Acp, const int32_t* __restrict__ Ari,
                                 const S* __restrict__ Av, const S* __restrict__ dinv, int j, int k, int p_l,
                                 int keep, SpWarp<S>& w, int lane) {
  int nt = 1, ns = 1;
  if (lane == 0) {
    w.tR[0] = j; w.tV[0] = sc_real_s<S>(1.0);
    w.sR[0] = j; w.sV[0] = sc_real_s<S>(1.0);
  }
  __syncwarp();
  for (int level = 0; level < k; ++level) {
    // products S(:, c) t_c for the entries c of t, keyed (row, position of c in t)
    int np = 0, carry = 0;
    for (int base = 0; base < nt; base += 32) {
      const int e = base + lane;
      int cnt = 0;
      if (e < nt) {
        const int c = w.tR[e];
        cnt = Acp[c + 1] - Acp[c];
        for (int p = Acp[c]; p < Acp[c + 1]; ++p) cnt -= Ari[p] == c;
      }
      int tot;
      const int off = carry + warp_excl_scan(cnt, lane, &tot);
      if (carry + tot > kSpCap) return -1;  // warp-uniform
      if (e < nt) {
        const int c = w.tR[e];
        const S tc = w.tV[e];
        int o = off;
        for (int p = Acp[c]; p < Acp[c + 1]; ++p) {
          const int i = Ari[p];
          if (i == c) continue;
          const S sic = neg(mul_rn(dinv[i], Av[p]));  // S_ic = -(1/d_i) a_ic
          w.pK[o] = ((uint64_t)(uint32_t)i << 32) | (uint32_t)e;
          w.pV[o] = mul_rn(sic, tc);
          ++o;
        }
      }
      carry += tot;
    }
    np = carry;
    __syncwarp();
    warp_sort_pairs(w, np, lane);
    nt = warp_segment_sums(w, np, w.tR, w.tV, -1, lane);
    nt = warp_drop_by_count(w, w.tR, w.tV, nt, j, p_l > 0 ? p_l : -1, lane);
    // s = s + t: both row-sorted; s first so each sum is s_r + t_r
    if (ns + nt > kSpCap) return -1;
    for (int i = lane; i < ns; i += 32) { w.pK[i] = ((uint64_t)(uint32_t)w.sR[i] << 32); w.pV[i] = w.sV[i]; }
    for (int i = lane; i < nt; i += 32) { w.pK[ns + i] = ((uint64_t)(uint32_t)w.tR[i] << 32) | 1u; w.pV[ns + i] = w.tV[i]; }
    __syncwarp();
    warp_sort_pairs(w, ns + nt, lane);
    ns = warp_segment_sums(w, ns + nt, w.sR, w.sV, j, lane);
  }
  if (keep == 1) {  // the diagonal only
    int has = 0;
    for (int i = lane; i < ns; i += 32) has |= w.sR[i] == j;
    has = __any_sync(DIAF_FULL, has);
    __syncwarp();
    if (lane == 0 && has) w.sR[0] = j;
    __syncwarp();
    return has ? 1 : 0;
  }
  if (keep > 1) ns = warp_drop_by_count(w, w.sR, w.sV, ns, j, keep - 1, lane);
  return ns;
}

template <class S>
__global__ void __launch_bounds__(kSpWarps * 32)
    sparsified_kernel(int n, const int32_t* __restrict__ Acp, const int32_t* __restrict__ Ari,
                      const S* __restrict__ Av, const S* __restrict__ dinv, int k, int p_l, int keep,
                      const int32_t* __restrict__ colptr, int32_t* __restrict__ counts, int32_t* __restrict__ rowidx,
                      uint32_t* status) {
  extern __shared__ __align__(16) unsigned char sp_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  SpWarp<S>& w = reinterpret_cast<SpWarp<S>*>(sp_smem)[wib];
  for (int j = blockIdx.x * kSpWarps + wib; j < n; j += gridDim.x * kSpWarps) {
    const int cnt = sparsified_column<S>(Acp, Ari, Av, dinv, j, k, p_l, keep, w, lane);
    if (cnt < 0) {
      if (lane == 0) {
        atomicOr(status, DEV_ST_CAPACITY);
        if (counts) counts[j] = 0;
      }
    } else if (counts) {
      if (lane == 0) counts[j] = cnt;
    } else {
      const int o = colptr[j];
      if (colptr[j + 1] - o != cnt) {  // the second pass must reproduce the first
        if (lane == 0) atomicOr(status, DEV_ST_BAD_INPUT);
      } else {
        for (int i = lane; i < cnt; i += 32) rowidx[o + i] = w.sR[i];
      }
    }
    __syncwarp();
  }
}

template <class S>
diaf_status sparsified_run(const diaf_csc* A, int k, int p_l, int keep, int32_t* colptr, int32_t* counts,
                           int32_t* rowidx, cudaStream_t s) {
  const int n = A->n;
  uint32_t* st = nullptr;
  S* dinv = nullptr;
  if (cudaMallocAsync(&st, sizeof(uint32_t), s) != cudaSuccess) return DIAF_ENOMEM;
  if (cudaMallocAsync(&dinv, sizeof(S) * n, s) != cudaSuccess) { cudaFreeAsync(st, s); return DIAF_ENOMEM; }
  cudaMemsetAsync(st, 0, sizeof(uint32_t), s);
  diag_recip_kernel<S><<<ceil_div(n, 256), 256, 0, s>>>(n, A->colptr, A->rowidx, (const S*)A->vals, dinv, st);
  DIAF_COUNT_LAUNCH();
  const size_t smem = sizeof(SpWarp<S>) * kSpWarps;
  static int configured_device = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_device != dev) {
    if (cudaFuncSetAttribute(sparsified_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return DIAF_ECUDA;
    configured_device = dev;
  }
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int blocks = ceil_div(n, kSpWarps);
  if (blocks > sms * 8) blocks = sms * 8;
  sparsified_kernel<S><<<blocks, kSpWarps * 32, smem, s>>>(n, A->colptr, A->rowidx, (const S*)A->vals, dinv, k, p_l,
                                                            keep, colptr, counts, rowidx, st);
  DIAF_COUNT_LAUNCH();
  uint32_t h = 0;
  cudaMemcpyAsync(&h, st, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(dinv, s);
  cudaFreeAsync(st, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return DIAF_ECUDA;
  if (h & DEV_ST_BAD_INPUT) {
    diaf_set_last_error("A has a zero or missing diagonal entry (or the passes disagree)");
    return DIAF_EINVAL;
  }
  if (h & DEV_ST_CAPACITY) {
    diaf_set_last_error("a column's product list exceeds 512 entries: use dropping by count (p_l)");
    return DIAF_EUNSUPPORTED;
  }
  return DIAF_OK;
}

}  // namespace

extern "C" {

diaf_status diaf_sparsified_count(const diaf_csc* A, int32_t k, int32_t p_l, int32_t keep, int32_t* d_colptr,
                                  int64_t* nnz_out, void* stream) {
  if (!A || !d_colptr || !nnz_out || k < 0 || A->n < 0 || (A->dtype != DIAF_F64 && A->dtype != DIAF_C128))
    return DIAF_EINVAL;
  *nnz_out = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n = A->n;
  if (n == 0) return cudaMemsetAsync(d_colptr, 0, sizeof(int32_t), s) == cudaSuccess ? DIAF_OK : DIAF_ECUDA;
  int32_t *counts = nullptr, *bs = nullptr;
  if (cudaMallocAsync(&counts, sizeof(int32_t) * n, s) != cudaSuccess) return DIAF_ENOMEM;
  if (cudaMallocAsync(&bs, sizeof(int32_t) * scan_blocksums_size(n), s) != cudaSuccess) {
    cudaFreeAsync(counts, s);
    return DIAF_ENOMEM;
  }
  diaf_status st = A->dtype == DIAF_C128 ? sparsified_run<Cx<double>>(A, k, p_l, keep, nullptr, counts, nullptr, s)
                                         : sparsified_run<double>(A, k, p_l, keep, nullptr, counts, nullptr, s);
  if (st == DIAF_OK) {
    exclusive_scan_i32(counts, d_colptr, n, bs, s);
    int32_t last = 0;
    cudaMemcpyAsync(&last, d_colptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) st = DIAF_ECUDA;
    *nnz_out = last;
  }
  cudaFreeAsync(counts, s);
  cudaFreeAsync(bs, s);
  return st;
}

diaf_status diaf_sparsified_fill(const diaf_csc* A, int32_t k, int32_t p_l, int32_t keep, const int32_t* d_colptr,
                                 int32_t* d_rowidx, void* stream) {
  if (!A || !d_colptr || k < 0 || A->n < 0 || (A->dtype != DIAF_F64 && A->dtype != DIAF_C128)) return DIAF_EINVAL;
  if (A->n == 0) return DIAF_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return A->dtype == DIAF_C128
             ? sparsified_run<Cx<double>>(A, k, p_l, keep, const_cast<int32_t*>(d_colptr), nullptr, d_rowidx, s)
             : sparsified_run<double>(A, k, p_l, keep, const_cast<int32_t*>(d_colptr), nullptr, d_rowidx, s);
}

}  // extern "C"
