// Symbolic pass (row unions, V counts, buckets) and the scans it needs.
#include <climits>

#include "plan.cuh"

namespace {

constexpr int kWarpGather = 256;  // E_j capacity of the warp path
constexpr int kPlanWarps = 8;     // warps per CTA in the warp path
constexpr int kPlanCtaThreads = 256;

__device__ __forceinline__ bool admissible(int rule, int i, int j, const int32_t* blk) {
  if (i == j) return false;
  if (rule == DIAF_RULE_UPPER) return i < j;
  if (rule == DIAF_RULE_LOWER) return i > j;
  if (rule == DIAF_RULE_BLOCK) return blk[i] == blk[j];
  return true;
}

// Input check: column pointers monotone, rows in range and strictly increasing.
__global__ void check_csc_kernel(int n, const int32_t* __restrict__ cp, const int32_t* __restrict__ ri, int64_t nnz,
                                 uint32_t* status) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int a = cp[j], b = cp[j + 1];
  bool bad = (a < 0) || (b < a) || ((int64_t)b > nnz) || (j == 0 && a != 0) || (j == n - 1 && (int64_t)b != nnz);
  if (!bad) {
    int prev = -1;
    for (int p = a; p < b; ++p) {
      int r = ri[p];
      if (r <= prev || r >= n) { bad = true; break; }
      prev = r;
    }
  }
  if (bad) atomicOr(status, DEV_ST_BAD_INPUT);
}

// k_j, E_j and the list of columns whose gather exceeds the warp capacity.
__global__ void plan_count_kernel(PlanArgs a) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.n) return;
  // the input check ran before on the stream: with bad indices, read nothing
  // (E stays unset; the host sees the status before it uses E)
  if (*(volatile const uint32_t*)a.status & DEV_ST_BAD_INPUT) return;
  int w0 = a.Wcp[j], w1 = a.Wcp[j + 1];
  int E = 0;
  for (int p = w0; p < w1; ++p) {
    int c = a.Wri[p];
    E += a.Acp[c + 1] - a.Acp[c];
  }
  a.k[j] = w1 - w0;
  a.E[j] = E;
  if (E > kWarpGather) {
    int pos = atomicAdd(a.big_count, 1);
    a.big_list[pos] = j;
  }
  atomicMax(&a.stats[0], w1 - w0);
  atomicMax(&a.stats[3], E);
}

// Finishes column j once its sorted gathered rows are in s[0..E): writes the
// unique rows R_j, counts admissible candidates, l_j, bucket.
// mx: null, or (warp path) a thread-0 accumulator of max m (mx[0]) and
// max l (mx[1]) that the caller publishes once instead of per column.
template <int NT>
__device__ void finish_column(const PlanArgs& a, int j, const int32_t* s, int E, int tid, int* sh_cnt,
                              int* mx = nullptr) {
  // unique + compaction (NT threads cooperating; s is sorted)
  int32_t* out = a.rows + a.Eoff[j];
  int base = 0, ncand = 0, jin = 0;
  for (int c0 = 0; c0 < E; c0 += NT) {
    int e = c0 + tid;
    bool f = false;
    int r = 0;
    if (e < E) {
      r = s[e];
      f = (e == 0) || (s[e - 1] != r);
    }
    // block-level exclusive prefix of f
    if (NT == 32) {
      unsigned b = __ballot_sync(DIAF_FULL, f);
      int pos = base + __popc(b & ((1u << tid) - 1u));
      if (f) {
        out[pos] = r;
        ncand += admissible(a.rule, r, j, a.blk);
        jin |= (r == j);
      }
      base += __popc(b);
    } else {
      unsigned b = __ballot_sync(DIAF_FULL, f);
      int warp = tid >> 5, lane = tid & 31;
      if (lane == 0) sh_cnt[warp] = __popc(b);
      __syncthreads();
      int before = 0, tot = 0;
      for (int w = 0; w < NT / 32; ++w) {
        int c = sh_cnt[w];
        before += (w < warp) ? c : 0;
        tot += c;
      }
      int pos = base + before + __popc(b & ((1u << lane) - 1u));
      if (f) {
        out[pos] = r;
        ncand += admissible(a.rule, r, j, a.blk);
        jin |= (r == j);
      }
      base += tot;
      __syncthreads();
    }
  }
  // reduce ncand, jin
  if (NT == 32) {
    ncand = warp_sum(ncand);
    jin = warp_max(jin);
  } else {
    ncand = warp_sum(ncand);
    jin = warp_max(jin);
    int warp = tid >> 5, lane = tid & 31;
    __syncthreads();
    if (lane == 0) { sh_cnt[warp] = ncand; sh_cnt[NT / 32 + warp] = jin; }
    __syncthreads();
    ncand = 0; jin = 0;
    for (int w = 0; w < NT / 32; ++w) { ncand += sh_cnt[w]; jin |= sh_cnt[NT / 32 + w]; }
  }
  if (tid == 0) {
    int m = base;
    int k = a.k[j];
    int l;
    if (a.rule == DIAF_RULE_FIXED) {
      l = a.Vfcp[j + 1] - a.Vfcp[j];
    } else {
      int s_extra = a.budget ? a.budget[j] - 1 : ncand;
      s_extra = s_extra < 0 ? 0 : (s_extra > ncand ? ncand : s_extra);
      l = 1 + s_extra;
    }
    a.m[j] = m;
    a.l[j] = l;
    a.jin[j] = jin;
    int b = -1;
    for (int t = 0; t < kNumBuckets; ++t) {
      int mm = m > k ? m : k;
      BucketCap cap = bucket_cap(t);
      const int medge = t == 0 ? a.edge_m0 : (t == 1 ? a.edge_m1 : cap.mmax);
      if (k <= cap.kmax && mm <= cap.mmax && mm <= medge && l <= cap.lmax) { b = t; break; }
    }
    if (b < 0) {
      atomicOr(a.status, DEV_ST_CAPACITY);
    } else {
      int pos = atomicAdd(&a.bucket_count[b], 1);
      a.bucket_list[b * a.n + pos] = j;
    }
    if (mx) {
      mx[0] = m > mx[0] ? m : mx[0];
      mx[1] = l > mx[1] ? l : mx[1];
    } else {
      atomicMax(&a.stats[1], m);
      atomicMax(&a.stats[2], l);
    }
  }
}

template <int NT>
__device__ void bitonic_sort(int32_t* s, int N, int tid) {
  for (int size = 2; size <= N; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < (N >> 1); i += NT) {
        int lo = (i / stride) * 2 * stride + (i % stride);
        int hi = lo + stride;
        bool asc = (lo & size) == 0;
        int x = s[lo], y = s[hi];
        if ((x > y) == asc) { s[lo] = y; s[hi] = x; }
      }
      if (NT == 32) __syncwarp(); else __syncthreads();
    }
  }
}

template <int NT>
__device__ void gather_rows(const PlanArgs& a, int j, int32_t* s, int N, int tid) {
  int w0 = a.Wcp[j], w1 = a.Wcp[j + 1];
  int e0 = 0;
  for (int p = w0; p < w1; ++p) {
    int c = a.Wri[p];
    int c0 = a.Acp[c], len = a.Acp[c + 1] - c0;
    for (int t = tid; t < len; t += NT) s[e0 + t] = a.Ari[c0 + t];
    e0 += len;
  }
  for (int t = e0 + tid; t < N; t += NT) s[t] = INT_MAX;
  if (NT == 32) __syncwarp(); else __syncthreads();
}

// Bitonic sort of s[0..N) (N a power of two, 2 <= N <= 32 PER) by one warp
// with the keys in registers: element e = 32 i + lane sits in register i of
// its lane, so compare-exchange partners at distance >= 32 are two registers
// of one lane and those at distance < 32 are one register of two lanes (a
// shuffle).  Same network and result as bitonic_sort; reads s once and writes
// it back once instead of two loads and stores per stage.
template <int PER>
__device__ void bitonic_sort_regs(int32_t* s, int N, int lane) {
  int32_t x[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) x[i] = (32 * i + lane < N) ? s[32 * i + lane] : INT_MAX;
  for (int k = 2; k <= N; k <<= 1) {
    // partners at distance 32 JJ (JJ = PER / 2 .. 1, those below k): registers i and i + JJ
#pragma unroll
    for (int JJ = PER / 2; JJ >= 1; JJ >>= 1) {
      if (32 * JJ < k) {
#pragma unroll
        for (int i = 0; i < PER; ++i) {
          if ((i & JJ) == 0) {
            const int e = 32 * i + lane;
            const bool asc = (e & k) == 0;
            const int32_t a = x[i], b = x[i + JJ];
            const bool sw = asc ? (a > b) : (a < b);
            x[i] = sw ? b : a;
            x[i + JJ] = sw ? a : b;
          }
        }
      }
    }
    // partners at distance j < 32: the same register of lanes lane and lane ^ j
    for (int j = (k >> 1) < 16 ? (k >> 1) : 16; j > 0; j >>= 1) {
      const bool lower = (lane & j) == 0;
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        const int e = 32 * i + lane;
        const bool asc = (e & k) == 0;
        const int32_t p = __shfl_xor_sync(DIAF_FULL, x[i], j);
        const int32_t lo = x[i] < p ? x[i] : p, hi = x[i] < p ? p : x[i];
        x[i] = (lower == asc) ? lo : hi;
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < PER; ++i)
    if (32 * i + lane < N) s[32 * i + lane] = x[i];
  __syncwarp();
}

// The warp path's gather: lane p takes entry p of W(:,j) (its A column's
// start and length load in parallel), a warp scan of the lengths places each
// column's run, and each lane copies its run -- a few dependent round trips
// per column instead of three per entry of W(:,j).
__device__ void gather_rows_warp(const PlanArgs& a, int j, int32_t* s, int N, int lane) {
  const int w0 = a.Wcp[j], w1 = a.Wcp[j + 1];
  int e0 = 0;
  for (int p0 = w0; p0 < w1; p0 += 32) {
    const int p = p0 + lane;
    int c0 = 0, len = 0;
    if (p < w1) {
      const int c = a.Wri[p];
      c0 = a.Acp[c];
      len = a.Acp[c + 1] - c0;
    }
    int inc = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(DIAF_FULL, inc, o);
      if (lane >= o) inc += y;
    }
    const int off = e0 + inc - len;
#pragma unroll 4
    for (int t = 0; t < len; ++t) s[off + t] = a.Ari[c0 + t];
    e0 += __shfl_sync(DIAF_FULL, inc, 31);
  }
  for (int t = e0 + lane; t < N; t += 32) s[t] = INT_MAX;
  __syncwarp();
}

// Sorted unique rows of s[0..E) into s[0..m) (returns m) through a bitmap of
// the span [lo, lo + 32 nw) in `bits` (one warp): each entry sets its bit,
// then the words are read back in order.  The result equals sorting and
// removing duplicates.
__device__ int bitmap_unique_warp(int32_t* s, int E, int lo, int nw, uint32_t* bits, int lane) {
  for (int w = lane; w < nw; w += 32) bits[w] = 0u;
  __syncwarp();
  for (int t = lane; t < E; t += 32) {
    const int d = s[t] - lo;
    atomicOr(&bits[d >> 5], 1u << (d & 31));
  }
  __syncwarp();
  int base = 0;
  for (int w0 = 0; w0 < nw; w0 += 32) {
    const int w = w0 + lane;
    uint32_t b = w < nw ? bits[w] : 0u;
    const int c = __popc(b);
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(DIAF_FULL, inc, o);
      if (lane >= o) inc += y;
    }
    int pos = base + inc - c;
    while (b) {
      s[pos++] = lo + 32 * w + (__ffs(b) - 1);
      b &= b - 1u;
    }
    base += __shfl_sync(DIAF_FULL, inc, 31);
  }
  __syncwarp();
  return base;
}

constexpr int kBitmapWords = 64;  // spans of up to 2,048 rows take the bitmap

__global__ void __launch_bounds__(kPlanWarps * 32) plan_rows_warp_kernel(PlanArgs a) {
  __shared__ int32_t sbuf[kPlanWarps][kWarpGather];
  __shared__ uint32_t sbits[kPlanWarps][kBitmapWords];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int gw = blockIdx.x * kPlanWarps + warp, nw = gridDim.x * kPlanWarps;
  int mx[2] = {0, 0};
  for (int j = gw; j < a.n; j += nw) {
    int E = a.E[j];
    if (E > kWarpGather) continue;
    int N = 2;
    while (N < E) N <<= 1;
    gather_rows_warp(a, j, sbuf[warp], N, lane);
    // rows within a short span (banded operators): a bitmap instead of the sort
    int lo = INT_MAX, hi = -1;
    for (int t = lane; t < E; t += 32) {
      const int r = sbuf[warp][t];
      lo = r < lo ? r : lo;
      hi = r > hi ? r : hi;
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    if (E > 0 && hi - lo < 32 * kBitmapWords) {
      E = bitmap_unique_warp(sbuf[warp], E, lo, ((hi - lo) >> 5) + 1, sbits[warp], lane);
    } else {
      if (N <= 32) bitonic_sort_regs<1>(sbuf[warp], N, lane);
      else if (N <= 64) bitonic_sort_regs<2>(sbuf[warp], N, lane);
      else if (N <= 128) bitonic_sort_regs<4>(sbuf[warp], N, lane);
      else bitonic_sort_regs<8>(sbuf[warp], N, lane);
    }
    finish_column<32>(a, j, sbuf[warp], E, lane, nullptr, mx);
    __syncwarp();
  }
  if (lane == 0 && (mx[0] | mx[1])) {
    atomicMax(&a.stats[1], mx[0]);
    atomicMax(&a.stats[2], mx[1]);
  }
}

__global__ void __launch_bounds__(kPlanCtaThreads) plan_rows_cta_kernel(PlanArgs a) {
  __shared__ int32_t sbuf[kMaxGather];
  __shared__ int sh_cnt[2 * kPlanCtaThreads / 32];
  int cnt = *a.big_count;
  for (int t = blockIdx.x; t < cnt; t += gridDim.x) {
    int j = a.big_list[t];
    int E = a.E[j];
    if (E > kMaxGather) {
      if (threadIdx.x == 0) atomicOr(a.status, DEV_ST_CAPACITY);
      continue;
    }
    int N = 2;
    while (N < E) N <<= 1;
    gather_rows<kPlanCtaThreads>(a, j, sbuf, N, threadIdx.x);
    bitonic_sort<kPlanCtaThreads>(sbuf, N, threadIdx.x);
    finish_column<kPlanCtaThreads>(a, j, sbuf, E, threadIdx.x, sh_cnt);
    __syncthreads();
  }
}

// --------------------------------------------------------------- scans
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;

template <class TI, class TO>
__device__ TO block_exclusive_scan(TO v, TO* sh, TO& total) {
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  TO x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    TO y = __shfl_up_sync(DIAF_FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    TO w = lane < kScanThreads / 32 ? sh[lane] : TO(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      TO y = __shfl_up_sync(DIAF_FULL, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) sh[lane] = w;
  }
  __syncthreads();
  TO before = warp > 0 ? sh[warp - 1] : TO(0);
  total = sh[kScanThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

template <class TI, class TO>
__global__ void scan_reduce_kernel(const TI* in, int n, TO* blocksums) {
  __shared__ TO sh[kScanThreads / 32];
  int base = blockIdx.x * kScanBlock;
  TO s = 0;
  for (int i = 0; i < kScanItems; ++i) {
    int idx = base + threadIdx.x * kScanItems + i;
    if (idx < n) s += (TO)in[idx];
  }
  TO total;
  block_exclusive_scan<TI, TO>(s, sh, total);
  if (threadIdx.x == 0) blocksums[blockIdx.x] = total;
}

template <class TO>
__global__ void scan_blocksums_kernel(TO* blocksums, int nb) {
  __shared__ TO sh[kScanThreads / 32];
  TO carry = 0;
  for (int c0 = 0; c0 < nb; c0 += kScanThreads) {
    int i = c0 + threadIdx.x;
    TO v = i < nb ? blocksums[i] : TO(0);
    TO total;
    TO ex = block_exclusive_scan<TO, TO>(v, sh, total);
    if (i < nb) blocksums[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) blocksums[nb] = carry;
}

template <class TI, class TO>
__global__ void scan_apply_kernel(const TI* in, TO* out, int n, const TO* blocksums, int nb) {
  __shared__ TO sh[kScanThreads / 32];
  int base = blockIdx.x * kScanBlock;
  TO vals[kScanItems];
  TO s = 0;
  for (int i = 0; i < kScanItems; ++i) {
    int idx = base + threadIdx.x * kScanItems + i;
    vals[i] = idx < n ? (TO)in[idx] : TO(0);
    s += vals[i];
  }
  TO total;
  TO ex = block_exclusive_scan<TI, TO>(s, sh, total) + blocksums[blockIdx.x];
  for (int i = 0; i < kScanItems; ++i) {
    int idx = base + threadIdx.x * kScanItems + i;
    if (idx < n) out[idx] = ex;
    ex += vals[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = blocksums[nb];
}

template <class TI, class TO>
cudaError_t exclusive_scan(const TI* in, TO* out, int n, TO* blocksums, cudaStream_t s) {
  int nb = ceil_div(n > 0 ? n : 1, kScanBlock);
  scan_reduce_kernel<TI, TO><<<nb, kScanThreads, 0, s>>>(in, n, blocksums);
  DIAF_COUNT_LAUNCH();
  scan_blocksums_kernel<TO><<<1, kScanThreads, 0, s>>>(blocksums, nb);
  DIAF_COUNT_LAUNCH();
  scan_apply_kernel<TI, TO><<<nb, kScanThreads, 0, s>>>(in, out, n, blocksums, nb);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}

}  // namespace

int scan_blocksums_size(int n) { return ceil_div(n > 0 ? n : 1, kScanBlock) + 1; }

cudaError_t exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int n, int64_t* blocksums, cudaStream_t s) {
  return exclusive_scan<int32_t, long long>(in, reinterpret_cast<long long*>(out), n,
                                            reinterpret_cast<long long*>(blocksums), s);
}

cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int n, int32_t* blocksums, cudaStream_t s) {
  return exclusive_scan<int32_t, int>(in, out, n, blocksums, s);
}

cudaError_t check_csc(int n, const int32_t* cp, const int32_t* ri, int64_t nnz, uint32_t* status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  check_csc_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, cp, ri, nnz, status);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t plan_count(const PlanArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  plan_count_kernel<<<ceil_div(a.n, 256), 256, 0, s>>>(a);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t plan_rows(const PlanArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int blocks = ceil_div(a.n, kPlanWarps);
  if (blocks > sms * 8) blocks = sms * 8;
  plan_rows_warp_kernel<<<blocks, kPlanWarps * 32, 0, s>>>(a);
  DIAF_COUNT_LAUNCH();
  plan_rows_cta_kernel<<<sms * 2, kPlanCtaThreads, 0, s>>>(a);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}
