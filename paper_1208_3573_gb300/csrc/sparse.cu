// Row-oriented sparse operations for the solve phase.
#include <climits>

#include "plan.cuh"
#include "sparse.cuh"

namespace {

// CSC -> CSR.  kConvLanes lanes per column count the entries of every row
// and, after the scan, place them (independent loads and atomics across the
// lanes: the columns are short, so one thread per column would serialise
// them); the atomics leave each row's entries in no particular order, so one
// warp per row then sorts them by column.
constexpr int kConvLanes = 8;

__global__ void count_rows_kernel(int n, const int32_t* __restrict__ cp, const int32_t* __restrict__ ri,
                                  int32_t* __restrict__ cnt) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int j = (int)(gid / kConvLanes), sub = (int)(gid % kConvLanes);
  if (j >= n) return;
  const int e = cp[j + 1];
  for (int p = cp[j] + sub; p < e; p += kConvLanes) atomicAdd(&cnt[ri[p]], 1);
}

template <class S>
__global__ void fill_rows_kernel(int n, const int32_t* __restrict__ cp, const int32_t* __restrict__ ri,
                                 const S* __restrict__ v, const int32_t* __restrict__ rowptr,
                                 int32_t* __restrict__ cursor, int32_t* __restrict__ colidx, S* __restrict__ vals) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int j = (int)(gid / kConvLanes), sub = (int)(gid % kConvLanes);
  if (j >= n) return;
  const int e = cp[j + 1];
  for (int p = cp[j] + sub; p < e; p += kConvLanes) {
    const int i = ri[p];
    const int pos = rowptr[i] + atomicAdd(&cursor[i], 1);
    colidx[pos] = j;
    vals[pos] = v[p];
  }
}

// One warp per row: a row of up to 32 entries is sorted by column with a
// bitonic network of shuffles (each value follows its column through its
// source position); a longer row by insertion sort in lane 0.  The result is
// the same whatever order the atomics left.
template <class S>
__global__ void sort_rows_kernel(int n, const int32_t* __restrict__ rowptr, int32_t* __restrict__ colidx,
                                 S* __restrict__ vals) {
  const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= n) return;  // whole warps: blockDim.x is a multiple of 32
  const int a = rowptr[row], len = rowptr[row + 1] - a;
  if (len <= 1) return;
  if (len <= 32) {
    int key = lane < len ? colidx[a + lane] : INT_MAX;
    int src = lane;
    for (int size = 2; size <= 32; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        const int ok = __shfl_xor_sync(DIAF_FULL, key, stride);
        const int os = __shfl_xor_sync(DIAF_FULL, src, stride);
        const bool keep_min = ((lane & stride) == 0) == ((lane & size) == 0);
        const bool less = ok < key || (ok == key && os < src);  // (ok, os) before (key, src)
        if (keep_min ? less : !less) {
          key = ok;
          src = os;
        }
      }
    }
    S v = sc_zero<S>();
    if (lane < len) v = vals[a + src];
    __syncwarp();
    if (lane < len) {
      colidx[a + lane] = key;
      vals[a + lane] = v;
    }
  } else if (lane == 0) {
    for (int p = a + 1; p < a + len; ++p) {
      const int c = colidx[p];
      const S v = vals[p];
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
}

template <class S>
cudaError_t csc_to_csr_t(int n, int64_t nnz, const int32_t* cp, const int32_t* ri, const S* v, int32_t* rowptr,
                         int32_t* colidx, S* vals, int32_t* work, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int32_t* cnt = work;
  int32_t* bs = work + n;
  const int lane_blocks = (int)(((int64_t)n * kConvLanes + 255) / 256);
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n, s);
  count_rows_kernel<<<lane_blocks, 256, 0, s>>>(n, cp, ri, cnt);
  DIAF_COUNT_LAUNCH();
  exclusive_scan_i32(cnt, rowptr, n, bs, s);
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n, s);
  fill_rows_kernel<S><<<lane_blocks, 256, 0, s>>>(n, cp, ri, v, rowptr, cnt, colidx, vals);
  DIAF_COUNT_LAUNCH();
  sort_rows_kernel<S><<<ceil_div(n, 8), 256, 0, s>>>(n, rowptr, colidx, vals);
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

constexpr int kLevelThreads = 1024;
constexpr int kLevelPtrSmem = 8192;  // level pointers kept in shared memory up to this many levels
constexpr int kPrefetch = 4;         // off-diagonal entries of a row held in registers ahead of its level

// Row i of V goes to level position p = lvlptr[lev i] + rank i (the walk's
// place of row i in its level); len[p] = its number of off-diagonal entries.
__global__ void level_place_kernel(int n, const int32_t* __restrict__ lev, const int32_t* __restrict__ rank,
                                   const int32_t* __restrict__ rcnt, const int32_t* __restrict__ lvlptr,
                                   int32_t* __restrict__ pos, int32_t* __restrict__ xrow, int32_t* __restrict__ len) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p = lvlptr[lev[i]] + rank[i];
  pos[i] = p;
  xrow[p] = i;
  len[p] = rcnt[i];
}

// V's rows level by level, straight from its columns: kConvLanes lanes per
// column j; entry (i, j), i != j, goes to slot slot[e] of row position
// pos[i] with column position pos[j] and value v_ij / v_ii (the row scaled by
// its diagonal, which sits at entry dpos[i] of column i); the diagonal entry
// gives 1/v_jj at position pos[j] and raises *zflag when it is zero (or not
// a number).
template <class S>
__global__ void level_fill_kernel(int n, const int32_t* __restrict__ cp, const int32_t* __restrict__ ri,
                                  const S* __restrict__ v, const int32_t* __restrict__ dpos,
                                  const int32_t* __restrict__ slot, const int32_t* __restrict__ pos,
                                  const int32_t* __restrict__ rowptr, int32_t* __restrict__ pcol,
                                  S* __restrict__ pval, S* __restrict__ pdinv, uint32_t* __restrict__ zflag) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int j = (int)(gid / kConvLanes), sub = (int)(gid % kConvLanes);
  if (j >= n) return;
  const int e1 = cp[j + 1];
  for (int e = cp[j] + sub; e < e1; e += kConvLanes) {
    const int i = ri[e];
    if (i == j) {
      const S d = v[e];
      if (!(sc_abs2(d) > 0.0)) atomicOr(zflag, 1u);
      pdinv[pos[j]] = (1.0 / sc_abs2(d)) * sc_conj(d);
    } else {
      const S d = v[dpos[i]];
      const int q = rowptr[pos[i]] + slot[e];
      pcol[q] = pos[j];
      pval[q] = ((1.0 / sc_abs2(d)) * sc_conj(d)) * v[e];
    }
  }
}

// t[p] = x[xrow[p]] / diag of row p (level order): the scaled right-hand
// side the level solves start from, for all rows at once.
template <class S>
__global__ void scale_rhs_kernel(int n, const S* __restrict__ dinv, const int32_t* __restrict__ xrow,
                                 const S* __restrict__ x, S* __restrict__ t) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) t[p] = dinv[p] * x[xrow[p]];
}

__global__ void remap_cols_kernel(int64_t nnz, const int32_t* __restrict__ pos, const int32_t* __restrict__ cin,
                                  int32_t* __restrict__ cout) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    cout[e] = pos[cin[e]];
}

// Level-scheduled solve on the level-ordered matrix: the rows of level l are
// the contiguous positions lvlptr[l]..lvlptr[l+1], their off-diagonal
// entries point at positions of earlier levels, t is kept in level order.
// The rows are stored scaled by 1/diag and t starts as the scaled right-hand
// side (scale_rhs_kernel), so a row is t[p] -= sum v_pj t[j] in place, with
// no multiplication after the sum.  Nothing a row needs except t of earlier
// levels depends on the solve, so every thread loads its next row (bounds,
// its start value t[p] and the first kPrefetch entries) before the barrier
// that ends the current level; after the barrier only the loads of t remain
// on the critical path.  Those come from a ring of the last kWin
// positions of t in shared memory: while level [b, e) is written, slots of
// positions >= e - kWin are not overwritten, so reads of such positions use
// the ring and older ones use t in global memory (written too).
// One pass of the block over everything the solve will read (level-ordered
// rows and the start values in t), with 16-byte loads (the library's own
// arrays are 256-byte aligned).  The first solve after the level-ordered
// copies were built ran 0.42 ms instead of 0.29 ms on the 256^2
// convection-diffusion V, and a second solve right after it at full speed:
// the data was cold for the one SM that runs the solve.  With this pass
// (~30 us) in front, the first solve takes 0.35 ms; later solves skip it.
template <class S>
__device__ __forceinline__ void warm_level_data(int n, int nnz, const int32_t* rowptr, const int32_t* colidx,
                                                const S* vals, S* t) {
  unsigned acc = 0;
  const int4* r4 = reinterpret_cast<const int4*>(rowptr);
  const int4* c4 = reinterpret_cast<const int4*>(colidx);
  const int4* v4 = reinterpret_cast<const int4*>(vals);
  const int4* t4 = reinterpret_cast<const int4*>(t);
  for (int i = threadIdx.x; i < n / 4; i += blockDim.x) acc += r4[i].x;
  for (int i = threadIdx.x; i < nnz / 4; i += blockDim.x) acc += c4[i].z;
  for (int i = threadIdx.x; i < (int)(n * sizeof(S) / 16); i += blockDim.x) acc += t4[i].w;
  for (int i = threadIdx.x; i < (int)(nnz * sizeof(S) / 16); i += blockDim.x) acc += v4[i].y;
  if (acc == 0x9e3779b9u && n < 0) t[0] = sc_zero<S>();  // keeps the loads; never taken
}

template <class S>
constexpr int level_window() { return 131072 / (int)sizeof(S); }  // 128 KB ring

template <class S>
__global__ void __launch_bounds__(kLevelThreads, 1)
    trsv_levels_perm_kernel(int nlev, const int32_t* __restrict__ lvlptr, const int32_t* __restrict__ rowptr,
                            const int32_t* __restrict__ colidx, const S* __restrict__ vals,
                            S* t, int warm) {
  constexpr int kWin = level_window<S>();
  static_assert((kWin & (kWin - 1)) == 0, "ring size must be a power of two");
  extern __shared__ __align__(16) unsigned char level_ring[];
  S* tw = reinterpret_cast<S*>(level_ring);
  __shared__ int32_t sptr[kLevelPtrSmem + 1];
  const bool in_smem = nlev <= kLevelPtrSmem;
  if (in_smem)
    for (int i = threadIdx.x; i <= nlev; i += blockDim.x) sptr[i] = lvlptr[i];
  if (warm) {
    const int n_ = lvlptr[nlev];
    warm_level_data<S>(n_, rowptr[n_], rowptr, colidx, vals, t);
  }
  __syncthreads();
#define DIAF_LP(l) (in_smem ? sptr[(l)] : lvlptr[(l)])
  // registers for the first row this thread takes in the coming level
  int rb = 0, re = 0;
  S xb = sc_zero<S>();
  int pc[kPrefetch];
  S pv[kPrefetch];
#define DIAF_FETCH(pp)                                 \
  do {                                                 \
    const int p_ = (pp);                               \
    rb = rowptr[p_];                                   \
    re = rowptr[p_ + 1];                               \
    xb = t[p_];                                        \
    _Pragma("unroll") for (int q = 0; q < kPrefetch; ++q) { \
      const bool in = rb + q < re;                     \
      pc[q] = in ? colidx[rb + q] : 0;                 \
      pv[q] = in ? vals[rb + q] : sc_zero<S>();        \
    }                                                  \
  } while (0)
  if (nlev > 0 && DIAF_LP(0) + (int)threadIdx.x < DIAF_LP(1)) DIAF_FETCH(DIAF_LP(0) + (int)threadIdx.x);
  for (int lv = 0; lv < nlev; ++lv) {
    const int b = DIAF_LP(lv), e = DIAF_LP(lv + 1);
    const int lo = e - kWin;  // ring holds positions >= lo unchanged during this level
#define DIAF_TGET(c) ((c) >= lo ? tw[(c) & (kWin - 1)] : t[(c)])
    int p = b + threadIdx.x;
    if (p < e) {
      S acc = xb;
#pragma unroll
      for (int q = 0; q < kPrefetch; ++q)
        if (rb + q < re) acc = sc_msub(acc, pv[q], DIAF_TGET(pc[q]));
      for (int k = rb + kPrefetch; k < re; ++k) acc = sc_msub(acc, vals[k], DIAF_TGET(colidx[k]));
      t[p] = acc;
      tw[p & (kWin - 1)] = acc;
    }
    for (p += blockDim.x; p < e; p += blockDim.x) {  // levels wider than the block
      S acc = t[p];
      for (int k = rowptr[p]; k < rowptr[p + 1]; ++k) acc = sc_msub(acc, vals[k], DIAF_TGET(colidx[k]));
      t[p] = acc;
      tw[p & (kWin - 1)] = acc;
    }
    if (lv + 1 < nlev) {
      const int nb = e, ne = DIAF_LP(lv + 2);
      if (nb + (int)threadIdx.x < ne) DIAF_FETCH(nb + (int)threadIdx.x);
    }
    __syncthreads();
#undef DIAF_TGET
  }
#undef DIAF_FETCH
#undef DIAF_LP
}

// The same solve for matrices whose levels are at most kDeepThreads rows
// wide, with the row data fetched kDeep levels ahead instead of one.  A
// thread keeps its rows of the next kDeep levels in kDeep register sets (set
// k: the levels lv with lv mod kDeep = k).  A row's loads form two dependent
// round trips (the bounds in rowptr; then the entries and the start value
// t[p]), issued one level apart -- the first right after the set's previous level is done, the
// second one level later -- so no thread waits on a load before a barrier.
constexpr int kDeepThreads = 256;
constexpr int kDeep = 4;

template <class S>
__global__ void __launch_bounds__(kDeepThreads, 1)
    trsv_levels_deep_kernel(int nlev, const int32_t* __restrict__ lvlptr, const int32_t* __restrict__ rowptr,
                            const int32_t* __restrict__ colidx, const S* __restrict__ vals,
                            S* t, int warm) {
  constexpr int kWin = level_window<S>();
  extern __shared__ __align__(16) unsigned char level_ring[];
  S* tw = reinterpret_cast<S*>(level_ring);
  __shared__ int32_t sptr[kLevelPtrSmem + 1];
  const bool in_smem = nlev <= kLevelPtrSmem;
  if (in_smem)
    for (int i = threadIdx.x; i <= nlev; i += blockDim.x) sptr[i] = lvlptr[i];
  if (warm) {
    const int n_ = lvlptr[nlev];
    warm_level_data<S>(n_, rowptr[n_], rowptr, colidx, vals, t);
  }
  __syncthreads();
#define DIAF_LP(l) (in_smem ? sptr[(l)] : lvlptr[(l)])
  int rb[kDeep], re[kDeep], xr[kDeep];
  S xb[kDeep];
  int pc[kDeep][kPrefetch];
  S pv[kDeep][kPrefetch];
  // first round trip: the row's bounds (xr = its position, -1: no row)
#define DIAF_STAGE_A(k, lvl)                                      \
  do {                                                            \
    rb[k] = 0;                                                    \
    re[k] = 0;                                                    \
    xr[k] = -1;                                                   \
    const int p_ = DIAF_LP(lvl) + (int)threadIdx.x;               \
    if (p_ < DIAF_LP((lvl) + 1)) {                                \
      rb[k] = rowptr[p_];                                         \
      re[k] = rowptr[p_ + 1];                                     \
      xr[k] = p_;                                                 \
    }                                                             \
  } while (0)
  // second round trip: the start value t[p] and the first kPrefetch entries
#define DIAF_STAGE_B(k)                                           \
  do {                                                            \
    if (xr[k] >= 0) {                                             \
      xb[k] = t[xr[k]];                                           \
      _Pragma("unroll") for (int q = 0; q < kPrefetch; ++q) {     \
        const bool in = rb[k] + q < re[k];                        \
        pc[k][q] = in ? colidx[rb[k] + q] : 0;                    \
        pv[k][q] = in ? vals[rb[k] + q] : sc_zero<S>();           \
      }                                                           \
    }                                                             \
  } while (0)
#pragma unroll
  for (int k = 0; k < kDeep; ++k)
    if (k < nlev) DIAF_STAGE_A(k, k);
#pragma unroll
  for (int k = 0; k < kDeep; ++k)
    if (k < nlev) DIAF_STAGE_B(k);
  for (int lv0 = 0; lv0 < nlev; lv0 += kDeep) {
#pragma unroll
    for (int k = 0; k < kDeep; ++k) {
      const int lv = lv0 + k;
      if (lv < nlev) {  // uniform over the block
        const int b = DIAF_LP(lv), e = DIAF_LP(lv + 1);
        const int lo = e - kWin;
#define DIAF_TGET(c) ((c) >= lo ? tw[(c) & (kWin - 1)] : t[(c)])
        const int p = b + (int)threadIdx.x;
        if (p < e) {
          S acc = xb[k];
#pragma unroll
          for (int q = 0; q < kPrefetch; ++q)
            if (rb[k] + q < re[k]) acc = sc_msub(acc, pv[k][q], DIAF_TGET(pc[k][q]));
          for (int j = rb[k] + kPrefetch; j < re[k]; ++j) acc = sc_msub(acc, vals[j], DIAF_TGET(colidx[j]));
          t[p] = acc;
          tw[p & (kWin - 1)] = acc;
        }
#undef DIAF_TGET
        if (lv + kDeep < nlev) DIAF_STAGE_A(k, lv + kDeep);
        // the set whose first round trip was issued one level ago
        const int kb = (k + kDeep - 1) % kDeep;
        if (lv >= 1 && lv + kDeep - 1 < nlev) DIAF_STAGE_B(kb);
        __syncthreads();
      }
    }
  }
#undef DIAF_STAGE_A
#undef DIAF_STAGE_B
#undef DIAF_LP
}

}  // namespace

cudaError_t level_place(int n, const int32_t* lev, const int32_t* rank, const int32_t* rcnt, const int32_t* lvlptr,
                        int32_t* pos, int32_t* xrow, int32_t* work, int32_t* rowptr, cudaStream_t s) {
  if (n <= 0) return cudaMemsetAsync(rowptr, 0, sizeof(int32_t), s);
  int32_t* len = work;
  int32_t* bs = work + n;
  level_place_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, lev, rank, rcnt, lvlptr, pos, xrow, len);
  DIAF_COUNT_LAUNCH();
  return exclusive_scan_i32(len, rowptr, n, bs, s);
}

cudaError_t level_fill(int n, bool cplx, const int32_t* cp, const int32_t* ri, const void* v, const int32_t* dpos,
                       const int32_t* slot, const int32_t* pos, LevelCsr& L, uint32_t* zflag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)(((int64_t)n * kConvLanes + 255) / 256);
  if (cplx)
    level_fill_kernel<Cx<double>><<<blocks, 256, 0, s>>>(n, cp, ri, (const Cx<double>*)v, dpos, slot, pos, L.rowptr,
                                                          L.colidx, (Cx<double>*)L.vals, (Cx<double>*)L.dinv, zflag);
  else
    level_fill_kernel<double><<<blocks, 256, 0, s>>>(n, cp, ri, (const double*)v, dpos, slot, pos, L.rowptr, L.colidx,
                                                      (double*)L.vals, (double*)L.dinv, zflag);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t remap_columns(int64_t nnz, const int32_t* pos, const int32_t* cin, int32_t* cout, cudaStream_t s) {
  if (nnz <= 0) return cudaSuccess;
  int blocks = (int)((nnz + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  remap_cols_kernel<<<blocks, 256, 0, s>>>(nnz, pos, cin, cout);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <class S>
static cudaError_t trsv_levels_perm_t(const LevelCsr& L, const void* x, void* t, bool warm, cudaStream_t s) {
  constexpr size_t ring = sizeof(S) * level_window<S>();
  static int configured_device = -1;  // the attribute is per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_device != dev) {
    cudaError_t e = cudaFuncSetAttribute(trsv_levels_perm_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ring);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(trsv_levels_deep_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring);
    if (e != cudaSuccess) return e;
    configured_device = dev;
  }
  scale_rhs_kernel<S><<<ceil_div(L.n, 256), 256, 0, s>>>(L.n, (const S*)L.dinv, L.xrow, (const S*)x, (S*)t);
  DIAF_COUNT_LAUNCH();
  if (L.maxw <= kDeepThreads)
    trsv_levels_deep_kernel<S><<<1, kDeepThreads, ring, s>>>(L.nlev, L.lvlptr, L.rowptr, L.colidx,
                                                             (const S*)L.vals, (S*)t, warm ? 1 : 0);
  else
    trsv_levels_perm_kernel<S><<<1, kLevelThreads, ring, s>>>(L.nlev, L.lvlptr, L.rowptr, L.colidx,
                                                              (const S*)L.vals, (S*)t, warm ? 1 : 0);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t trsv_levels_perm(const LevelCsr& L, bool cplx, const void* x, void* t, cudaStream_t s, bool warm) {
  if (L.n <= 0) return cudaSuccess;
  return cplx ? trsv_levels_perm_t<Cx<double>>(L, x, t, warm, s) : trsv_levels_perm_t<double>(L, x, t, warm, s);
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


