// Symbolic pass of the columnwise setup: for every column j, the tile sizes
// (k_j = |J_j|, E_j = gathered entries, m_j = |R_j|), the sorted row union
// R_j (the nonzero rows of A(:,J_j), Sec. 2.1), the V count l_j, and the size
// bucket the numeric pass will run it in.
#pragma once

#include "common.cuh"

// Size buckets of the numeric pass: (KMAX, MMAX) capacities, checked in order.
struct BucketCap {
  int kmax, mmax, lmax;
};
constexpr int kNumBuckets = 3;
// 0, 1: one warp per column, tile in shared memory; 2: one CTA per column,
// tile in global scratch.
__host__ __device__ constexpr BucketCap bucket_cap(int b) {
  return b == 0 ? BucketCap{16, 32, 32} : (b == 1 ? BucketCap{32, 64, 64} : BucketCap{64, 1024, 1024});
}
constexpr int kMaxGather = 4096;  // E_j capacity of the planner's CTA path

struct PlanArgs {
  int n;
  const int32_t* Acp;
  const int32_t* Ari;
  const int32_t* Wcp;
  const int32_t* Wri;
  int rule;
  const int32_t* Vfcp;
  const int32_t* Vfri;
  const int32_t* budget;
  const int32_t* blk;  // DIAF_RULE_BLOCK: block of every row
  int edge_m0;      // size-bucket edges (tuning): max(m, k) <= edge_m0 -> bucket 0, <= edge_m1 -> bucket 1
  int edge_m1;
  // outputs
  int32_t* k;       // [n]
  int32_t* E;       // [n]
  int64_t* Eoff;    // [n+1]
  int32_t* rows;    // [sum E]: R_j at Eoff[j], m_j entries
  int32_t* m;       // [n]
  int32_t* l;       // [n]
  int32_t* jin;     // [n] 1 if j is a row of the tile
  int32_t* bucket_list;   // [kNumBuckets * n]
  int32_t* bucket_count;  // [kNumBuckets]
  int32_t* big_list;      // [n] columns with E_j > warp capacity
  int32_t* big_count;     // [1]
  int32_t* stats;         // [4]: max k, max m, max l, max E
  uint32_t* status;
};

// Host-side launches (plan.cu).
cudaError_t plan_count(const PlanArgs& a, cudaStream_t s);
cudaError_t plan_rows(const PlanArgs& a, cudaStream_t s);
cudaError_t exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int n, int64_t* blocksums, cudaStream_t s);
cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int n, int32_t* blocksums, cudaStream_t s);
int scan_blocksums_size(int n);
cudaError_t check_csc(int n, const int32_t* cp, const int32_t* ri, int64_t nnz, uint32_t* status, cudaStream_t s);
