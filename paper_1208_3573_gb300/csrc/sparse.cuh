// Row-oriented sparse operations used by the solve phase: CSC -> CSR
// transpose, CSR SpMV, and the triangular solve with V (x -> V^-1 x) that
// the preconditioner A^-1 ~ W V^-1 needs (eq. afac).
#pragma once

#include "common.cuh"

struct Csr {
  int n = 0;
  int64_t nnz = 0;
  int32_t* rowptr = nullptr;
  int32_t* colidx = nullptr;
  void* vals = nullptr;  // double or Cx<double>
};

// Transpose of a CSC matrix into CSR (column order within each row).
// Buffers rowptr (n+1), colidx (nnz), vals (nnz * elem) are provided by the
// caller; `work` needs (n + scan_blocksums_size(n)) int32.
cudaError_t csc_to_csr(int n, int64_t nnz, const int32_t* cp, const int32_t* ri, const void* v, bool cplx,
                       int32_t* rowptr, int32_t* colidx, void* vals, int32_t* work, cudaStream_t s);

// y = M x (CSR); beta_zero: y overwritten.  Complex when cplx.
cudaError_t csr_spmv(const Csr& M, bool cplx, const void* x, void* y, cudaStream_t s);

// Checks that CSR V is triangular: status bit 1 = has strictly lower entries,
// 2 = has strictly upper entries, 4 = missing or zero diagonal.
cudaError_t csr_triangle_check(const Csr& V, bool cplx, uint32_t* out, cudaStream_t s);

// V in level order for the level-scheduled solve: position p holds row
// xrow[p] of V; the rows of level l (their depth in V's dependency graph) are
// positions lvlptr[l]..lvlptr[l+1]; rowptr/colidx/vals hold each row's
// off-diagonal entries with columns renumbered to positions; dinv = 1 / diag.
struct LevelCsr {
  int n = 0;
  int nlev = 0;
  int64_t nnz = 0;              // off-diagonal entries
  int32_t* lvlptr = nullptr;    // nlev + 1
  int32_t* rowptr = nullptr;    // n + 1
  int32_t* colidx = nullptr;    // nnz
  void* vals = nullptr;         // nnz
  void* dinv = nullptr;         // n
  int32_t* xrow = nullptr;      // n
  int maxw = 0;                 // rows of the widest level (picks the solve kernel)
};

// Builds L (buffers allocated by the caller; L.n, L.nlev, L.lvlptr set) from
// the triangular CSR V (every diagonal entry present) and the level order
// `order` (rows level by level); pos[i] receives the position of row i;
// work needs n + scan_blocksums_size(n) int32.
cudaError_t csr_level_permute(const Csr& V, bool cplx, const int32_t* order, int32_t* pos, int32_t* work,
                              LevelCsr& L, cudaStream_t s);

// cout[e] = pos[cin[e]] (column indices renumbered to level positions).
cudaError_t remap_columns(int64_t nnz, const int32_t* pos, const int32_t* cin, int32_t* cout, cudaStream_t s);
// The rows of V level by level: order[lvlptr[lev[i]] + rank[i]] = i (rank[i]:
// row i's place among the rows of its level).
cudaError_t level_order(int n, const int32_t* lev, const int32_t* rank, const int32_t* lvlptr, int32_t* order,
                        cudaStream_t s);

// t = V^-1 x by level scheduling on L: one block, a barrier between levels;
// t in level order (t[p] belongs to row xrow[p]).  warm: read all of the
// solve's data once first (for the first solve after L was built, whose data
// is cold on the solving SM).
cudaError_t trsv_levels_perm(const LevelCsr& L, bool cplx, const void* x, void* t, cudaStream_t s,
                             bool warm = false);

// Block-diagonal V: dense LU with partial pivoting of every diagonal block
// (blocks = runs of equal, non-decreasing block ids; at most 64 rows each).
struct BlockLu {
  int nblocks = 0;
  int32_t* bstart = nullptr;  // nblocks + 1 (capacity n + 1)
  void* lu = nullptr;         // block_lu_elems(n) scalars: column c of a block at (first row + c) * 64
  int32_t* piv = nullptr;     // n: block-local pivot row of every elimination step
};
size_t block_lu_elems(int n);
// Finds the blocks and factors them; `work` needs 2 n + scan_blocksums_size(n)
// int32; synchronises `s` once (the block count).  *status receives
// DEV_ST_BAD_INPUT (decreasing ids, or an entry of V outside its block),
// DEV_ST_CAPACITY (a block above 64 rows), DEV_ST_SINGULAR (a zero pivot).
cudaError_t block_prepare(int n, bool cplx, const int32_t* blk, const int32_t* Vcp, const int32_t* Vri,
                          const void* Vv, BlockLu& B, int32_t* work, uint32_t* status, cudaStream_t s);
// t = V^-1 x with the factored blocks.
cudaError_t block_solve(const BlockLu& B, bool cplx, const void* x, void* t, cudaStream_t s);
