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

// V in level order for the level-scheduled solve: position p holds row
// xrow[p] of V; the rows of level l (their depth in V's dependency graph) are
// positions lvlptr[l]..lvlptr[l+1]; rowptr/colidx/vals hold each row's
// off-diagonal entries with columns renumbered to positions, scaled by the
// row's 1 / diag; dinv = 1 / diag.
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

// L's row layout from the host's level walk (device arrays): row i of V goes
// to position pos[i] = lvlptr[lev[i]] + rank[i] (xrow[pos[i]] = i), and
// rowptr (n + 1) counts rcnt[i] off-diagonal entries at that position.  work
// needs n + scan_blocksums_size(n) int32.
cudaError_t level_place(int n, const int32_t* lev, const int32_t* rank, const int32_t* rcnt, const int32_t* lvlptr,
                        int32_t* pos, int32_t* xrow, int32_t* work, int32_t* rowptr, cudaStream_t s);

// L's entries straight from V's columns (cp, ri, v: V in CSC): entry e =
// (i, j) of column j, i != j, goes to L.rowptr[pos[i]] + slot[e] with column
// pos[j] and value v_ij / v_ii (v_ii at entry dpos[i]); the diagonal gives
// L.dinv[pos[j]] = 1 / v_jj.  *zflag (zeroed by the caller) becomes nonzero
// when a diagonal value is zero or not a number.
cudaError_t level_fill(int n, bool cplx, const int32_t* cp, const int32_t* ri, const void* v, const int32_t* dpos,
                       const int32_t* slot, const int32_t* pos, LevelCsr& L, uint32_t* zflag, cudaStream_t s);

// cout[e] = pos[cin[e]] (column indices renumbered to level positions).
cudaError_t remap_columns(int64_t nnz, const int32_t* pos, const int32_t* cin, int32_t* cout, cudaStream_t s);

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
