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

// t = V^-1 x for upper (upper=true) or lower triangular CSR V.  Sync-free:
// each warp takes the next row by an atomic ticket, in dependency order, and
// waits (bounded) for the rows it needs.  `ready` holds one flag per row,
// `counter` one ticket counter (zeroed here); `gen` must differ from every
// value left in `ready` by earlier solves.  A wait that runs out sets
// DEV_ST_TIMEOUT in *status and the row is finished with what it has.
cudaError_t csr_trsv_syncfree(const Csr& V, bool cplx, bool upper, const void* x, void* t, uint32_t* ready,
                              int32_t* counter, uint32_t gen, uint32_t* status, cudaStream_t s);

// t = V^-1 x by level scheduling: rows grouped by their depth in the
// dependency graph of the triangular V (order = rows level by level,
// lvlptr[l]..lvlptr[l+1] the rows of level l, nlev levels), solved by one
// 1024-thread block with a barrier between levels; dinv = 1 / diag(V).
cudaError_t csr_trsv_levels(const Csr& V, bool cplx, int nlev, const int32_t* lvlptr, const int32_t* order,
                            const void* dinv, const void* x, void* t, cudaStream_t s);

// dinv[i] = 1 / V_ii (CSR V with a nonzero diagonal).
cudaError_t csr_diag_inverse(const Csr& V, bool cplx, void* dinv, cudaStream_t s);
