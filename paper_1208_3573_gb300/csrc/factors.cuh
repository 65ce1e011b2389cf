// The factorisation handle behind the opaque diaf_factors of include/diaf.h.
#pragma once

#include <vector>

#include "plan.cuh"
#include "sparse.cuh"

// Sets the thread's diaf_last_error() text (api.cu).
void diaf_set_last_error(const char* msg);

// Stream-ordered device allocations of the setup and apply paths, counted
// against the process-wide cap of diaf_set_device_memory_limit (api.cu).  A
// request beyond the cap fails with cudaErrorMemoryAllocation without
// reaching the allocator.
cudaError_t diaf_dev_alloc(void** p, size_t bytes, cudaStream_t s);
void diaf_dev_free(void* p, cudaStream_t s);

// Several arrays from one stream-ordered allocation (each start 256-byte
// aligned): add() records where each pointer goes and its size, and the
// owner's carve() makes one allocation and sets the pointers.  Fewer
// allocation calls on the host path of a setup, which otherwise outruns the
// small device operations between them.
struct Carve {
  struct Req {
    void** p;
    size_t bytes;
  };
  std::vector<Req> reqs;
  template <class T>
  void add(T** p, size_t count) {
    reqs.push_back({reinterpret_cast<void**>(p), sizeof(T) * (count > 0 ? count : 1)});
  }
  static size_t round(size_t b) { return (b + 255) & ~size_t(255); }
  size_t total() const {
    size_t t = 0;
    for (const Req& r : reqs) t += round(r.bytes);
    return t;
  }
  void assign(unsigned char* base) const {
    size_t off = 0;
    for (const Req& r : reqs) {
      *r.p = base + off;
      off += round(r.bytes);
    }
  }
};

struct diaf_factors {
  int device = 0;
  cudaStream_t stream = nullptr;
  int n = 0;
  int dtype = DIAF_F64, alg = DIAF_ALG_S, prec = DIAF_PREC_FP64, rule = DIAF_RULE_UPPER;
  int64_t nnz_w = 0, nnz_v = 0;
  int32_t *Wcp = nullptr, *Wri = nullptr, *Vcp = nullptr, *Vri = nullptr;
  void *Wv = nullptr, *Vv = nullptr;
  double* res = nullptr;
  uint32_t* flags = nullptr;
  uint32_t* status = nullptr;
  diaf_factor_info info{};
  std::vector<void*> owned;
  // CUDA events: [0] start, [1] numeric start, [2] end, [3 + 2b], [4 + 2b] around bucket b
  static constexpr int kEvents = 3 + 2 * kNumBuckets;
  cudaEvent_t ev[kEvents] = {};
  bool bucket_ran[kNumBuckets] = {};
  int32_t* fb_counts = nullptr;  // mixed precision: columns per bucket finished by the FP64 kernel
  // V's structure streamed to the host during the numeric pass (api.cu): set
  // while this factorisation owns the process's mapped mirror buffer
  bool mirror = false;
  int32_t* mir_cp = nullptr;    // host: V's column pointers (n + 1)
  int32_t* mir_ri = nullptr;    // host: V's row indices (nnz_v), filled by the column kernels
  uint32_t* mir_word = nullptr; // host: per column, set to mir_gen once column j's rows are there
  uint32_t mir_gen = 0;
  int32_t* mir_ri_dev = nullptr;    // the same row indices and words as the column kernels address them
  uint32_t* mir_word_dev = nullptr;
  // apply
  bool apply_ready = false;
  bool solve_cold = false;  // the level-ordered copies were just built: the next solve warms them
  // W's row-oriented copy is built on the library's side stream while V is
  // solved: wev[0] orders the side stream after F's stream, wev[1] marks the
  // end of F's side-stream work (the first SpMV waits for it: w_pending)
  cudaEvent_t wev[2] = {};
  bool w_pending = false;
  bool v_upper = true;
  Csr Wr;  // W's rows (V goes straight to its level-ordered form Vl)
  void* tbuf = nullptr;
  // level-scheduled V solve: V in level order, W's columns renumbered to it
  LevelCsr Vl;
  Csr Wl;
  // block-diagonal V (DIAF_RULE_BLOCK): dense LU of every diagonal block
  int32_t* blk = nullptr;        // block of every row (owned copy)
  bool v_block = false;
  BlockLu Vb;

  template <class T>
  cudaError_t alloc(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = diaf_dev_alloc(&q, sizeof(T) * (count > 0 ? count : 1), stream);
    if (e != cudaSuccess) return e;
    owned.push_back(q);
    *p = static_cast<T*>(q);
    return cudaSuccess;
  }
  cudaError_t carve(const Carve& c) {
    unsigned char* base = nullptr;
    cudaError_t e = alloc(&base, c.total());
    if (e == cudaSuccess) c.assign(base);
    return e;
  }
};
