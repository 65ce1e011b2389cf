// C ABI of the DIAF library: argument checks, the symbolic pass, bucketed
// numeric launches, output ownership, and the preconditioner apply.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "factors.cuh"
#include "launch.cuh"
#include "plan.cuh"
#include "sparse.cuh"

#ifdef DIAF_PREP_TIMING
#include <chrono>
namespace {
struct PrepTimer {
  const char* tag;
  explicit PrepTimer(const char* t) : tag(t) { for (auto& e : ev) cudaEventCreate(&e); }
  cudaEvent_t ev[8];
  double host[8];
  int ne = 0, nh = 0;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  void dev(cudaStream_t s) { cudaEventRecord(ev[ne++], s); }
  void hst() { host[nh++] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count(); }
  ~PrepTimer() {
    cudaDeviceSynchronize();
    fprintf(stderr, "%s dev:", tag);
    for (int i = 1; i < ne; ++i) { float ms = 0; cudaEventElapsedTime(&ms, ev[0], ev[i]); fprintf(stderr, " %.3f", ms); }
    fprintf(stderr, " | host:");
    for (int i = 0; i < nh; ++i) fprintf(stderr, " %.3f", host[i]);
    fprintf(stderr, "\n");
    for (auto& e : ev) cudaEventDestroy(e);
  }
};
}  // namespace
#define PT_DEV(s) pt.dev(s)
#define PT_HOST() pt.hst()
#else
#define PT_DEV(s) (void)0
#define PT_HOST() (void)0
#endif

static std::atomic<long long> g_launches{0};
#ifdef DIAF_PHASE_TIMING
static unsigned long long* g_phase = nullptr;  // device, 32 counters
extern "C" int diaf_phase_cycles(unsigned long long* out, int reset) {
  if (!g_phase) {
    for (int i = 0; i < 32; ++i) out[i] = 0;
    return 0;
  }
  if (cudaMemcpy(out, g_phase, sizeof(unsigned long long) * 32, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  if (reset && cudaMemset(g_phase, 0, sizeof(unsigned long long) * 32) != cudaSuccess) return 1;
  return 0;
}
#endif
static thread_local std::string g_last_error;
void diaf_set_last_error(const char* msg) { g_last_error = msg; }

namespace {
// Device bytes held by the setup and apply paths, and the cap on them.
std::mutex g_mem_mu;
std::unordered_map<void*, size_t> g_mem_held;
size_t g_mem_total = 0;
size_t g_mem_cap = 0;  // 0: no cap

// The library's own stream-ordered memory pool per device.  Its release
// threshold is unlimited, so memory freed by one setup stays in the pool
// for the next instead of going back to the driver at every synchronisation
// (the default pool's behaviour), which would make every allocation map
// fresh pages.  The pool holds the high-water mark of the library's use.
constexpr int kPoolDevices = 64;
cudaMemPool_t g_pool[kPoolDevices] = {};

cudaError_t library_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kPoolDevices) return cudaErrorInvalidDevice;
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}
}  // namespace

cudaError_t diaf_dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mem_mu);
    if (g_mem_cap && g_mem_total + bytes > g_mem_cap) return cudaErrorMemoryAllocation;
    g_mem_total += bytes;  // reserved before the call, so concurrent requests see it
  }
  void* q = nullptr;
  cudaMemPool_t pool = nullptr;
  cudaError_t e;
  {
    std::lock_guard<std::mutex> lock(g_mem_mu);
    e = library_pool(&pool);
  }
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&q, bytes, pool, s);
  std::lock_guard<std::mutex> lock(g_mem_mu);
  if (e != cudaSuccess) {
    g_mem_total -= bytes;
    return e;
  }
  g_mem_held[q] = bytes;
  *p = q;
  return cudaSuccess;
}

void diaf_dev_free(void* p, cudaStream_t s) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lock(g_mem_mu);
    auto it = g_mem_held.find(p);
    if (it != g_mem_held.end()) {
      g_mem_total -= it->second;
      g_mem_held.erase(it);
    }
  }
  cudaFreeAsync(p, s);
}
void diaf_note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

namespace {

diaf_status fail(diaf_status st, const std::string& why) {
  g_last_error = why;
  return st;
}

diaf_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? DIAF_ENOMEM : DIAF_ECUDA;
}

#define DIAF_CU(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// Stream-ordered device allocations released together.
struct Pool {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Pool(cudaStream_t st) : s(st) {}
  template <class T>
  cudaError_t get(T** p, size_t count) {
    size_t bytes = sizeof(T) * (count > 0 ? count : 1);
    void* q = nullptr;
    cudaError_t e = diaf_dev_alloc(&q, bytes, s);
    if (e != cudaSuccess) return e;
    ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return cudaSuccess;
  }
  cudaError_t carve(const Carve& c) {
    unsigned char* base = nullptr;
    cudaError_t e = get(&base, c.total());
    if (e == cudaSuccess) c.assign(base);
    return e;
  }
  void release() {
    for (void* p : ptrs) diaf_dev_free(p, s);
    ptrs.clear();
  }
  ~Pool() { release(); }
};

// Per-device tables of the library (event cache, side streams) have this
// many slots; devices beyond them go without (fresh events, no side stream).
constexpr int kDeviceSlots = 64;

// CUDA events of the factor handles, recycled per device: a setup takes
// kEvents of them, and creating them anew each time cost host time in front
// of the setup's first device operation.
struct EventCache {
  std::mutex mu;
  std::vector<cudaEvent_t> free[kDeviceSlots];
};
EventCache g_events;

cudaError_t event_get(cudaEvent_t* e, int dev) {
  if (dev >= 0 && dev < kDeviceSlots) {
    std::lock_guard<std::mutex> lock(g_events.mu);
    std::vector<cudaEvent_t>& v = g_events.free[dev];
    if (!v.empty()) {
      *e = v.back();
      v.pop_back();
      return cudaSuccess;
    }
  }
  return cudaEventCreate(e);
}

void event_put(cudaEvent_t e, int dev) {
  if (!e) return;
  if (dev >= 0 && dev < kDeviceSlots) {
    std::lock_guard<std::mutex> lock(g_events.mu);
    if (g_events.free[dev].size() < 256) {
      g_events.free[dev].push_back(e);
      return;
    }
  }
  cudaEventDestroy(e);
}

diaf_status check_device() {
  int dev = 0, n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) return fail(DIAF_ECUDA, "no CUDA device");
  cudaGetDevice(&dev);
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return fail(DIAF_ECUDA, "this library is built for sm_103 (GB300) only");
  return DIAF_OK;
}

// ---- V's structure streamed to the host during the numeric pass
// One pinned buffer per process, mapped into the devices' address space: one
// word per column first, then V's column pointers (copied after the symbolic
// pass), then V's row indices, which the column kernels write as each column
// becomes final before they set the column's word to the owner's generation
// (system-scope release).  One factorisation at a time owns it, so the first
// apply can build the level schedule from the columns as they arrive, while
// the numeric pass still runs; a factorisation that finds it taken goes
// without (its apply copies V's structure after the numeric pass).
struct Mirror {
  std::mutex mu;
  unsigned char* buf = nullptr;
  unsigned char* dbuf = nullptr;  // buf's device address
  size_t cap = 0;    // bytes
  size_t words = 0;  // columns the word area holds (zeroed when allocated)
  uint32_t gen = 0;
  bool busy = false;
};
Mirror g_mirror;
std::atomic<long long> g_prep_streamed{0}, g_prep_copied{0};

// Takes the mirror for F (F->n, F->nnz_v known) when it is free; grows it
// when it is too small.  Returns false (F without a mirror) when it is taken
// or cannot be had.
bool mirror_acquire(diaf_factors* F) {
  const size_t n = (size_t)F->n, nnz = (size_t)F->nnz_v;
  std::lock_guard<std::mutex> lock(g_mirror.mu);
  if (g_mirror.busy) return false;
  auto bytes_for = [&](size_t words) { return sizeof(uint32_t) * words + sizeof(int32_t) * (words + 1 + nnz); };
  if (n > g_mirror.words || bytes_for(g_mirror.words) > g_mirror.cap) {
    // no kernel writes into the old buffer: every owner released it only
    // after reading all of its columns or synchronising its stream
    if (g_mirror.buf) cudaFreeHost(g_mirror.buf);
    g_mirror.buf = nullptr;
    g_mirror.cap = g_mirror.words = 0;
    const size_t words = n + n / 4;
    const size_t want = bytes_for(words) + sizeof(int32_t) * (nnz / 4);
    if (cudaHostAlloc((void**)&g_mirror.buf, want, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
      (void)cudaGetLastError();
      g_mirror.buf = nullptr;
      return false;
    }
    if (cudaHostGetDevicePointer((void**)&g_mirror.dbuf, g_mirror.buf, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      cudaFreeHost(g_mirror.buf);
      g_mirror.buf = g_mirror.dbuf = nullptr;
      return false;
    }
    std::memset(g_mirror.buf, 0, sizeof(uint32_t) * words);
    g_mirror.cap = want;
    g_mirror.words = words;
  }
  if (++g_mirror.gen == 0) {  // wrapped: no word may hold a stale generation equal to a new one
    std::memset(g_mirror.buf, 0, sizeof(uint32_t) * g_mirror.words);
    g_mirror.gen = 1;
  }
  F->mir_word = reinterpret_cast<uint32_t*>(g_mirror.buf);
  F->mir_cp = reinterpret_cast<int32_t*>(F->mir_word + g_mirror.words);
  F->mir_ri = F->mir_cp + (n + 1);
  F->mir_word_dev = reinterpret_cast<uint32_t*>(g_mirror.dbuf);
  F->mir_ri_dev = reinterpret_cast<int32_t*>(F->mir_word_dev + g_mirror.words) + (n + 1);
  F->mir_gen = g_mirror.gen;
  F->mirror = true;
  g_mirror.busy = true;
  return true;
}

// The library's side stream on the current device (created on first use;
// nullptr when it cannot be had, and the caller stays on its own stream).
cudaStream_t side_stream() {
  static std::mutex mu;
  static cudaStream_t st[kDeviceSlots] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDeviceSlots) {
    (void)cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!st[dev] && cudaStreamCreateWithFlags(&st[dev], cudaStreamNonBlocking) != cudaSuccess) {
    (void)cudaGetLastError();
    st[dev] = nullptr;
  }
  return st[dev];
}

// Gives the mirror back.  The caller has read every column of it, or has
// synchronised F's stream: none of F's kernels writes into it any more.
void mirror_release(diaf_factors* F) {
  if (!F->mirror) return;
  std::lock_guard<std::mutex> lock(g_mirror.mu);
  g_mirror.busy = false;
  F->mirror = false;
}

}  // namespace

extern "C" {

const char* diaf_status_string(diaf_status s) {
  switch (s) {
    case DIAF_OK: return "ok";
    case DIAF_EINVAL: return "invalid argument";
    case DIAF_ENOMEM: return "out of device memory";
    case DIAF_ECUDA: return "CUDA error";
    case DIAF_ENUMERIC: return "non-finite values";
    case DIAF_ETIMEOUT: return "device wait timed out";
    case DIAF_EUNSUPPORTED: return "tile beyond the compiled capacity";
  }
  return "unknown status";
}

const char* diaf_last_error(void) { return g_last_error.c_str(); }

void diaf_free(diaf_factors* F) {
  if (!F) return;
  if (F->mirror) {  // an apply never read it: the numeric pass may still write into it
    (void)cudaStreamSynchronize(F->stream);
    mirror_release(F);
  }
  if (F->wev[1]) (void)cudaStreamWaitEvent(F->stream, F->wev[1], 0);  // F's side-stream work first
  for (cudaEvent_t e : F->wev)
    if (e) cudaEventDestroy(e);
  for (void* p : F->owned) diaf_dev_free(p, F->stream);
  for (cudaEvent_t e : F->ev) event_put(e, F->device);
  delete F;
}

long long diaf_launch_count(void) { return g_launches.load(); }

void diaf_apply_prep_counts(int64_t* streamed, int64_t* copied) {
  if (streamed) *streamed = g_prep_streamed.load();
  if (copied) *copied = g_prep_copied.load();
}

diaf_status diaf_set_device_memory_limit(int64_t bytes) {
  if (bytes < 0) return fail(DIAF_EINVAL, "the limit must be >= 0 (0: no limit)");
  std::lock_guard<std::mutex> lock(g_mem_mu);
  g_mem_cap = static_cast<size_t>(bytes);
  return DIAF_OK;
}

diaf_status diaf_release_pool_memory(void) {
  g_last_error.clear();
  cudaMemPool_t pool = nullptr;
  cudaError_t e;
  {
    std::lock_guard<std::mutex> lock(g_mem_mu);
    e = library_pool(&pool);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
  if (e != cudaSuccess) return cuda_fail(e, "diaf_release_pool_memory");
  return DIAF_OK;
}

int64_t diaf_device_memory_in_use(void) {
  std::lock_guard<std::mutex> lock(g_mem_mu);
  return static_cast<int64_t>(g_mem_total);
}

diaf_status diaf_factor_fallbacks(const diaf_factors* F, int32_t* counts, int32_t nb) {
  if (!F || !counts || nb < kNumBuckets) return fail(DIAF_EINVAL, "need a handle and room for n_buckets counts");
  for (int i = 0; i < nb; ++i) counts[i] = 0;
  if (!F->fb_counts) return DIAF_OK;
  DIAF_CU(cudaMemcpyAsync(counts, F->fb_counts, sizeof(int32_t) * kNumBuckets, cudaMemcpyDeviceToHost, F->stream));
  DIAF_CU(cudaStreamSynchronize(F->stream));

  return DIAF_OK;
}

diaf_status diaf_factor_timings(const diaf_factors* F, float* ms, int32_t nms) {
  if (!F || !ms || nms < 2 + kNumBuckets) return fail(DIAF_EINVAL, "need a handle and room for 2 + n_buckets values");
  for (int i = 0; i < nms; ++i) ms[i] = 0.0f;
  if (!F->ev[0]) return DIAF_OK;
  DIAF_CU(cudaEventSynchronize(F->ev[2]));
  DIAF_CU(cudaEventElapsedTime(&ms[0], F->ev[0], F->ev[2]));
  DIAF_CU(cudaEventElapsedTime(&ms[1], F->ev[1], F->ev[2]));
  for (int b = 0; b < kNumBuckets; ++b)
    if (F->bucket_ran[b]) DIAF_CU(cudaEventElapsedTime(&ms[2 + b], F->ev[3 + 2 * b], F->ev[4 + 2 * b]));
  return DIAF_OK;
}

}  // extern "C"

namespace {

// Everything the numeric pass needs; built by symbolic_pass.
struct NumericPlan {
  ColArgs ca{};
  int32_t* bucket_list = nullptr;
  int32_t* bucket_count = nullptr;
  int32_t* work = nullptr;      // kWorkCounters: per bucket the main, FP64 hand-back and deferred
                                // launches' work counters, then the defer count
  int32_t* fb_list = nullptr;   // mixed: columns handed to the FP64 kernels
  int32_t* fb_count = nullptr;
  int h_bc[kNumBuckets] = {0};
  CtaScratch cs{};
  int cta_grid = 0;
  int cta_grid_mixed = 0;  // mixed large-tile kernel (0: not used)
  bool mixed = false, cplx = false;
  int alg = DIAF_ALG_S, dtype = DIAF_F64, n = 0;
  int wpb[2] = {0, 0};
  // bucket 0 of real mixed DIAF-S: four lanes per column, deferred columns to the warp kernel
  bool thread_cols = false;
  ThreadArgs ta{};
  ThreadShape tsh{};
};
constexpr int kWorkCounters = 3 * kNumBuckets + 1;

diaf_status check_args(const diaf_csc* A, const diaf_pattern* PW, const diaf_vspec* V, int32_t alg, int32_t prec,
                       const diaf_tuning* tuning) {
  if (!A || !PW || !V) return fail(DIAF_EINVAL, "A, PW and V must be non-NULL");
  if (alg != DIAF_ALG_Q && alg != DIAF_ALG_S) return fail(DIAF_EINVAL, "alg must be DIAF_ALG_Q or DIAF_ALG_S");
  if (prec != DIAF_PREC_FP64 && prec != DIAF_PREC_MIXED32) return fail(DIAF_EINVAL, "unknown precision");
  if (A->dtype != DIAF_F64 && A->dtype != DIAF_C128) return fail(DIAF_EINVAL, "unknown dtype");
  if (A->n < 0 || PW->n != A->n) return fail(DIAF_EINVAL, "PW->n must equal A->n >= 0");
  if (A->nnz < 0 || PW->nnz < 0 || A->nnz >= (1ll << 31) || PW->nnz >= (1ll << 31))
    return fail(DIAF_EINVAL, "nnz out of range");
  if (V->rule < DIAF_RULE_FIXED || V->rule > DIAF_RULE_BLOCK) return fail(DIAF_EINVAL, "unknown V rule");
  if (V->rule == DIAF_RULE_BLOCK && A->n > 0 && !V->blocks)
    return fail(DIAF_EINVAL, "DIAF_RULE_BLOCK needs the block of every row (V->blocks)");
  if (V->rule == DIAF_RULE_FIXED && (!V->fixed || V->fixed->n != A->n || !V->fixed->colptr))
    return fail(DIAF_EINVAL, "fixed V pattern missing or of the wrong size");
  if (A->n > 0 && (!A->colptr || !PW->colptr || (A->nnz > 0 && (!A->rowidx || !A->vals)) ||
                   (PW->nnz > 0 && !PW->rowidx)))
    return fail(DIAF_EINVAL, "NULL array in A or PW");
  if (tuning) {
    if (tuning->m_edge0 < 0 || tuning->m_edge0 > 32 || tuning->m_edge1 < 0 || tuning->m_edge1 > 64)
      return fail(DIAF_EINVAL, "tuning: m_edge0 must be in 0..32 and m_edge1 in 0..64");
    for (int b = 0; b < 2; ++b)
      if (tuning->warps_per_block[b] < 0 || tuning->warps_per_block[b] > 8)
        return fail(DIAF_EINVAL, "tuning: warps_per_block must be in 0..8");
    if (tuning->small_tiles < 0 || tuning->small_tiles > 2) return fail(DIAF_EINVAL, "tuning: small_tiles must be 0, 1 or 2");
    if (tuning->large_tiles < 0 || tuning->large_tiles > 2) return fail(DIAF_EINVAL, "tuning: large_tiles must be 0, 1 or 2");
  }
  return check_device();
}

// Symbolic pass: input checks, row unions, V counts, buckets; allocates the
// outputs into F and the numeric pass's scratch into `scratch`.  Synchronises
// `s` (twice: after the input check and to size V).
diaf_status symbolic_pass(const diaf_csc* A, const diaf_pattern* PW, const diaf_vspec* V, int32_t alg, int32_t prec,
                          const diaf_tuning* tuning, cudaStream_t s, diaf_factors* F, Pool& pool, NumericPlan& np) {
#ifdef DIAF_PREP_TIMING
  PrepTimer pt("symbolic");
#endif
  PT_DEV(s);
  PT_HOST();
  const int n = A->n;
  const bool cplx = A->dtype == DIAF_C128;
  const size_t esz = cplx ? 16 : 8;
  F->stream = s;
  cudaGetDevice(&F->device);
  F->n = n;
  F->dtype = A->dtype;
  F->alg = alg;
  F->prec = prec;
  F->rule = V->rule;
  if (V->rule == DIAF_RULE_BLOCK && n > 0) {  // the apply needs the blocks after the caller's buffer is gone
    DIAF_CU(F->alloc(&F->blk, n));
    DIAF_CU(cudaMemcpyAsync(F->blk, V->blocks, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  }
  F->nnz_w = PW->nnz;
  np.n = n; np.alg = alg; np.dtype = A->dtype; np.cplx = cplx;
  np.mixed = prec == DIAF_PREC_MIXED32;
  np.wpb[0] = tuning ? tuning->warps_per_block[0] : 0;
  np.wpb[1] = tuning ? tuning->warps_per_block[1] : 0;

  uint32_t* status;
  int32_t *stats, *big_count;
  int64_t* bs64;
  int32_t* bs32;
  PlanArgs pa{};
  DIAF_CU(F->alloc(&status, 1));
  F->status = status;
  // the symbolic scratch in one allocation; the small counters in one block
  // (stats[4], then the bucket counts, then the large-tile count: one memset)
  {
    Carve c;
    c.add(&stats, 4 + kNumBuckets + 1);
    c.add(&np.work, kWorkCounters);
    c.add(&pa.k, n);
    c.add(&pa.E, n);
    c.add(&pa.Eoff, n + 1);
    c.add(&pa.m, n);
    c.add(&pa.l, n);
    c.add(&pa.jin, n);
    c.add(&np.bucket_list, (size_t)kNumBuckets * n);
    c.add(&pa.big_list, n);
    c.add(&bs64, scan_blocksums_size(n));
    c.add(&bs32, scan_blocksums_size(n));
    DIAF_CU(pool.carve(c));
  }
  np.bucket_count = stats + 4;
  big_count = stats + 4 + kNumBuckets;
  DIAF_CU(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
  DIAF_CU(cudaMemsetAsync(stats, 0, sizeof(int32_t) * (4 + kNumBuckets + 1), s));

  // ---- input checks on the device (sorted, in range)
  DIAF_CU(check_csc(n, A->colptr, A->rowidx, A->nnz, status, s));
  DIAF_CU(check_csc(n, PW->colptr, PW->rowidx, PW->nnz, status, s));
  if (V->rule == DIAF_RULE_FIXED) DIAF_CU(check_csc(n, V->fixed->colptr, V->fixed->rowidx, V->fixed->nnz, status, s));

  // ---- symbolic pass 1: k_j, E_j
  pa.n = n;
  pa.Acp = A->colptr; pa.Ari = A->rowidx;
  pa.Wcp = PW->colptr; pa.Wri = PW->rowidx;
  pa.rule = V->rule;
  pa.Vfcp = V->rule == DIAF_RULE_FIXED ? V->fixed->colptr : nullptr;
  pa.Vfri = V->rule == DIAF_RULE_FIXED ? V->fixed->rowidx : nullptr;
  pa.budget = V->budget;
  pa.blk = V->rule == DIAF_RULE_BLOCK ? V->blocks : nullptr;
  pa.edge_m0 = tuning && tuning->m_edge0 > 0 ? tuning->m_edge0 : 32;
  pa.edge_m1 = tuning && tuning->m_edge1 > 0 ? tuning->m_edge1 : 64;
  pa.bucket_list = np.bucket_list;
  pa.bucket_count = np.bucket_count;
  pa.big_count = big_count;
  pa.stats = stats;
  pa.status = status;

  uint32_t h_status = 0;
  int64_t h_Etot = 0;
  if (n > 0) {
    // the count kernel reads J_j only when the input check (earlier on the
    // stream) passed: it tests the status flag itself, so no sync here
    DIAF_CU(plan_count(pa, s));
    DIAF_CU(exclusive_scan_i32_to_i64(pa.E, pa.Eoff, n, bs64, s));
    DIAF_CU(cudaMemcpyAsync(&h_Etot, pa.Eoff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    DIAF_CU(cudaMemcpyAsync(&h_status, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    PT_DEV(s);
    PT_HOST();
    DIAF_CU(cudaStreamSynchronize(s));
    PT_HOST();
    if (h_status & DEV_ST_BAD_INPUT) return fail(DIAF_EINVAL, "unsorted or out-of-range indices in A, PW or V");
  }
  DIAF_CU(pool.get(&pa.rows, (size_t)h_Etot));
  DIAF_CU(F->alloc(&F->Vcp, n + 1));
  if (n > 0) {
    DIAF_CU(plan_rows(pa, s));
    DIAF_CU(exclusive_scan_i32(pa.l, F->Vcp, n, bs32, s));
  } else {
    DIAF_CU(cudaMemsetAsync(F->Vcp, 0, sizeof(int32_t), s));
  }
  int32_t h_nnzv = 0, h_blk[4 + kNumBuckets] = {0};  // stats, then the bucket counts
  int32_t* const h_stats = h_blk;
  if (n > 0) {
    DIAF_CU(cudaMemcpyAsync(&h_nnzv, F->Vcp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    DIAF_CU(cudaMemcpyAsync(h_blk, stats, sizeof(h_blk), cudaMemcpyDeviceToHost, s));
    DIAF_CU(cudaMemcpyAsync(&h_status, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    PT_DEV(s);
    PT_HOST();
    DIAF_CU(cudaStreamSynchronize(s));
    PT_HOST();
  }
  for (int b = 0; b < kNumBuckets; ++b) np.h_bc[b] = h_blk[4 + b];
  if (h_status & DEV_ST_CAPACITY)
    return fail(DIAF_EUNSUPPORTED, "a column needs more than 4096 gathered entries or a tile beyond 1024 x 64");
  F->nnz_v = h_nnzv;
  F->info.n = n;
  F->info.dtype = A->dtype;
  F->info.alg = alg;
  F->info.prec = prec;
  F->info.nnz_w = PW->nnz;
  F->info.nnz_v = h_nnzv;
  F->info.max_k = h_stats[0];
  F->info.max_m = h_stats[1];
  F->info.max_l = h_stats[2];
  F->info.n_buckets = kNumBuckets;
  for (int b = 0; b < kNumBuckets; ++b) F->info.bucket_cols[b] = np.h_bc[b];

  // ---- outputs
  {
    Carve c;
    c.add(&F->Wcp, n + 1);
    c.add(&F->Wri, PW->nnz);
    c.add((char**)&F->Wv, esz * PW->nnz);
    c.add(&F->Vri, h_nnzv);
    c.add((char**)&F->Vv, esz * h_nnzv);
    c.add(&F->res, n);
    c.add(&F->flags, n);
    if (prec == DIAF_PREC_MIXED32) c.add(&F->fb_counts, kNumBuckets);
    DIAF_CU(F->carve(c));
  }
  DIAF_CU(cudaMemcpyAsync(F->Wcp, PW->colptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToDevice, s));
  if (PW->nnz > 0)
    DIAF_CU(cudaMemcpyAsync(F->Wri, PW->rowidx, sizeof(int32_t) * PW->nnz, cudaMemcpyDeviceToDevice, s));

  // ---- numeric-pass arguments and scratch
  Carve nc;
  ColArgs& ca = np.ca;
  ca.n = n;
  ca.Acp = A->colptr; ca.Ari = A->rowidx; ca.Av = A->vals;
  ca.Wcp = PW->colptr; ca.Wri = PW->rowidx;
  ca.Eoff = pa.Eoff; ca.rows = pa.rows; ca.m = pa.m; ca.l = pa.l; ca.jin = pa.jin;
  ca.rule = V->rule; ca.Vfcp = pa.Vfcp; ca.Vfri = pa.Vfri;
  ca.blk = pa.blk;
  ca.Vcp = F->Vcp;
  ca.tie_tol = V->tie_tol > 0 ? V->tie_tol : 1e-9;
  ca.stab_tol = (alg == DIAF_ALG_Q && V->stab_tol > 0) ? V->stab_tol : 0.0;
  ca.stab_r = V->stab_r > 0 ? V->stab_r : 2.0;
  ca.Wv = F->Wv; ca.Vri = F->Vri; ca.Vv = F->Vv;
  ca.res = F->res; ca.flags = F->flags; ca.status = status;
#ifdef DIAF_PHASE_TIMING
  if (!g_phase) {
    DIAF_CU(cudaMalloc(&g_phase, sizeof(unsigned long long) * 32));
    DIAF_CU(cudaMemset(g_phase, 0, sizeof(unsigned long long) * 32));
  }
  ca.phase = g_phase;
#endif
  if (np.mixed) {
    nc.add(&np.fb_list, (size_t)kNumBuckets * n);
    nc.add(&np.fb_count, kNumBuckets);
    // the warp buckets' FP64 tiles: one per warp of the larger persistent grid
    // (the buckets run one after the other on the stream)
    size_t tiles = 0;
    for (int b = 0; b < 2; ++b) {
      if (np.h_bc[b] == 0) continue;
      const size_t t = np.cplx ? mixed_tile_scratch_c64(b, alg, np.h_bc[b], np.wpb[b])
                               : mixed_tile_scratch_f32(b, alg, np.h_bc[b], np.wpb[b]);
      if (t > tiles) tiles = t;
    }
    if (tiles > 0) nc.add((char**)&ca.tile_scratch, tiles);
    // bucket 0 of real DIAF-S: four lanes per column (unless the tuning asks for the warp kernel)
    const int small = tuning ? tuning->small_tiles : 0;
    if (!np.cplx && alg == DIAF_ALG_S && np.h_bc[0] > 0 && small != 2 && V->rule != DIAF_RULE_FIXED) {
      const int M = h_stats[1] < pa.edge_m0 ? h_stats[1] : pa.edge_m0;
      const int K = h_stats[0] < kThreadKMax ? h_stats[0] : kThreadKMax;
      if (M >= 1 && K >= 1) {
        DIAF_CU(thread_columns_shape(M, K, np.h_bc[0], &np.tsh));
        np.ta.M = M;
        np.ta.K = K;
        np.ta.arena = thread_arena_floats(M, K);
        np.ta.nquads = np.tsh.nquads;
        nc.add(&np.ta.slab, (size_t)np.tsh.nquads * thread_slab_doubles(M, K));
        nc.add(&np.ta.defer_list, np.h_bc[0]);
        np.ta.defer_count = np.work + 3 * kNumBuckets;
        np.thread_cols = np.tsh.grid > 0;
      }
    }
  }
  const int bl = kNumBuckets - 1;
  if (np.h_bc[bl] > 0) {
    // large tiles: one CTA per column, FP64 in both precisions (tiles in scratch slabs)
    const int mk = h_stats[1] > h_stats[0] ? h_stats[1] : h_stats[0];
    np.cs.ldm = (mk + 31) / 32 * 32;
    np.cs.kcap = h_stats[0] > 0 ? h_stats[0] : 1;
    np.cs.gram = (tuning && tuning->large_tiles == 2) ? 0 : 1;  // the tensor-core Gram path unless asked off
    np.cta_grid = cta_columns_grid(A->dtype, alg, np.cs.ldm, np.h_bc[bl]);
    if (np.cta_grid <= 0) return fail(DIAF_EUNSUPPORTED, "large-tile kernel does not fit this tile size");
    // the mixed kernel needs less shared memory: its own occupancy-sized grid
    np.cta_grid_mixed = np.mixed ? cta_columns_grid_mixed(A->dtype, alg, np.cs.ldm, np.h_bc[bl]) : 0;
    const int slabs = np.cta_grid > np.cta_grid_mixed ? np.cta_grid : np.cta_grid_mixed;
    nc.add((char**)&np.cs.slab, (size_t)slabs * 2 * np.cs.ldm * np.cs.kcap * esz);
  }
  if (!nc.reqs.empty()) DIAF_CU(pool.carve(nc));  // the numeric pass's scratch, one allocation
  PT_DEV(s);
  PT_HOST();
  return DIAF_OK;
}

// Numeric pass: work-counter resets and one launch per non-empty bucket (plus
// the FP64 kernel over the columns the mixed kernel handed back).  Only
// stream work: no allocation, no synchronisation (graph-capturable).
diaf_status enqueue_numeric(diaf_factors* F, NumericPlan& np, cudaStream_t s, bool events) {
  const int n = np.n;
  DIAF_CU(cudaMemsetAsync(np.work, 0, sizeof(int32_t) * kWorkCounters, s));
  if (np.mixed) DIAF_CU(cudaMemsetAsync(np.fb_count, 0, sizeof(int32_t) * kNumBuckets, s));
  ColArgs ca = np.ca;
  auto fp64_launch = [&](int b, const ColArgs& c, int hint) {
    const int w = b < 2 ? np.wpb[b] : 0;
    return np.cplx ? launch_columns_c128(b, np.alg, c, hint, w, s) : launch_columns_f64(b, np.alg, c, hint, w, s);
  };
  for (int b = 0; b < kNumBuckets; ++b) {
    if (np.h_bc[b] == 0) continue;
    ca.list = np.bucket_list + (size_t)b * n;
    ca.list_count = np.bucket_count + b;
    ca.work_counter = np.work + b;
    ca.extra_flags = 0;
    if (events) DIAF_CU(cudaEventRecord(F->ev[3 + 2 * b], s));
    cudaError_t e;
    if (b == kNumBuckets - 1) {
      e = cudaErrorNotSupported;
      if (np.mixed) {
        ca.fb_list = np.fb_list + (size_t)b * n;
        ca.fb_count = np.fb_count + b;
        e = np.cta_grid_mixed > 0 ? launch_columns_cta_mixed(np.dtype, np.alg, ca, np.cs, np.cta_grid_mixed, s)
                                  : cudaErrorNotSupported;
        if (e == cudaSuccess) {  // the FP64 kernel finishes the handed-back columns
          ColArgs cf = ca;
          cf.list = ca.fb_list;
          cf.list_count = ca.fb_count;
          cf.work_counter = np.work + kNumBuckets + b;
          cf.extra_flags = DIAF_FLAG_FP64_FALLBACK;
          e = launch_columns_cta(np.dtype, np.alg, cf, np.cs, np.cta_grid, s);
        }
      }
      if (e == cudaErrorNotSupported) {  // every large column on the FP64 kernel
        (void)cudaGetLastError();
        ca.extra_flags = np.mixed ? DIAF_FLAG_FP64_FALLBACK : 0;
        if (np.mixed) DIAF_CU(cudaMemcpyAsync(np.fb_count + b, np.bucket_count + b, sizeof(int32_t),
                                              cudaMemcpyDeviceToDevice, s));
        e = launch_columns_cta(np.dtype, np.alg, ca, np.cs, np.cta_grid, s);
      }
    } else if (np.mixed) {
      ca.fb_list = np.fb_list + (size_t)b * n;
      ca.fb_count = np.fb_count + b;
      e = cudaSuccess;
      if (b == 0 && np.thread_cols) {
        // four lanes per column; the columns it defers run in the warp kernel
        e = launch_columns_thread_f32(ca, np.ta, np.tsh, s);
        ca.list = np.ta.defer_list;
        ca.list_count = np.ta.defer_count;
        ca.work_counter = np.work + 2 * kNumBuckets + b;
      }
      if (e == cudaSuccess)
        e = np.cplx ? launch_columns_mixed_c64(b, np.alg, ca, np.h_bc[b], np.wpb[b], s)
                    : launch_columns_mixed_f32(b, np.alg, ca, np.h_bc[b], np.wpb[b], s);
      if (e == cudaSuccess) {
        // the FP64 kernel finishes the columns the mixed kernel handed back
        ColArgs cf = ca;
        cf.list = ca.fb_list;
        cf.list_count = ca.fb_count;
        cf.work_counter = np.work + kNumBuckets + b;
        cf.extra_flags = DIAF_FLAG_FP64_FALLBACK;
        e = fp64_launch(b, cf, np.h_bc[b]);
      }
    } else {
      e = fp64_launch(b, ca, np.h_bc[b]);
    }
    if (e == cudaErrorNotSupported)
      return fail(DIAF_EUNSUPPORTED, "bucket " + std::to_string(b) + " has no kernel for this configuration yet");
    if (e != cudaSuccess) return cuda_fail(e, "column kernel launch");
    if (events) DIAF_CU(cudaEventRecord(F->ev[4 + 2 * b], s));
    F->bucket_ran[b] = true;
  }
  if (np.mixed) DIAF_CU(cudaMemcpyAsync(F->fb_counts, np.fb_count, sizeof(int32_t) * kNumBuckets,
                                        cudaMemcpyDeviceToDevice, s));
  return DIAF_OK;
}

}  // namespace

struct diaf_plan {
  diaf_factors* F = nullptr;
  Pool* scratch = nullptr;
  NumericPlan np;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

diaf_status diaf_factor_tuned(const diaf_csc* A, const diaf_pattern* PW, const diaf_vspec* V, int32_t alg,
                              int32_t prec, const diaf_tuning* tuning, void* stream, diaf_factors** out) {
  g_last_error.clear();
  if (!out) return fail(DIAF_EINVAL, "out is NULL");
  *out = nullptr;
  diaf_status st = check_args(A, PW, V, alg, prec, tuning);
  if (st != DIAF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto F = new diaf_factors();
  F->stream = s;
  struct Guard {
    diaf_factors*& f;
    bool keep = false;
    ~Guard() { if (!keep) diaf_free(f); }
  } guard{F};
  cudaGetDevice(&F->device);
  for (cudaEvent_t& e : F->ev) DIAF_CU(event_get(&e, F->device));
  DIAF_CU(cudaEventRecord(F->ev[0], s));
  Pool pool(s);
  NumericPlan np;
  st = symbolic_pass(A, PW, V, alg, prec, tuning, s, F, pool, np);
  if (st != DIAF_OK) return st;
  // a triangular V by rule: its structure goes to the host column by column
  // during the numeric pass (the columns of an upper V in descending order,
  // the order in which the level schedule visits them)
  if ((V->rule == DIAF_RULE_UPPER || V->rule == DIAF_RULE_LOWER) && F->n > 0 && mirror_acquire(F)) {
    DIAF_CU(cudaMemcpyAsync(F->mir_cp, F->Vcp, sizeof(int32_t) * (F->n + 1), cudaMemcpyDeviceToHost, s));
    np.ca.Hri = F->mir_ri_dev;
    np.ca.Hgen = F->mir_word_dev;
    np.ca.gen = F->mir_gen;
    np.ca.list_desc = V->rule == DIAF_RULE_UPPER;
  }
  DIAF_CU(cudaEventRecord(F->ev[1], s));  // after the copy of V's column pointers
  st = enqueue_numeric(F, np, s, true);
  if (st != DIAF_OK) return st;
  DIAF_CU(cudaEventRecord(F->ev[2], s));
  pool.release();
  guard.keep = true;
  *out = F;
  return DIAF_OK;
}

diaf_status diaf_factor(const diaf_csc* A, const diaf_pattern* PW, const diaf_vspec* V, int32_t alg, int32_t prec,
                        void* stream, diaf_factors** out) {
  return diaf_factor_tuned(A, PW, V, alg, prec, nullptr, stream, out);
}

diaf_status diaf_plan_create(const diaf_csc* A, const diaf_pattern* PW, const diaf_vspec* V, int32_t alg,
                             int32_t prec, const diaf_tuning* tuning, void* stream, diaf_plan** out) {
  g_last_error.clear();
  if (!out) return fail(DIAF_EINVAL, "out is NULL");
  *out = nullptr;
  diaf_status st = check_args(A, PW, V, alg, prec, tuning);
  if (st != DIAF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto P = new diaf_plan();
  P->F = new diaf_factors();
  P->F->stream = s;
  P->scratch = new Pool(s);
  struct Guard {
    diaf_plan*& p;
    bool keep = false;
    ~Guard() { if (!keep) diaf_plan_free(p); }
  } guard{P};
  st = symbolic_pass(A, PW, V, alg, prec, tuning, s, P->F, *P->scratch, P->np);
  if (st != DIAF_OK) return st;
  DIAF_CU(cudaStreamSynchronize(s));
  // capture the numeric pass on a private stream (the caller's may be the legacy default stream)
  cudaStream_t cs;
  DIAF_CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  st = enqueue_numeric(P->F, P->np, cs, false);
  e = cudaStreamEndCapture(cs, &P->graph);
  cudaStreamDestroy(cs);
  if (st != DIAF_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  DIAF_CU(cudaGraphInstantiate(&P->exec, P->graph, 0));
  guard.keep = true;
  *out = P;
  return DIAF_OK;
}

diaf_status diaf_plan_execute(diaf_plan* P, void* stream) {
  if (!P || !P->exec) return fail(DIAF_EINVAL, "NULL plan");
  DIAF_CU(cudaGraphLaunch(P->exec, static_cast<cudaStream_t>(stream)));
  DIAF_COUNT_LAUNCH();
  return DIAF_OK;
}

diaf_factors* diaf_plan_factors(diaf_plan* P) { return P ? P->F : nullptr; }

diaf_status diaf_autotune(const diaf_csc* A, const diaf_pattern* PW, const diaf_vspec* V, int32_t alg, int32_t prec,
                          void* stream, diaf_tuning* best, float* best_ms) {
  if (!best) return fail(DIAF_EINVAL, "best is NULL");
  diaf_tuning cur{};
  auto time_of = [&](const diaf_tuning& t, float* ms_out) -> diaf_status {
    float ms[2] = {0, 0};
    for (int rep = 0; rep < 2; ++rep) {
      diaf_factors* F = nullptr;
      diaf_status st = diaf_factor_tuned(A, PW, V, alg, prec, &t, stream, &F);
      if (st != DIAF_OK) return st;
      float tm[2 + kNumBuckets];
      st = diaf_factor_timings(F, tm, 2 + kNumBuckets);
      diaf_free(F);
      if (st != DIAF_OK) return st;
      ms[rep] = tm[1];  // the numeric pass
    }
    *ms_out = ms[0] < ms[1] ? ms[0] : ms[1];
    return DIAF_OK;
  };
  float cur_ms = 0;
  diaf_status st = time_of(cur, &cur_ms);
  if (st != DIAF_OK) return st;
  // coordinate descent over the bucket edges, the CTA sizes of the warp
  // kernels and the small-tile kernel (thread or warp per column)
  const int edge0[] = {32, 24, 16}, edge1[] = {64, 48, 32}, wpbs[] = {0, 2, 4, 8}, kernels[] = {1, 2};
  for (int knob = 0; knob < 6; ++knob) {
    const int* vals = knob == 0 ? edge0 : (knob == 1 ? edge1 : (knob >= 4 ? kernels : wpbs));
    const int nv = knob < 2 ? 3 : (knob >= 4 ? 2 : 4);
    for (int i = 0; i < nv; ++i) {
      diaf_tuning t = cur;
      int* field = knob == 0   ? &t.m_edge0
                   : knob == 1 ? &t.m_edge1
                   : knob == 4 ? &t.small_tiles
                   : knob == 5 ? &t.large_tiles
                               : &t.warps_per_block[knob - 2];
      const int* curf = knob == 0   ? &cur.m_edge0
                        : knob == 1 ? &cur.m_edge1
                        : knob == 4 ? &cur.small_tiles
                        : knob == 5 ? &cur.large_tiles
                                    : &cur.warps_per_block[knob - 2];
      const int eff = (*curf == 0 && (knob < 2 || knob >= 4)) ? vals[0] : *curf;
      if (vals[i] == eff) continue;
      *field = vals[i];
      float ms = 0;
      st = time_of(t, &ms);
      if (st != DIAF_OK) return st;
      if (ms < cur_ms * 0.98f) { cur = t; cur_ms = ms; }
    }
  }
  *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return DIAF_OK;
}

void diaf_plan_free(diaf_plan* P) {
  if (!P) return;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  delete P->scratch;  // stream-ordered frees on the creation stream
  diaf_free(P->F);
  delete P;
}

diaf_status diaf_factor_info_get(const diaf_factors* F, diaf_factor_info* info) {
  if (!F || !info) return fail(DIAF_EINVAL, "NULL argument");
  *info = F->info;
  return DIAF_OK;
}

diaf_status diaf_get_factors(const diaf_factors* F, diaf_csc* W, diaf_csc* V, const double** col_res,
                             const uint32_t** col_flags) {
  if (!F) return fail(DIAF_EINVAL, "NULL handle");
  if (W) *W = diaf_csc{F->n, F->nnz_w, F->Wcp, F->Wri, F->Wv, F->dtype};
  if (V) *V = diaf_csc{F->n, F->nnz_v, F->Vcp, F->Vri, F->Vv, F->dtype};
  if (col_res) *col_res = F->res;
  if (col_flags) *col_flags = F->flags;
  return DIAF_OK;
}

diaf_status diaf_sync(diaf_factors* F, void* stream) {
  if (!F) return fail(DIAF_EINVAL, "NULL handle");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t h = 0;
  DIAF_CU(cudaMemcpyAsync(&h, F->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  DIAF_CU(cudaStreamSynchronize(s));
  if (h & DEV_ST_CAPACITY) return fail(DIAF_EUNSUPPORTED, "capacity exceeded on the device");
  return DIAF_OK;
}

// Block-diagonal V: W in CSR for the SpMV, the blocks of V factored by LU.
static diaf_status prepare_apply_blocks(diaf_factors* F, cudaStream_t s) {
  const int n = F->n;
  const bool cplx = F->dtype == DIAF_C128;
  const size_t esz = cplx ? 16 : 8;
  int32_t* work;
  DIAF_CU(F->alloc(&work, 2 * n + scan_blocksums_size(n)));
  F->Wr.n = n; F->Wr.nnz = F->nnz_w;
  DIAF_CU(F->alloc(&F->Wr.rowptr, n + 1));
  DIAF_CU(F->alloc(&F->Wr.colidx, F->nnz_w));
  DIAF_CU(F->alloc((char**)&F->Wr.vals, esz * F->nnz_w));
  DIAF_CU(csc_to_csr(n, F->nnz_w, F->Wcp, F->Wri, F->Wv, cplx, F->Wr.rowptr, F->Wr.colidx, F->Wr.vals, work, s));
  DIAF_CU(F->alloc(&F->Vb.bstart, n + 1));
  DIAF_CU(F->alloc((char**)&F->Vb.lu, esz * block_lu_elems(n)));
  DIAF_CU(F->alloc(&F->Vb.piv, n));
  uint32_t* st;
  DIAF_CU(F->alloc(&st, 1));
  DIAF_CU(cudaMemsetAsync(st, 0, sizeof(uint32_t), s));
  DIAF_CU(block_prepare(n, cplx, F->blk, F->Vcp, F->Vri, F->Vv, F->Vb, work, st, s));
  uint32_t h = 0;
  DIAF_CU(cudaMemcpyAsync(&h, st, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  DIAF_CU(cudaStreamSynchronize(s));
  if (h & DEV_ST_BAD_INPUT) return fail(DIAF_EINVAL, "block ids decrease, or V has an entry outside its block");
  if (h & DEV_ST_CAPACITY) return fail(DIAF_EUNSUPPORTED, "a block of V has more than 64 rows");
  if (h & DEV_ST_SINGULAR) return fail(DIAF_EINVAL, "V has a singular diagonal block");
  DIAF_CU(F->alloc((char**)&F->tbuf, esz * n));
  F->v_block = true;
  F->apply_ready = true;
  return DIAF_OK;
}

// Pinned host staging for prepare_apply's copies of V's structure (to the
// host) and of the level order (back): pageable copies go through the
// driver's bounce buffer at a fraction of the bandwidth and block the host.
// One buffer per process, grown as needed and reused; `done` (one event per
// device) marks the end of the last copy out of it.
namespace {
constexpr int kStageDevices = 64;
struct PinnedStage {
  std::mutex mu;
  unsigned char* buf = nullptr;
  size_t cap = 0;
  cudaEvent_t done[kStageDevices] = {};
};
PinnedStage g_stage;

// Waits for the previous user's copies and returns at least `bytes` of
// pinned memory (nullptr on failure).  Call with g_stage.mu held.
unsigned char* stage_get(size_t bytes) {
  for (int d = 0; d < kStageDevices; ++d)
    if (g_stage.done[d]) cudaEventSynchronize(g_stage.done[d]);
  if (bytes > g_stage.cap) {
    if (g_stage.buf) cudaFreeHost(g_stage.buf);
    g_stage.buf = nullptr;
    g_stage.cap = 0;
    const size_t want = bytes + bytes / 4;
    if (cudaHostAlloc((void**)&g_stage.buf, want, cudaHostAllocPortable) != cudaSuccess) {
      (void)cudaGetLastError();
      g_stage.buf = nullptr;
      return nullptr;
    }
    g_stage.cap = want;
  }
  return g_stage.buf;
}


// True once event e has completed (or failed: a waiter then stops waiting).
bool event_passed(cudaEvent_t e) {
  if (cudaEventQuery(e) != cudaErrorNotReady) return true;
  if (cudaPeekAtLastError() == cudaErrorNotReady) (void)cudaGetLastError();  // not an error
  return false;
}

// The level schedule of a triangular V from its columns (host arrays cp,
// ri), visited in the solve's order: descending for an upper V, ascending for
// a lower one.  With `word` (the mirror), column j is visited once its word
// holds the owner's generation `gen` (acquire load, after which its rows are
// visible); without, every column is there.  lev[j] is final when the walk
// reaches column j, so the walk also gives row j its place among the rows of
// its level (rank[j]; cnt[0..nlev) counts the rows per level), numbers the
// off-diagonal entries of every row in the order it meets them (slot[p] for
// entry p of the columns, rcnt[i] entries in row i) and notes where each
// column's diagonal entry is (dpos[j]): all the device needs to lay V's rows
// out level by level.  Returns 0, 1 (an entry on the wrong side of the
// diagonal), 2 (a diagonal entry missing), 3 (a row index out of range) or 4
// (`done`, the end of the numeric pass, passed while a column had not
// arrived).  After 1, 3 or 4 the kernels may still write into the mirror.
struct LevelWalk {
  int32_t *lev, *rank, *rcnt, *dpos, *slot, *cnt;
  int nlev;
};

int level_walk(int n, const int32_t* cp, const int32_t* ri, const uint32_t* word, uint32_t gen, bool up,
               cudaEvent_t done, LevelWalk& w) {
  auto arrived = [&](int j) { return !word || __atomic_load_n(word + j, __ATOMIC_ACQUIRE) == gen; };
  for (int i = 0; i < n; ++i) {
    w.lev[i] = 0;
    w.rcnt[i] = 0;
  }
  int nl = 0;
  bool nodiag = false;
  for (int step = 0; step < n; ++step) {
    const int j = up ? n - 1 - step : step;
    if (!arrived(j)) {
      for (unsigned spin = 1; !arrived(j); ++spin) {
        if ((spin & 1023u) == 0 && event_passed(done)) {
          if (arrived(j)) break;  // the pass's writes are all visible once it has ended
          return 4;
        }
      }
    }
    const int lj = w.lev[j];
    while (nl <= lj) w.cnt[nl++] = 0;
    w.rank[j] = w.cnt[lj]++;
    bool d = false;
    for (int p = cp[j]; p < cp[j + 1]; ++p) {
      const int i = ri[p];
      if (i < 0 || i >= n) return 3;
      if (i == j) {
        d = true;
        w.dpos[j] = p;
        w.slot[p] = -1;
        continue;
      }
      if (up ? i > j : i < j) return 1;
      w.slot[p] = w.rcnt[i]++;
      if (w.lev[i] <= lj) w.lev[i] = lj + 1;
    }
    if (!d) w.dpos[j] = -1;
    nodiag |= !d;
  }
  w.nlev = nl;
  return nodiag ? 2 : 0;
}

// Marks the end of the copies out of the staging buffer on stream s.
cudaError_t stage_release(cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kStageDevices) return cudaStreamSynchronize(s);
  if (!g_stage.done[dev]) {
    e = cudaEventCreateWithFlags(&g_stage.done[dev], cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  return cudaEventRecord(g_stage.done[dev], s);
}
}  // namespace


// y = W V^-1 x on the level-ordered V: the level solve, then (after W's
// row-oriented copy, when that is still being built on the side stream) the
// W SpMV.  Stream work only.
static diaf_status enqueue_level_apply(diaf_factors* F, const void* x, void* y, cudaStream_t s) {
  const bool cplx = F->dtype == DIAF_C128;
#ifdef DIAF_PREP_TIMING
  PrepTimer pt("apply");
#endif
  PT_DEV(s);
  DIAF_CU(trsv_levels_perm(F->Vl, cplx, x, F->tbuf, s, F->solve_cold));
  F->solve_cold = false;
  PT_DEV(s);
  if (F->w_pending) {  // W's row-oriented copy, built on the side stream during the solve
    DIAF_CU(cudaStreamWaitEvent(s, F->wev[1], 0));
    F->w_pending = false;
  }
  DIAF_CU(csr_spmv(F->Wl, cplx, F->tbuf, y, s));
  PT_DEV(s);
  return DIAF_OK;
}

// Prepares the apply on F (row-oriented W, V level by level) and, for a
// triangular V with n > 0, enqueues the first y = W V^-1 x right behind the
// preparation's kernels, before it waits for the zero-diagonal check (which
// precedes the solve on the stream; *applied = true then); on that check's
// failure y is not valid and the call fails.
static diaf_status prepare_apply(diaf_factors* F, cudaStream_t s, const void* x, void* y, bool* applied) {
  *applied = false;
  if (F->rule == DIAF_RULE_BLOCK) return prepare_apply_blocks(F, s);
#ifdef DIAF_PREP_TIMING
  PrepTimer pt("prep");
#endif
  PT_DEV(s);
  const int n = F->n;
  const bool cplx = F->dtype == DIAF_C128;
  const size_t esz = cplx ? 16 : 8;
  const size_t nnzv = (size_t)F->nnz_v;
  int32_t* work;
  DIAF_CU(F->alloc(&work, n + scan_blocksums_size(n)));
  // V's structure is walked on the host (level of every row, its place in
  // its level, the numbering of every row's entries, the diagonals) -- when F
  // holds the mirror, while the numeric pass still writes V's columns there;
  // otherwise from a copy taken after the pass (pinned staging: cp, ri).
  // Meanwhile the device converts W to rows.  The walk's arrays go to the
  // device in one copy, and the device lays V's rows out level by level.
  const bool mir = F->mirror;
  std::lock_guard<std::mutex> stage_lock(g_stage.mu);
  const size_t n1 = (size_t)n + 1;
  const size_t nri = mir ? 0 : nnzv;
  const size_t blk = 4 * (size_t)n + nnzv;  // lev, rank, rcnt, dpos, slot
  unsigned char* stage = stage_get(sizeof(int32_t) * (n1 + nri + n1 + blk) + sizeof(uint32_t));
  if (!stage) {
    if (mir) {
      (void)cudaStreamSynchronize(s);
      mirror_release(F);
    }
    return fail(DIAF_ENOMEM, "pinned host staging for the level schedule");
  }
  int32_t* const st32 = reinterpret_cast<int32_t*>(stage);
  int32_t* cp = mir ? F->mir_cp : st32;
  int32_t* ri = mir ? F->mir_ri : st32 + n1;
  int32_t* ptr = st32 + (mir ? 0 : n1 + nri);  // level pointers (at most n + 1)
  int32_t* hblk = ptr + n1;
  LevelWalk lw{hblk, hblk + n, hblk + 2 * (size_t)n, hblk + 3 * (size_t)n, hblk + 4 * (size_t)n, nullptr, 0};
  uint32_t* hp = reinterpret_cast<uint32_t*>(hblk + blk);
  if (!mir) {
    DIAF_CU(cudaMemcpyAsync(cp, F->Vcp, sizeof(int32_t) * n1, cudaMemcpyDeviceToHost, s));
    if (nnzv > 0) DIAF_CU(cudaMemcpyAsync(ri, F->Vri, sizeof(int32_t) * nnzv, cudaMemcpyDeviceToHost, s));
  }
  PT_DEV(s);
  cudaEvent_t ev[2];
  DIAF_CU(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
  cudaError_t ce = cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
  if (ce != cudaSuccess) {
    cudaEventDestroy(ev[0]);
    DIAF_CU(cudaStreamSynchronize(s));  // the copies write into the staging buffer
    DIAF_CU(ce);
  }
  ce = cudaEventRecord(ev[0], s);
  // W to rows, on the side stream when there is one (its own scratch)
  F->Wr.n = n;
  F->Wr.nnz = F->nnz_w;
  if (ce == cudaSuccess) ce = F->alloc(&F->Wr.rowptr, n + 1);
  if (ce == cudaSuccess) ce = F->alloc(&F->Wr.colidx, F->nnz_w);
  if (ce == cudaSuccess) ce = F->alloc((char**)&F->Wr.vals, esz * F->nnz_w);
  cudaStream_t ws = side_stream();
  int32_t* wwork = work;
  if (ws && ce == cudaSuccess) {
    ce = F->alloc(&wwork, n + scan_blocksums_size(n));
    for (int i = 0; i < 2 && ce == cudaSuccess; ++i)
      if (!F->wev[i]) ce = cudaEventCreateWithFlags(&F->wev[i], cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventRecord(F->wev[0], s);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(ws, F->wev[0], 0);
  }
  cudaStream_t wsx = ws ? ws : s;
  if (ce == cudaSuccess)
    ce = csc_to_csr(n, F->nnz_w, F->Wcp, F->Wri, F->Wv, cplx, F->Wr.rowptr, F->Wr.colidx, F->Wr.vals, wwork, wsx);
  if (ws && ce == cudaSuccess) ce = cudaEventRecord(F->wev[1], ws);  // diaf_free waits for it
  // the level-ordered copy of V and its inputs (sizes known now; the level
  // count is at most n), so that only copies and kernels follow the walk
  LevelCsr& Vl = F->Vl;
  int32_t *pos = nullptr, *dblk = nullptr;
  uint32_t* zflag = nullptr;
  Vl.n = n;
  Vl.nnz = F->nnz_v - n;
  {
    Carve c;
    c.add(&Vl.lvlptr, n + 1);
    c.add(&Vl.rowptr, n + 1);
    c.add(&Vl.colidx, Vl.nnz > 0 ? Vl.nnz : 0);
    c.add((char**)&Vl.vals, esz * (Vl.nnz > 0 ? Vl.nnz : 0));
    c.add((char**)&Vl.dinv, esz * n);
    c.add(&Vl.xrow, n);
    c.add(&pos, n);
    c.add(&dblk, blk);
    c.add(&zflag, 1);
    c.add(&F->Wl.colidx, F->nnz_w);
    c.add((char**)&F->tbuf, esz * n);
    if (ce == cudaSuccess) ce = F->carve(c);
  }
  if (ce == cudaSuccess) ce = cudaMemsetAsync(zflag, 0, sizeof(uint32_t), s);
  int32_t* const wl_colidx = F->Wl.colidx;
  PT_DEV(s);
  PT_HOST();
  // wait for the copies even after an error: they write into the staging
  // buffer (the mirror's columns are read as they arrive instead)
  cudaError_t se = mir ? cudaSuccess : cudaEventSynchronize(ev[0]);
  PT_HOST();
  if (ce != cudaSuccess || se != cudaSuccess) {
    (void)cudaStreamSynchronize(s);
    mirror_release(F);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    DIAF_CU(ce);
    DIAF_CU(se);
  }
  // the walk (host, O(nnz)); rows per level in host scratch reused across
  // calls of this thread (the walk sets what it uses)
  static thread_local std::vector<int32_t> cnt;
  if (cnt.size() < n1) cnt.resize(n1);
  lw.cnt = cnt.data();
  bool vup = true;
  int ls = -1;
  if (mir) {
    // V's column pointers reached the host before the numeric pass began
    se = cudaEventSynchronize(F->ev[1]);
    if (se == cudaSuccess) {
      vup = F->rule == DIAF_RULE_UPPER;
      ls = level_walk(n, cp, ri, F->mir_word, F->mir_gen, vup, F->ev[2], lw);
    }
    if (ls == 0 || ls == 2) {
      g_prep_streamed.fetch_add(1, std::memory_order_relaxed);
    } else {
      // not every column arrived, or an entry is out of place: V's whole
      // structure once the numeric pass has ended
      se = cudaStreamSynchronize(s);
      if (se == cudaSuccess && nnzv > 0) se = cudaMemcpy(ri, F->Vri, sizeof(int32_t) * nnzv, cudaMemcpyDeviceToHost);
      if (se != cudaSuccess) {
        mirror_release(F);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        DIAF_CU(se);
      }
      ls = -1;
    }
  }
  if (ls < 0) {  // the whole structure at hand: an upper V, else a lower one
    vup = true;
    ls = level_walk(n, cp, ri, nullptr, 0, true, nullptr, lw);
    if (ls == 1) {
      vup = false;
      ls = level_walk(n, cp, ri, nullptr, 0, false, nullptr, lw);
    }
    g_prep_copied.fetch_add(1, std::memory_order_relaxed);
  }
  // every column of the mirror has been read (or the stream synchronised)
  mirror_release(F);
  F->v_upper = vup;
  if (ls != 0) {
    (void)cudaStreamSynchronize(s);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    return fail(DIAF_EINVAL, ls == 1   ? "V is not triangular"
                             : ls == 3 ? "V has a row index out of range"
                                       : "V has a zero or missing diagonal entry");
  }
  PT_HOST();
  const int nlev = lw.nlev;
  ptr[0] = 0;
  Vl.maxw = 0;
  for (int l = 0; l < nlev; ++l) {
    ptr[l + 1] = ptr[l] + cnt[l];
    Vl.maxw = std::max(Vl.maxw, cnt[l]);
  }
  Vl.nlev = nlev;
  // the device places the rows (position of row i: ptr[lev i] + rank i),
  // lays V's rows out level by level from its columns, and checks the
  // diagonal's values; the zero-diagonal flag is read after all of that is
  // enqueued
  ce = cudaMemcpyAsync(Vl.lvlptr, ptr, sizeof(int32_t) * (nlev + 1), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(dblk, hblk, sizeof(int32_t) * blk, cudaMemcpyHostToDevice, s);
  PT_DEV(s);
  if (ce == cudaSuccess) ce = stage_release(s);  // the next user of the staging buffer waits for these copies
  if (ce != cudaSuccess) {
    (void)cudaStreamSynchronize(s);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    DIAF_CU(ce);
  }
  const int32_t* dlev = dblk;
  const int32_t* drank = dblk + n;
  const int32_t* drcnt = dblk + 2 * (size_t)n;
  const int32_t* ddpos = dblk + 3 * (size_t)n;
  const int32_t* dslot = dblk + 4 * (size_t)n;
  ce = level_place(n, dlev, drank, drcnt, Vl.lvlptr, pos, Vl.xrow, work, Vl.rowptr, s);
  F->Wl = F->Wr;
  F->Wl.colidx = wl_colidx;
  if (ws) {  // W's columns renumbered to V's level order on the side stream, once the positions are known
    if (ce == cudaSuccess) ce = cudaEventRecord(F->wev[0], s);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(ws, F->wev[0], 0);
  }
  if (ce == cudaSuccess) ce = remap_columns(F->nnz_w, pos, F->Wr.colidx, F->Wl.colidx, wsx);
  if (ws && ce == cudaSuccess) {
    ce = cudaEventRecord(F->wev[1], ws);
    F->w_pending = ce == cudaSuccess;
  }
  if (ce == cudaSuccess)
    ce = level_fill(n, cplx, F->Vcp, F->Vri, F->Vv, ddpos, dslot, pos, Vl, zflag, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(hp, zflag, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaEventRecord(ev[1], s);
  PT_DEV(s);
  // the first apply goes right behind, before the host waits for the
  // zero-diagonal flag (which reaches it while the solve runs): no host round
  // trip between the preparation and the solve, and the call returns while
  // the solve is still running
  F->solve_cold = true;
  diaf_status ast = DIAF_OK;
  if (ce == cudaSuccess && n > 0) {
    ast = enqueue_level_apply(F, x, y, s);
    *applied = ast == DIAF_OK;
  }
  PT_HOST();
  se = ce == cudaSuccess ? cudaEventSynchronize(ev[1]) : cudaStreamSynchronize(s);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  DIAF_CU(ce);
  DIAF_CU(se);
  if (*hp) {
    *applied = false;
    return fail(DIAF_EINVAL, "V has a zero or missing diagonal entry");
  }
  if (ast != DIAF_OK) return ast;
  PT_HOST();
  F->apply_ready = true;
  return DIAF_OK;
}

diaf_status diaf_level_schedule(int32_t n, const int32_t* colptr, const int32_t* rowidx, int32_t* level,
                                int32_t* nlev, int32_t* upper) {
  g_last_error.clear();
  if (n < 0) return fail(DIAF_EINVAL, "n must be >= 0");
  if (!colptr || !level || !nlev || !upper || (n > 0 && colptr[n] > 0 && !rowidx))
    return fail(DIAF_EINVAL, "NULL argument");
  if (colptr[0] != 0) return fail(DIAF_EINVAL, "colptr[0] must be 0");
  for (int32_t j = 0; j < n; ++j)
    if (colptr[j + 1] < colptr[j]) return fail(DIAF_EINVAL, "colptr must be non-decreasing");
  // the walk of the apply's preparation, on the whole structure: an upper V,
  // else a lower one
  const size_t nn = (size_t)n, nnz = (size_t)colptr[n];
  std::vector<int32_t> scratch(4 * nn + 1 + nnz);
  LevelWalk w{level, scratch.data(), scratch.data() + nn, scratch.data() + 2 * nn, scratch.data() + 4 * nn + 1,
              scratch.data() + 3 * nn, 0};
  bool up = true;
  int r = level_walk(n, colptr, rowidx, nullptr, 0, true, nullptr, w);
  if (r == 1) {
    up = false;
    r = level_walk(n, colptr, rowidx, nullptr, 0, false, nullptr, w);
  }
  const int nl = w.nlev;
  if (r == 1) return fail(DIAF_EINVAL, "V is not triangular");
  if (r == 2) return fail(DIAF_EINVAL, "V has a missing diagonal entry");
  if (r == 3) return fail(DIAF_EINVAL, "V has a row index out of range");
  *nlev = nl;
  *upper = up ? 1 : 0;
  return DIAF_OK;
}

diaf_status diaf_apply(diaf_factors* F, const void* x, void* y, void* stream) {
  if (!F || (F->n > 0 && (!x || !y))) return fail(DIAF_EINVAL, "NULL argument");
  if (x == y) return fail(DIAF_EINVAL, "x and y must not overlap");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!F->apply_ready) {
    bool applied = false;
    diaf_status st = prepare_apply(F, s, x, y, &applied);
    if (st != DIAF_OK || applied) return st;
  }
  if (F->n == 0) return DIAF_OK;
  const bool cplx = F->dtype == DIAF_C128;
  if (F->v_block) {
    DIAF_CU(block_solve(F->Vb, cplx, x, F->tbuf, s));
    DIAF_CU(csr_spmv(F->Wr, cplx, F->tbuf, y, s));
    return DIAF_OK;
  }
  return enqueue_level_apply(F, x, y, s);
}

}  // extern "C"
