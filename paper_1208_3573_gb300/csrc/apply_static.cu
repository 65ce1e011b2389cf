// diaf_apply_static: y = W V^-1 x without any device allocation.
//
// For callers that may not allocate device memory at the point where they
// apply the preconditioner: code running under a fixed device-memory budget
// reserved at start-up, or a host framework whose own allocator owns all
// device memory and forbids allocations by the libraries it calls.  Such
// callers set the factors up beforehand (diaf_factor, and one diaf_apply,
// which builds the row-oriented copies of W and V), and from then on apply
// through this entry point.
//
// The scratch the triangular solve needs -- one ready flag per row, the
// ticket counter, and the intermediate vector t = V^-1 x -- lives in one
// file-scope __device__ array of fixed size, which every GPU that loads the
// library keeps until the process exits.  Every call clears the ready flags
// of its rows and the ticket counter on the stream before the solve, so what
// an earlier call left in the array never counts as ready.
#include <mutex>
#include <string>

#include "factors.cuh"

namespace {

constexpr int kStaticMaxN = 1 << 18;  // rows; the array below is about 5.3 MB
constexpr size_t kCounterBytes = 256;
constexpr size_t kFlagBytes = (sizeof(uint32_t) * kStaticMaxN + 255) / 256 * 256;
constexpr size_t kVecBytes = 16 * (size_t)kStaticMaxN;  // complex128 worst case
constexpr size_t kScratchBytes = kCounterBytes + kFlagBytes + kVecBytes;

// Device-side scratch shared by every call on a device.  In host code this
// name is only a stand-in for the symbol, not a device address: the address
// handed to the kernels comes from cudaGetSymbolAddress, looked up once per
// device in diaf_apply_static.
static __device__ __align__(256) unsigned char g_apply_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
// Device address of g_apply_scratch per device, looked up on the first call
// made with that device current.
unsigned char* g_base[kMaxDevices] = {};
std::mutex g_mu;

diaf_status fail(diaf_status st, const std::string& why) {
  diaf_set_last_error(why.c_str());
  return st;
}

}  // namespace

extern "C" diaf_status diaf_apply_static(diaf_factors* F, const void* x, void* y, void* stream) {
  diaf_set_last_error("");
  if (!F || (F->n > 0 && (!x || !y))) return fail(DIAF_EINVAL, "NULL argument");
  if (x == y) return fail(DIAF_EINVAL, "x and y must not overlap");
  if (F->rule == DIAF_RULE_BLOCK) return fail(DIAF_EUNSUPPORTED, "block-diagonal V: use diaf_apply");
  if (F->n > kStaticMaxN)
    return fail(DIAF_EINVAL, "n = " + std::to_string(F->n) + " exceeds the static scratch limit of " +
                                 std::to_string(kStaticMaxN) + " rows");
  if (!F->apply_ready)
    return fail(DIAF_EINVAL, "the factors have no row-oriented copies yet: call diaf_apply on them once first");
  if (F->n == 0) return DIAF_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(DIAF_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(DIAF_ECUDA, "device index beyond the static table");

  unsigned char* base;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
      // once per device, with that device current: the device address of the array
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_apply_scratch);
      if (e != cudaSuccess) return fail(DIAF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_base[dev] = static_cast<unsigned char*>(ptr);
    }
    base = g_base[dev];
  }
  int32_t* counter = reinterpret_cast<int32_t*>(base);
  uint32_t* ready = reinterpret_cast<uint32_t*>(base + kCounterBytes);
  void* t = base + kCounterBytes + kFlagBytes;
  const bool cplx = F->dtype == DIAF_C128;
  // the array keeps the previous call's flags: clear this call's rows (the
  // solve clears the ticket counter itself), then wait on flag value 1
  e = cudaMemsetAsync(ready, 0, sizeof(uint32_t) * (size_t)F->n, s);
  if (e != cudaSuccess) return fail(DIAF_ECUDA, cudaGetErrorString(e));
  e = csr_trsv_syncfree(F->Vr, cplx, F->v_upper, x, t, ready, counter, 1u, F->status, s);
  if (e != cudaSuccess) return fail(DIAF_ECUDA, cudaGetErrorString(e));
  e = csr_spmv(F->Wr, cplx, t, y, s);
  if (e != cudaSuccess) return fail(DIAF_ECUDA, cudaGetErrorString(e));
  return DIAF_OK;
}
