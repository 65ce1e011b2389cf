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
// The one piece of scratch the apply needs -- the intermediate vector
// t = V^-1 x, in the level order of the solve -- lives in a file-scope
// __device__ array of fixed size, which every GPU that loads the library
// keeps until the process exits.  The solve is the level-scheduled one of
// diaf_apply (one block, a barrier between levels, no waits on flags), and
// it writes every entry of t before the SpMV reads it, so nothing in the
// array has to start at zero and nothing an earlier call left there is read.
#include <mutex>
#include <string>

#include "factors.cuh"

namespace {

constexpr int kStaticMaxN = 1 << 18;             // rows
constexpr size_t kScratchBytes = 16 * (size_t)kStaticMaxN;  // t, complex128 worst case: 4 MB

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
  void* t = base;
  const bool cplx = F->dtype == DIAF_C128;
  if (F->w_pending) {  // the first diaf_apply stopped before its SpMV: W's copy may still be in the making
    e = cudaStreamWaitEvent(s, F->wev[1], 0);
    if (e != cudaSuccess) return fail(DIAF_ECUDA, cudaGetErrorString(e));
    F->w_pending = false;
  }
  e = trsv_levels_perm(F->Vl, cplx, x, t, s);
  if (e != cudaSuccess) return fail(DIAF_ECUDA, cudaGetErrorString(e));
  e = csr_spmv(F->Wl, cplx, t, y, s);
  if (e != cudaSuccess) return fail(DIAF_ECUDA, cudaGetErrorString(e));
  return DIAF_OK;
}
