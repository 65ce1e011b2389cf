// Shared device helpers of the DIAF CUDA library: scalar types (real and
// complex, FP64 and FP32), warp reductions, and the status / flag words.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/diaf.h"

#define DIAF_WARP 32
#define DIAF_FULL 0xffffffffu

// Device status bits (a uint32 in device memory, OR-ed by kernels).
enum : uint32_t {
  DEV_ST_CAPACITY = 1u,     // a column exceeded the capacity of the kernel that got it
  DEV_ST_BAD_INPUT = 4u,    // index out of range / unsorted column found on the device
  DEV_ST_SINGULAR = 8u,     // a zero pivot (block LU of V)
};

// System-scope release store: a host thread that reads *p == v with acquire
// semantics also sees every write the storing thread (and any thread ordered
// before it by a barrier and a system fence) made before it, host memory
// included.
__device__ __forceinline__ void store_release_sys(uint32_t* p, uint32_t v) {
  asm volatile("st.release.sys.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ----------------------------------------------------------------- scalars
template <class R>
struct Cx {
  R re, im;
};

template <class S> struct ScalarInfo;
template <> struct ScalarInfo<double> { using R = double; static constexpr bool cplx = false; };
template <> struct ScalarInfo<float> { using R = float; static constexpr bool cplx = false; };
template <> struct ScalarInfo<Cx<double>> { using R = double; static constexpr bool cplx = true; };
template <> struct ScalarInfo<Cx<float>> { using R = float; static constexpr bool cplx = true; };

template <class S> using RealOf = typename ScalarInfo<S>::R;

__device__ __forceinline__ double sc_conj(double a) { return a; }
__device__ __forceinline__ float sc_conj(float a) { return a; }
template <class R> __device__ __forceinline__ Cx<R> sc_conj(Cx<R> a) { return {a.re, -a.im}; }

__device__ __forceinline__ double sc_abs2(double a) { return a * a; }
__device__ __forceinline__ float sc_abs2(float a) { return a * a; }
template <class R> __device__ __forceinline__ R sc_abs2(Cx<R> a) { return a.re * a.re + a.im * a.im; }

__device__ __forceinline__ double sc_real(double a) { return a; }
__device__ __forceinline__ float sc_real(float a) { return a; }
template <class R> __device__ __forceinline__ R sc_real(Cx<R> a) { return a.re; }
__device__ __forceinline__ double sc_imag(double) { return 0.0; }
__device__ __forceinline__ float sc_imag(float) { return 0.0f; }
template <class R> __device__ __forceinline__ R sc_imag(Cx<R> a) { return a.im; }

template <class S> __device__ __forceinline__ S sc_make(RealOf<S> re, RealOf<S> im);
template <> __device__ __forceinline__ double sc_make<double>(double re, double) { return re; }
template <> __device__ __forceinline__ float sc_make<float>(float re, float) { return re; }
template <> __device__ __forceinline__ Cx<double> sc_make<Cx<double>>(double re, double im) { return {re, im}; }
template <> __device__ __forceinline__ Cx<float> sc_make<Cx<float>>(float re, float im) { return {re, im}; }

template <class S> __device__ __forceinline__ S sc_zero() { return sc_make<S>(RealOf<S>(0), RealOf<S>(0)); }
template <class S> __device__ __forceinline__ S sc_real_s(RealOf<S> r) { return sc_make<S>(r, RealOf<S>(0)); }

template <class R> __device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> __device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> __device__ __forceinline__ Cx<R> operator-(Cx<R> a) { return {-a.re, -a.im}; }
template <class R> __device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R> __device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) { return {s * a.re, s * a.im}; }
// acc - a b as fused multiply-adds: one for real scalars, four for complex
// ones (two independent chains of two, against two products and two
// subtractions of the plain form).
__device__ __forceinline__ double sc_msub(double acc, double a, double b) { return fma(-a, b, acc); }
template <class R> __device__ __forceinline__ Cx<R> sc_msub(Cx<R> acc, Cx<R> a, Cx<R> b) {
  const R re = fma(a.im, b.im, fma(-a.re, b.re, acc.re));
  const R im = fma(-a.im, b.re, fma(-a.re, b.im, acc.im));
  return {re, im};
}
template <class R> __device__ __forceinline__ Cx<R> operator*(Cx<R> a, R s) { return {s * a.re, s * a.im}; }
template <class R> __device__ __forceinline__ Cx<R>& operator+=(Cx<R>& a, Cx<R> b) { a.re += b.re; a.im += b.im; return a; }
template <class R> __device__ __forceinline__ Cx<R>& operator-=(Cx<R>& a, Cx<R> b) { a.re -= b.re; a.im -= b.im; return a; }

// conj(a) * b, the inner-product term
__device__ __forceinline__ double sc_cmul(double a, double b) { return a * b; }
__device__ __forceinline__ float sc_cmul(float a, float b) { return a * b; }
template <class R> __device__ __forceinline__ Cx<R> sc_cmul(Cx<R> a, Cx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}

// conversions between precisions
template <class D, class S> __device__ __forceinline__ D sc_cast(S a);
template <> __device__ __forceinline__ double sc_cast<double, double>(double a) { return a; }
template <> __device__ __forceinline__ float sc_cast<float, double>(double a) { return (float)a; }
template <> __device__ __forceinline__ double sc_cast<double, float>(float a) { return (double)a; }
template <> __device__ __forceinline__ float sc_cast<float, float>(float a) { return a; }
template <> __device__ __forceinline__ Cx<double> sc_cast<Cx<double>, Cx<double>>(Cx<double> a) { return a; }
template <> __device__ __forceinline__ Cx<float> sc_cast<Cx<float>, Cx<double>>(Cx<double> a) { return {(float)a.re, (float)a.im}; }
template <> __device__ __forceinline__ Cx<double> sc_cast<Cx<double>, Cx<float>>(Cx<float> a) { return {(double)a.re, (double)a.im}; }
template <> __device__ __forceinline__ Cx<float> sc_cast<Cx<float>, Cx<float>>(Cx<float> a) { return a; }

// ----------------------------------------------------------------- shuffles
__device__ __forceinline__ double shfl_xor(double v, int m) { return __shfl_xor_sync(DIAF_FULL, v, m); }
__device__ __forceinline__ float shfl_xor(float v, int m) { return __shfl_xor_sync(DIAF_FULL, v, m); }
__device__ __forceinline__ int shfl_xor(int v, int m) { return __shfl_xor_sync(DIAF_FULL, v, m); }
template <class R> __device__ __forceinline__ Cx<R> shfl_xor(Cx<R> v, int m) {
  return {shfl_xor(v.re, m), shfl_xor(v.im, m)};
}
__device__ __forceinline__ double shfl_idx(double v, int l) { return __shfl_sync(DIAF_FULL, v, l); }
__device__ __forceinline__ float shfl_idx(float v, int l) { return __shfl_sync(DIAF_FULL, v, l); }
__device__ __forceinline__ int shfl_idx(int v, int l) { return __shfl_sync(DIAF_FULL, v, l); }
template <class R> __device__ __forceinline__ Cx<R> shfl_idx(Cx<R> v, int l) { return {shfl_idx(v.re, l), shfl_idx(v.im, l)}; }

template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
  return v;
}
template <class R> __device__ __forceinline__ Cx<R> warp_sum(Cx<R> v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) { v.re += shfl_xor(v.re, o); v.im += shfl_xor(v.im, o); }
  return v;
}
template <class T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) { T u = shfl_xor(v, o); v = u > v ? u : v; }
  return v;
}
template <class T> __device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) { T u = shfl_xor(v, o); v = u < v ? u : v; }
  return v;
}
// sum over aligned groups of G lanes (G a power of two <= 32)
template <int G, class T> __device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += shfl_xor(v, o);
  return v;
}
template <int G, class R> __device__ __forceinline__ Cx<R> group_sum(Cx<R> v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) { v.re += shfl_xor(v.re, o); v.im += shfl_xor(v.im, o); }
  return v;
}

// ----------------------------------------------------------------- phase timers
// Built only with -DDIAF_PHASE_TIMING (profiling builds): lane 0 of every warp
// adds the clock64 cycles spent between consecutive marks to phase[id], a
// device buffer handed to the kernel (ColArgs::phase); diaf_phase_cycles()
// (api.cu) reads it back.  No work is skipped.
#ifdef DIAF_PHASE_TIMING
#define DIAF_PHASE_START() long long diaf_t0_ = clock64()
#define DIAF_PHASE(id)                                                                               \
  do {                                                                                               \
    long long diaf_t1_ = clock64();                                                                  \
    if ((threadIdx.x & 31) == 0 && a.phase)                                                          \
      atomicAdd(&a.phase[id], (unsigned long long)(diaf_t1_ - diaf_t0_));                           \
    diaf_t0_ = diaf_t1_;                                                                             \
  } while (0)
#else
#define DIAF_PHASE_START() \
  do {                     \
  } while (0)
#define DIAF_PHASE(id) \
  do {                 \
  } while (0)
#endif

// ----------------------------------------------------------------- misc
// Process-wide count of kernels launched by this library (for the benchmark's
// launch accounting); defined in api.cu.
void diaf_note_launches(int k);
#define DIAF_COUNT_LAUNCH() diaf_note_launches(1)

__host__ __device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }

template <class T> __device__ __forceinline__ T dmin(T a, T b) { return a < b ? a : b; }
template <class T> __device__ __forceinline__ T dmax(T a, T b) { return a > b ? a : b; }

// first index with a[i] > key in a sorted int array
__device__ __forceinline__ int upper_bound_i32(const int32_t* a, int n, int key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] <= key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// lower_bound in a sorted int array
__device__ __forceinline__ int lower_bound_i32(const int32_t* a, int n, int key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}
