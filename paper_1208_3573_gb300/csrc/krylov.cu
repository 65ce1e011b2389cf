// Right-preconditioned BiCGSTAB (the evaluation solver of Sec. 5) with the
// scalars kept on the device: one device-to-host read per iteration.
#include <string>
#include <vector>

#include "plan.cuh"
#include "sparse.cuh"

extern "C" diaf_status diaf_apply(diaf_factors* F, const void* x, void* y, void* stream);

struct diaf_solver {
  cudaStream_t stream = nullptr;
  int n = 0;
  int dtype = DIAF_F64;
  Csr A;
  std::vector<void*> owned;
};

namespace {

thread_local std::string g_kry_err;

template <class T>
cudaError_t salloc(diaf_solver* S, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMallocAsync(&q, sizeof(T) * (count > 0 ? count : 1), S->stream);
  if (e != cudaSuccess) return e;
  S->owned.push_back(q);
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 304;  // 2 x 152 SMs

// Scalars of one BiCGSTAB run (device).
template <class S>
struct KState {
  S rho, rho_old, alpha, omega, beta;
  S dot[4];        // scratch results of the reductions
  double nrm[2];   // ||s||^2, ||r||^2
  int breakdown;   // 0, or 1 rho, 2 (rh, v), 3 (t, t), 4 omega
};

// partial sums of conj(a_i) b_i for up to two pairs at once
template <class S>
__global__ void dot2_partial(int n, const S* a0, const S* b0, const S* a1, const S* b1, S* part) {
  __shared__ S sh[2][kRedThreads / 32];
  S s0 = sc_zero<S>(), s1 = sc_zero<S>();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    s0 += sc_cmul(a0[i], b0[i]);
    if (a1) s1 += sc_cmul(a1[i], b1[i]);
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sh[0][w] = s0; sh[1][w] = s1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    S t0 = sc_zero<S>(), t1 = sc_zero<S>();
    for (int k = 0; k < kRedThreads / 32; ++k) { t0 += sh[0][k]; t1 += sh[1][k]; }
    part[2 * blockIdx.x] = t0;
    part[2 * blockIdx.x + 1] = t1;
  }
}

template <class S>
__global__ void dot2_final(const S* part, int nb, S* out0, S* out1) {
  __shared__ S sh[2][kRedThreads / 32];
  S s0 = sc_zero<S>(), s1 = sc_zero<S>();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) { s0 += part[2 * b]; s1 += part[2 * b + 1]; }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sh[0][w] = s0; sh[1][w] = s1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    S t0 = sc_zero<S>(), t1 = sc_zero<S>();
    for (int k = 0; k < kRedThreads / 32; ++k) { t0 += sh[0][k]; t1 += sh[1][k]; }
    *out0 = t0;
    if (out1) *out1 = t1;
  }
}

template <class S>
cudaError_t dot2(int n, const S* a0, const S* b0, const S* a1, const S* b1, S* part, S* out0, S* out1,
                 cudaStream_t s) {
  dot2_partial<S><<<kRedBlocks, kRedThreads, 0, s>>>(n, a0, b0, a1, b1, part);
  DIAF_COUNT_LAUNCH();
  dot2_final<S><<<1, kRedThreads, 0, s>>>(part, kRedBlocks, out0, out1);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <class S> __device__ __forceinline__ bool is_zero(S a) { return sc_abs2(a) == 0.0; }
template <class S> __device__ __forceinline__ S sdiv(S a, S b) { return (1.0 / sc_abs2(b)) * (a * sc_conj(b)); }

// rho = (rh, r); beta = (rho / rho_old) (alpha / omega)
template <class S>
__global__ void k_beta(KState<S>* st, int first) {
  S rho = st->dot[0];
  st->rho = rho;
  if (is_zero(rho)) { st->breakdown = 1; return; }
  st->beta = first ? sc_zero<S>() : sdiv(rho, st->rho_old) * sdiv(st->alpha, st->omega);
}
// alpha = rho / (rh, v)
template <class S>
__global__ void k_alpha(KState<S>* st) {
  if (st->breakdown) return;
  S den = st->dot[1];
  if (is_zero(den)) { st->breakdown = 2; return; }
  st->alpha = sdiv(st->rho, den);
}
// omega = (t, s) / (t, t)
template <class S>
__global__ void k_omega(KState<S>* st) {
  if (st->breakdown) return;
  S tt = st->dot[3];
  if (is_zero(tt)) { st->breakdown = 3; return; }
  st->omega = sdiv(st->dot[2], tt);
  st->rho_old = st->rho;
  if (is_zero(st->omega)) st->breakdown = 4;
}

// p = r + beta (p - omega v)
template <class S>
__global__ void k_update_p(int n, const KState<S>* st, const S* r, const S* v, S* p) {
  S beta = st->beta, omega = st->omega;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = r[i] + beta * (p[i] - omega * v[i]);
}
// s = r - alpha v ; xh = x + alpha ph
template <class S>
__global__ void k_update_s(int n, const KState<S>* st, const S* r, const S* v, const S* x, const S* ph, S* sv, S* xh) {
  S alpha = st->alpha;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    sv[i] = r[i] - alpha * v[i];
    xh[i] = x[i] + alpha * ph[i];
  }
}
// xn = xh + omega sh ; r = s - omega t
template <class S>
__global__ void k_update_x(int n, const KState<S>* st, const S* xh, const S* sh, const S* sv, const S* t, S* xn, S* r) {
  S omega = st->omega;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    xn[i] = xh[i] + omega * sh[i];
    r[i] = sv[i] - omega * t[i];
  }
}
template <class S>
__global__ void k_norms(KState<S>* st) {
  st->nrm[0] = sc_real(st->dot[0]);
  st->nrm[1] = sc_real(st->dot[1]);
}
template <class S>
__global__ void k_copy(int n, const S* a, S* b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = a[i];
}
template <class S>
__global__ void k_zero(int n, S* b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = sc_zero<S>();
}

template <class S>
diaf_status bicgstab_t(diaf_solver* SV, diaf_factors* F, const S* b, S* xout, double tol, int maxit,
                       cudaStream_t s, diaf_solve_info* info) {
  const int n = SV->n;
  const int vb = 304, vt = 256;
  S *r, *rh, *p, *v, *sv, *t, *ph, *sh, *x, *xh, *xn, *part;
  KState<S>* st;
  std::vector<void*> tmp;
  auto get = [&](S** q) -> cudaError_t {
    void* z = nullptr;
    cudaError_t e = cudaMallocAsync(&z, sizeof(S) * (n > 0 ? n : 1), s);
    if (e == cudaSuccess) { tmp.push_back(z); *q = (S*)z; }
    return e;
  };
  struct Free {
    std::vector<void*>& v;
    cudaStream_t s;
    ~Free() { for (void* p : v) cudaFreeAsync(p, s); }
  } fr{tmp, s};
  cudaError_t e = cudaSuccess;
  for (S** q : {&r, &rh, &p, &v, &sv, &t, &ph, &sh, &x, &xh, &xn}) {
    e = get(q);
    if (e != cudaSuccess) return DIAF_ENOMEM;
  }
  void* z = nullptr;
  if (cudaMallocAsync(&z, sizeof(S) * 2 * kRedBlocks, s) != cudaSuccess) return DIAF_ENOMEM;
  tmp.push_back(z); part = (S*)z;
  if (cudaMallocAsync(&z, sizeof(KState<S>), s) != cudaSuccess) return DIAF_ENOMEM;
  tmp.push_back(z); st = (KState<S>*)z;
  cudaMemsetAsync(st, 0, sizeof(KState<S>), s);
  // x0 = 0, r = b, rh = r
  k_zero<S><<<vb, vt, 0, s>>>(n, x);
  DIAF_COUNT_LAUNCH();
  k_zero<S><<<vb, vt, 0, s>>>(n, p);
  DIAF_COUNT_LAUNCH();
  k_zero<S><<<vb, vt, 0, s>>>(n, v);
  DIAF_COUNT_LAUNCH();
  k_copy<S><<<vb, vt, 0, s>>>(n, b, r);
  DIAF_COUNT_LAUNCH();
  k_copy<S><<<vb, vt, 0, s>>>(n, b, rh);
  DIAF_COUNT_LAUNCH();
  dot2<S>(n, r, r, nullptr, nullptr, part, &st->dot[0], nullptr, s);
  S h_dot;
  cudaMemcpyAsync(&h_dot, &st->dot[0], sizeof(S), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return DIAF_ECUDA;
  double r0n;
  {
    double re;
    memcpy(&re, &h_dot, sizeof(double));
    r0n = sqrt(re);
  }
  info->iterations = 0; info->converged = 0; info->breakdown = 0; info->relres = 0.0;
  if (r0n == 0.0) {
    k_copy<S><<<vb, vt, 0, s>>>(n, x, xout);
    DIAF_COUNT_LAUNCH();
    info->converged = 1;
    return DIAF_OK;
  }
  auto M = [&](const S* in, S* out) -> diaf_status {
    if (F) return diaf_apply(F, in, out, s);
    k_copy<S><<<vb, vt, 0, s>>>(n, in, out);
    DIAF_COUNT_LAUNCH();
    return DIAF_OK;
  };
  struct Host { double nrm[2]; int breakdown; } hst;
  for (int it = 1; it <= maxit; ++it) {
    dot2<S>(n, rh, r, nullptr, nullptr, part, &st->dot[0], nullptr, s);
    k_beta<S><<<1, 1, 0, s>>>(st, it == 1);
    DIAF_COUNT_LAUNCH();
    k_update_p<S><<<vb, vt, 0, s>>>(n, st, r, v, p);
    DIAF_COUNT_LAUNCH();
    diaf_status ms = M(p, ph);
    if (ms != DIAF_OK) return ms;
    csr_spmv(SV->A, SV->dtype == DIAF_C128, ph, v, s);
    dot2<S>(n, rh, v, nullptr, nullptr, part, &st->dot[1], nullptr, s);
    k_alpha<S><<<1, 1, 0, s>>>(st);
    DIAF_COUNT_LAUNCH();
    k_update_s<S><<<vb, vt, 0, s>>>(n, st, r, v, x, ph, sv, xh);
    DIAF_COUNT_LAUNCH();
    ms = M(sv, sh);
    if (ms != DIAF_OK) return ms;
    csr_spmv(SV->A, SV->dtype == DIAF_C128, sh, t, s);
    dot2<S>(n, t, sv, t, t, part, &st->dot[2], &st->dot[3], s);
    k_omega<S><<<1, 1, 0, s>>>(st);
    DIAF_COUNT_LAUNCH();
    k_update_x<S><<<vb, vt, 0, s>>>(n, st, xh, sh, sv, t, xn, r);
    DIAF_COUNT_LAUNCH();
    dot2<S>(n, sv, sv, r, r, part, &st->dot[0], &st->dot[1], s);
    k_norms<S><<<1, 1, 0, s>>>(st);
    DIAF_COUNT_LAUNCH();
    cudaMemcpyAsync(&hst.nrm, &st->nrm, sizeof(double) * 2, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&hst.breakdown, &st->breakdown, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return DIAF_ECUDA;
    const double sn = sqrt(hst.nrm[0]), rn = sqrt(hst.nrm[1]);
    info->iterations = it;
    int bd = hst.breakdown;
    if (bd == 1 || bd == 2) { info->breakdown = 1; info->relres = NAN; break; }  // x unchanged
    if (sn <= tol * r0n) {
      std::swap(x, xh);
      info->converged = 1;
      info->relres = sn / r0n;
      break;
    }
    if (bd == 3) { info->breakdown = 1; info->relres = sn / r0n; break; }
    std::swap(x, xn);
    info->relres = rn / r0n;
    if (rn <= tol * r0n) { info->converged = 1; break; }
    if (bd == 4) { info->breakdown = 1; break; }
  }
  k_copy<S><<<vb, vt, 0, s>>>(n, x, xout);
  DIAF_COUNT_LAUNCH();
  if (cudaStreamSynchronize(s) != cudaSuccess) return DIAF_ECUDA;
  return DIAF_OK;
}

// ------------------------------------------------------------------ GMRES(m)
// Right-preconditioned restarted GMRES (the solver of Sec. 5 for the complex
// problems): Arnoldi with classical Gram-Schmidt applied twice (two passes
// of one multi-dot and one multi-update each, so an iteration costs a fixed
// number of launches), Givens rotations on the device, x += M (V y) at the
// end of every cycle.  One device-to-host read per iteration: |g_{j+1}|.
constexpr int kGmresMax = 64;

template <class S>
struct GState {
  S H[(kGmresMax + 1) * kGmresMax];  // Hessenberg, column-major (ld kGmresMax + 1), rotated in place
  double cs[kGmresMax];              // rotations [c, s; -conj(s), c], c real
  S sn[kGmresMax];
  S g[kGmresMax + 1];
  S y[kGmresMax];
  S h[kGmresMax + 1];                // current Gram-Schmidt coefficients
  S dot;                             // scratch result
  double resid;                      // |g_{j+1}|
  double hnext;                      // H(j+1, j) (read together with resid)
};

// part[i * nb + block] = partial sum of conj(V_i) w over the block's elements
template <class S>
__global__ void k_mdot_partial(int n, const S* __restrict__ V, int cnt, const S* __restrict__ w, S* part) {
  __shared__ S sh[kRedThreads / 32];
  for (int i = 0; i < cnt; ++i) {
    const S* vi = V + (size_t)i * n;
    S acc = sc_zero<S>();
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
      acc += sc_cmul(vi[e], w[e]);
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      S t = sc_zero<S>();
      for (int k = 0; k < kRedThreads / 32; ++k) t += sh[k];
      part[(size_t)i * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// out[i] (+)= sum of part[i * nb ..]; one block per i
template <class S>
__global__ void k_mdot_final(const S* part, int nb, S* out, int accumulate) {
  __shared__ S sh[kRedThreads / 32];
  const int i = blockIdx.x;
  S acc = sc_zero<S>();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[(size_t)i * nb + b];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    S t = sc_zero<S>();
    for (int k = 0; k < kRedThreads / 32; ++k) t += sh[k];
    out[i] = accumulate ? out[i] + t : t;
  }
}

// w -= sum_i c[i] V_i
template <class S>
__global__ void k_mupdate(int n, const S* __restrict__ V, int cnt, const S* __restrict__ c, S* w) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    S acc = sc_zero<S>();
    for (int i = 0; i < cnt; ++i) acc += c[i] * V[(size_t)i * n + e];
    w[e] -= acc;
  }
}

// u = sum_i c[i] V_i
template <class S>
__global__ void k_combine(int n, const S* __restrict__ V, int cnt, const S* __restrict__ c, S* u) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    S acc = sc_zero<S>();
    for (int i = 0; i < cnt; ++i) acc += c[i] * V[(size_t)i * n + e];
    u[e] = acc;
  }
}

// v = w / ||w|| from the reduction result (||w||^2 in st->dot); H(j+1, j) = ||w||
template <class S>
__global__ void k_normalize(int n, GState<S>* st, int j, const S* w, S* v) {
  const double nrm = sqrt(fmax(sc_real(st->dot), 0.0));
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) v[e] = inv * w[e];
  if (blockIdx.x == 0 && threadIdx.x == 0) st->hnext = nrm;
}

// column j of H from h and hnext; old rotations, a new one, g updated
template <class S>
__global__ void k_givens(GState<S>* st, int j) {
  constexpr int LD = kGmresMax + 1;
  S* col = st->H + (size_t)j * LD;
  for (int i = 0; i <= j; ++i) col[i] = st->h[i];
  col[j + 1] = sc_real_s<S>(st->hnext);
  for (int i = 0; i < j; ++i) {
    const S a = col[i], b = col[i + 1];
    col[i] = st->cs[i] * a + st->sn[i] * b;
    col[i + 1] = st->cs[i] * b - sc_conj(st->sn[i]) * a;
  }
  const S a = col[j];
  const double bb = sc_real(col[j + 1]);  // a norm: real, >= 0
  const double aa = sqrt((double)sc_abs2(a));
  const double t = sqrt(aa * aa + bb * bb);
  double c;
  S sv;
  if (t == 0.0) {
    c = 1.0; sv = sc_zero<S>();
  } else if (aa == 0.0) {
    c = 0.0; sv = sc_real_s<S>(1.0);
  } else {
    c = aa / t;
    sv = (bb / (aa * t)) * a;  // (a / |a|) (b / t)
  }
  st->cs[j] = c;
  st->sn[j] = sv;
  col[j] = c * a + sv * col[j + 1];
  col[j + 1] = sc_zero<S>();
  const S gj = st->g[j];
  st->g[j + 1] = -(sc_conj(sv) * gj);
  st->g[j] = c * gj;
  st->resid = sqrt((double)sc_abs2(st->g[j + 1]));
}

// y = R^-1 g for the rotated k x k upper triangle; zero pivots give 0
template <class S>
__global__ void k_backsolve(GState<S>* st, int k) {
  constexpr int LD = kGmresMax + 1;
  for (int i = k - 1; i >= 0; --i) {
    S acc = st->g[i];
    for (int t = i + 1; t < k; ++t) acc -= st->H[i + (size_t)t * LD] * st->y[t];
    const S d = st->H[i + (size_t)i * LD];
    st->y[i] = sc_abs2(d) > 0.0 ? sdiv(acc, d) : sc_zero<S>();
  }
}

// start of a cycle: g = (beta, 0, ...), v_0 = r / beta (beta from st->dot)
template <class S>
__global__ void k_cycle_start(int n, GState<S>* st, const S* r, S* v0) {
  const double beta = sqrt(fmax(sc_real(st->dot), 0.0));
  const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) v0[e] = inv * r[e];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int i = 0; i <= kGmresMax; ++i) st->g[i] = sc_zero<S>();
    st->g[0] = sc_real_s<S>(beta);
    st->resid = beta;
  }
}

template <class S>
__global__ void k_add_small(int cnt, const S* a, S* h) {  // h += a (cnt <= blockDim)
  if ((int)threadIdx.x < cnt) h[threadIdx.x] += a[threadIdx.x];
}

template <class S>
__global__ void k_axpy1(int n, const S* a, S* x) {  // x += a
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) x[e] += a[e];
}
template <class S>
__global__ void k_sub(int n, const S* a, const S* b, S* out) {  // out = a - b
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) out[e] = a[e] - b[e];
}

template <class S>
diaf_status gmres_t(diaf_solver* SV, diaf_factors* F, const S* b, S* xout, double tol, int m, int maxit,
                    cudaStream_t s, diaf_solve_info* info) {
  const int n = SV->n;
  const int vb = 304, vt = 256;
  std::vector<void*> tmp;
  struct Free {
    std::vector<void*>& v;
    cudaStream_t s;
    ~Free() { for (void* p : v) cudaFreeAsync(p, s); }
  } fr{tmp, s};
  auto get = [&](void** q, size_t bytes) -> bool {
    void* z = nullptr;
    if (cudaMallocAsync(&z, bytes > 0 ? bytes : 1, s) != cudaSuccess) return false;
    tmp.push_back(z);
    *q = z;
    return true;
  };
  S *V, *w, *x, *r, *u, *z, *part;
  GState<S>* st;
  const size_t nv = sizeof(S) * (size_t)(n > 0 ? n : 1);
  if (!get((void**)&V, nv * (m + 1)) || !get((void**)&w, nv) || !get((void**)&x, nv) || !get((void**)&r, nv) ||
      !get((void**)&u, nv) || !get((void**)&z, nv) ||
      !get((void**)&part, sizeof(S) * (size_t)kRedBlocks * (kGmresMax + 1)) || !get((void**)&st, sizeof(GState<S>)))
    return DIAF_ENOMEM;
  cudaMemsetAsync(st, 0, sizeof(GState<S>), s);
  info->iterations = 0; info->converged = 0; info->breakdown = 0; info->relres = 0.0;
  auto M = [&](const S* in, S* out) -> diaf_status {
    if (F) return diaf_apply(F, in, out, s);
    k_copy<S><<<vb, vt, 0, s>>>(n, in, out);
    DIAF_COUNT_LAUNCH();
    return DIAF_OK;
  };
  auto norm2_to_dot = [&](const S* a) {
    dot2<S>(n, a, a, nullptr, nullptr, part, &st->dot, nullptr, s);
  };
  auto read = [&](const double* dp) -> double {
    double h = 0.0;
    cudaMemcpyAsync(&h, dp, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return NAN;
    return h;
  };
  k_zero<S><<<vb, vt, 0, s>>>(n, x);
  DIAF_COUNT_LAUNCH();
  k_copy<S><<<vb, vt, 0, s>>>(n, b, r);
  DIAF_COUNT_LAUNCH();
  norm2_to_dot(r);
  k_cycle_start<S><<<vb, vt, 0, s>>>(n, st, r, V);
  DIAF_COUNT_LAUNCH();
  const double bn = read(&st->resid);
  if (!(bn == bn)) return DIAF_ECUDA;
  if (bn == 0.0) {
    k_copy<S><<<vb, vt, 0, s>>>(n, x, xout);
    DIAF_COUNT_LAUNCH();
    info->converged = 1;
    return cudaStreamSynchronize(s) == cudaSuccess ? DIAF_OK : DIAF_ECUDA;
  }
  int its = 0;
  double rel = 1.0;
  while (its < maxit) {
    int kdone = 0;
    bool happy = false;
    for (int j = 0; j < m && its < maxit; ++j) {
      S* vj = V + (size_t)j * n;
      diaf_status ms = M(vj, z);
      if (ms != DIAF_OK) return ms;
      csr_spmv(SV->A, SV->dtype == DIAF_C128, z, w, s);
      // classical Gram-Schmidt, twice: h = V^* w, w -= V h; c = V^* w, w -= V c, h += c
      k_mdot_partial<S><<<kRedBlocks, kRedThreads, 0, s>>>(n, V, j + 1, w, part);
      DIAF_COUNT_LAUNCH();
      k_mdot_final<S><<<j + 1, kRedThreads, 0, s>>>(part, kRedBlocks, st->h, 0);
      DIAF_COUNT_LAUNCH();
      k_mupdate<S><<<vb, vt, 0, s>>>(n, V, j + 1, st->h, w);
      DIAF_COUNT_LAUNCH();
      k_mdot_partial<S><<<kRedBlocks, kRedThreads, 0, s>>>(n, V, j + 1, w, part);
      DIAF_COUNT_LAUNCH();
      k_mdot_final<S><<<j + 1, kRedThreads, 0, s>>>(part, kRedBlocks, st->y, 0);  // y: scratch until the cycle ends
      DIAF_COUNT_LAUNCH();
      k_mupdate<S><<<vb, vt, 0, s>>>(n, V, j + 1, st->y, w);
      DIAF_COUNT_LAUNCH();
      k_add_small<S><<<1, kGmresMax, 0, s>>>(j + 1, st->y, st->h);
      DIAF_COUNT_LAUNCH();
      norm2_to_dot(w);
      k_normalize<S><<<vb, vt, 0, s>>>(n, st, j, w, V + (size_t)(j + 1) * n);
      DIAF_COUNT_LAUNCH();
      k_givens<S><<<1, 1, 0, s>>>(st, j);
      DIAF_COUNT_LAUNCH();
      ++its;
      kdone = j + 1;
      double rh[2] = {NAN, NAN};  // resid and hnext are adjacent: one read
      cudaMemcpyAsync(rh, &st->resid, sizeof(double) * 2, cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) return DIAF_ECUDA;
      if (!(rh[0] == rh[0])) { info->breakdown = 1; break; }
      rel = rh[0] / bn;
      if (rel <= tol || rh[1] == 0.0) { happy = rh[1] == 0.0; break; }
    }
    if (info->breakdown) break;
    k_backsolve<S><<<1, 1, 0, s>>>(st, kdone);
    DIAF_COUNT_LAUNCH();
    k_combine<S><<<vb, vt, 0, s>>>(n, V, kdone, st->y, u);
    DIAF_COUNT_LAUNCH();
    diaf_status ms = M(u, z);
    if (ms != DIAF_OK) return ms;
    k_axpy1<S><<<vb, vt, 0, s>>>(n, z, x);
    DIAF_COUNT_LAUNCH();
    // true residual, next cycle
    csr_spmv(SV->A, SV->dtype == DIAF_C128, x, w, s);
    k_sub<S><<<vb, vt, 0, s>>>(n, b, w, r);
    DIAF_COUNT_LAUNCH();
    norm2_to_dot(r);
    k_cycle_start<S><<<vb, vt, 0, s>>>(n, st, r, V);
    DIAF_COUNT_LAUNCH();
    rel = read(&st->resid) / bn;
    if (rel <= tol) { info->converged = 1; break; }
    if (happy) break;
  }
  info->iterations = its;
  info->relres = rel;
  k_copy<S><<<vb, vt, 0, s>>>(n, x, xout);
  DIAF_COUNT_LAUNCH();
  return cudaStreamSynchronize(s) == cudaSuccess ? DIAF_OK : DIAF_ECUDA;
}

}  // namespace

extern "C" {

diaf_status diaf_solver_create(const diaf_csc* A, void* stream, diaf_solver** out) {
  if (!A || !out) return DIAF_EINVAL;
  *out = nullptr;
  if (A->n < 0 || (A->dtype != DIAF_F64 && A->dtype != DIAF_C128)) return DIAF_EINVAL;
  auto S = new diaf_solver();
  S->stream = static_cast<cudaStream_t>(stream);
  S->n = A->n;
  S->dtype = A->dtype;
  const bool cplx = A->dtype == DIAF_C128;
  const size_t esz = cplx ? 16 : 8;
  int32_t* work = nullptr;
  bool ok = salloc(S, &S->A.rowptr, A->n + 1) == cudaSuccess && salloc(S, &S->A.colidx, A->nnz) == cudaSuccess &&
            salloc(S, (char**)&S->A.vals, esz * A->nnz) == cudaSuccess &&
            salloc(S, &work, A->n + scan_blocksums_size(A->n)) == cudaSuccess;
  if (!ok) { diaf_solver_free(S); return DIAF_ENOMEM; }
  S->A.n = A->n;
  S->A.nnz = A->nnz;
  if (csc_to_csr(A->n, A->nnz, A->colptr, A->rowidx, A->vals, cplx, S->A.rowptr, S->A.colidx, S->A.vals, work,
                 S->stream) != cudaSuccess) {
    diaf_solver_free(S);
    return DIAF_ECUDA;
  }
  *out = S;
  return DIAF_OK;
}

void diaf_solver_free(diaf_solver* S) {
  if (!S) return;
  for (void* p : S->owned) cudaFreeAsync(p, S->stream);
  delete S;
}

diaf_status diaf_gmres(diaf_solver* S, diaf_factors* F, const void* b, void* x, double tol, int32_t restart,
                       int32_t maxit, void* stream, diaf_solve_info* info) {
  if (!S || !b || !x || !info || maxit < 0 || restart < 1 || restart > kGmresMax) return DIAF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (S->dtype == DIAF_C128)
    return gmres_t<Cx<double>>(S, F, (const Cx<double>*)b, (Cx<double>*)x, tol, restart, maxit, s, info);
  return gmres_t<double>(S, F, (const double*)b, (double*)x, tol, restart, maxit, s, info);
}

diaf_status diaf_bicgstab(diaf_solver* S, diaf_factors* F, const void* b, void* x, double tol, int32_t maxit,
                          void* stream, diaf_solve_info* info) {
  if (!S || !b || !x || !info || maxit < 0) return DIAF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (S->dtype == DIAF_C128)
    return bicgstab_t<Cx<double>>(S, F, (const Cx<double>*)b, (Cx<double>*)x, tol, maxit, s, info);
  return bicgstab_t<double>(S, F, (const double*)b, (double*)x, tol, maxit, s, info);
}

}  // extern "C"
