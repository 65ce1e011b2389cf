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

diaf_status diaf_bicgstab(diaf_solver* S, diaf_factors* F, const void* b, void* x, double tol, int32_t maxit,
                          void* stream, diaf_solve_info* info) {
  if (!S || !b || !x || !info || maxit < 0) return DIAF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (S->dtype == DIAF_C128)
    return bicgstab_t<Cx<double>>(S, F, (const Cx<double>*)b, (Cx<double>*)x, tol, maxit, s, info);
  return bicgstab_t<double>(S, F, (const double*)b, (double*)x, tol, maxit, s, info);
}

}  // extern "C"
