// Learned proposal of the W pattern J_j (not part of the paper: the paper's
// W-pattern heuristics are in Sec. 4 and stay the fallback).  For every
// column j and candidate row c of a candidate pattern CAND(:,j) (e.g.
// pattern(A^2)): eight local features, an MLP 8 -> 32 -> 32 -> 1 with ReLU
// scoring the candidate, and the selection of the diagonal plus the best
// keep-1 candidates.  Training: mean squared error of the score against a
// per-candidate target, backward pass, Adam.
#include <string>

#include "factors.cuh"

namespace {

constexpr int F = DIAF_PROP_NFEAT;
constexpr int H = DIAF_PROP_HIDDEN;
// parameter layout: W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * F, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H, NPARAM = OFF_B3 + 1;
static_assert(NPARAM == DIAF_PROP_NPARAM, "parameter count");
constexpr int kCandMax = 128;  // candidates of one column (e.g. pattern(A^3) of a 7-point stencil: 63)
constexpr int kCandPerLane = kCandMax / 32;
constexpr int kFeatWarps = 8;

__device__ __forceinline__ int find_sorted(const int32_t* a, int n, int key) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int v = a[mid];
    if (v == key) return mid;
    if (v < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// |value| of the entry (row, col) of A, 0 when absent (binary search in the column)
template <class S>
__device__ __forceinline__ double entry_abs(const int32_t* Acp, const int32_t* Ari, const S* Av, int row, int col) {
  const int a0 = Acp[col];
  const int pos = find_sorted(Ari + a0, Acp[col + 1] - a0, row);
  return pos >= 0 ? sqrt((double)sc_abs2(Av[a0 + pos])) : 0.0;
}

// Features of candidate c of column j (one warp per column; lane l takes the
// candidates l, l + 32, l + 64, l + 96):
//   f0 diagonal (c == j)            f1 c is a row of A(:,j)
//   f2 |A_cj| / max_i |A_ij|        f3 |(A^2)_cj| / max over candidates |(A^2)_c'j|
//   f4 log(|a_cc| / |a_jj|) in [-10, 10]
//   f5 |A_jc| / |a_jj|              f6 nnz(A(:,c)) / nnz(A(:,j))
//   f7 +1 for c < j, -1 for c > j, 0 on the diagonal
template <class S>
__global__ void __launch_bounds__(kFeatWarps * 32)
    features_kernel(int n, const int32_t* __restrict__ Acp, const int32_t* __restrict__ Ari, const S* __restrict__ Av,
                    const int32_t* __restrict__ Ccp, const int32_t* __restrict__ Cri, float* __restrict__ feat,
                    uint32_t* status) {
  __shared__ int32_t cand[kFeatWarps][kCandMax];
  __shared__ S acc[kFeatWarps][kCandMax];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int j = blockIdx.x * kFeatWarps + wib;
  if (j >= n) return;  // warp-uniform
  const int c0 = Ccp[j], nc = Ccp[j + 1] - c0;
  if (nc > kCandMax) {
    if (lane == 0) atomicOr(status, DEV_ST_CAPACITY);
    return;
  }
  int cl[kCandPerLane];
  bool bad = false;
#pragma unroll
  for (int u = 0; u < kCandPerLane; ++u) {
    const int i = lane + 32 * u;
    cl[u] = i < nc ? Cri[c0 + i] : -1;
    bad |= i < nc && (cl[u] < 0 || cl[u] >= n);
  }
  if (__any_sync(DIAF_FULL, bad)) {
    if (lane == 0) atomicOr(status, DEV_ST_BAD_INPUT);
    return;
  }
#pragma unroll
  for (int u = 0; u < kCandPerLane; ++u) {
    cand[wib][lane + 32 * u] = lane + 32 * u < nc ? cl[u] : INT_MAX;
    acc[wib][lane + 32 * u] = sc_zero<S>();
  }
  __syncwarp();
  const int a0 = Acp[j], na = Acp[j + 1] - a0;
  double aj_max = 0.0, ajj = 0.0;
  double acj[kCandPerLane];
#pragma unroll
  for (int u = 0; u < kCandPerLane; ++u) acj[u] = 0.0;
  for (int p = 0; p < na; ++p) {
    const int r = Ari[a0 + p];
    const double v = sqrt((double)sc_abs2(Av[a0 + p]));
    aj_max = v > aj_max ? v : aj_max;
    if (r == j) ajj = v;
#pragma unroll
    for (int u = 0; u < kCandPerLane; ++u)
      if (r == cl[u]) acj[u] = v;
  }
  // (A^2)(c, j) = sum_k A(c, k) A(k, j): rows within one column k are distinct,
  // so the lanes of one k update distinct slots
  for (int p = 0; p < na; ++p) {
    const int kcol = Ari[a0 + p];
    if (kcol < 0 || kcol >= n) {  // warp-uniform
      if (lane == 0) atomicOr(status, DEV_ST_BAD_INPUT);
      return;
    }
    const S akj = Av[a0 + p];
    const int b0 = Acp[kcol], nb = Acp[kcol + 1] - b0;
    for (int q = lane; q < nb; q += 32) {
      const int pos = find_sorted(cand[wib], nc, Ari[b0 + q]);
      if (pos >= 0) acc[wib][pos] += Av[b0 + q] * akj;
    }
    __syncwarp();
  }
  double a2c[kCandPerLane];
  double a2m = 0.0;
#pragma unroll
  for (int u = 0; u < kCandPerLane; ++u) {
    const int i = lane + 32 * u;
    a2c[u] = i < nc ? sqrt((double)sc_abs2(acc[wib][i])) : 0.0;
    a2m = a2c[u] > a2m ? a2c[u] : a2m;
  }
  const double a2max = warp_max(a2m);
#pragma unroll
  for (int u = 0; u < kCandPerLane; ++u) {
    const int i = lane + 32 * u;
    if (i >= nc) continue;
    const int c = cl[u];
    const double acc_diag = entry_abs(Acp, Ari, Av, c, c);
    const double ajc = entry_abs(Acp, Ari, Av, j, c);
    float* f = feat + (size_t)(c0 + i) * F;
    f[0] = c == j ? 1.0f : 0.0f;
    f[1] = acj[u] > 0.0 ? 1.0f : 0.0f;
    f[2] = aj_max > 0.0 ? (float)(acj[u] / aj_max) : 0.0f;
    f[3] = a2max > 0.0 ? (float)(a2c[u] / a2max) : 0.0f;
    double lr = (acc_diag > 0.0 && ajj > 0.0) ? log(acc_diag / ajj) : 0.0;
    f[4] = (float)(lr > 10.0 ? 10.0 : (lr < -10.0 ? -10.0 : lr));
    f[5] = ajj > 0.0 ? (float)(ajc / ajj) : 0.0f;
    f[6] = na > 0 ? (float)(Acp[c + 1] - Acp[c]) / (float)na : 0.0f;
    f[7] = c < j ? 1.0f : (c > j ? -1.0f : 0.0f);
  }
}

// ---------------------------------------------------------------- MLP
struct Fwd {
  float h1[H], h2[H], y;
};

__device__ __forceinline__ void mlp_fwd(const float* P, const float* f, Fwd& o) {
#pragma unroll
  for (int h = 0; h < H; ++h) {
    float s = P[OFF_B1 + h];
#pragma unroll
    for (int i = 0; i < F; ++i) s = fmaf(P[OFF_W1 + h * F + i], f[i], s);
    o.h1[h] = s > 0.0f ? s : 0.0f;
  }
#pragma unroll 4
  for (int h = 0; h < H; ++h) {
    float s = P[OFF_B2 + h];
#pragma unroll
    for (int g = 0; g < H; ++g) s = fmaf(P[OFF_W2 + h * H + g], o.h1[g], s);
    o.h2[h] = s > 0.0f ? s : 0.0f;
  }
  float y = P[OFF_B3];
#pragma unroll
  for (int h = 0; h < H; ++h) y = fmaf(P[OFF_W3 + h], o.h2[h], y);
  o.y = y;
}

__global__ void mlp_forward_kernel(const float* __restrict__ params, const float* __restrict__ feat, int64_t nrows,
                                   float* __restrict__ out) {
  __shared__ float P[NPARAM];
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) P[i] = params[i];
  __syncthreads();
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nrows; s += (int64_t)gridDim.x * blockDim.x) {
    float f[F];
#pragma unroll
    for (int i = 0; i < F; ++i) f[i] = feat[s * F + i];
    Fwd o;
    mlp_fwd(P, f, o);
    out[s] = o.y;
  }
}

// Gradient of L = (1/nrows) sum_s (y_s - t_s)^2 for a block of kGradRows
// samples: per-sample backward into shared memory, then every parameter's
// gradient as a sum over the block's samples, written to the block's row of
// `part` (NPARAM + 1 floats: the gradient, then the loss); the blocks' rows
// are summed in block order afterwards, so the result is reproducible.
constexpr int kGradRows = 128;
constexpr int kPartLd = NPARAM + 1;

__global__ void __launch_bounds__(kGradRows)
    mlp_grad_kernel(const float* __restrict__ params, const float* __restrict__ feat, const float* __restrict__ target,
                    int64_t nrows, float* __restrict__ part) {
  extern __shared__ float sm[];
  float* P = sm;                        // NPARAM
  float* sF = P + NPARAM;               // [kGradRows][F]
  float* sH1 = sF + kGradRows * F;      // [kGradRows][H]
  float* sH2 = sH1 + kGradRows * H;     // [kGradRows][H]
  float* sD1 = sH2 + kGradRows * H;     // dL/d(pre-activation 1)
  float* sD2 = sD1 + kGradRows * H;     // dL/d(pre-activation 2)
  float* sDy = sD2 + kGradRows * H;     // [kGradRows]
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) P[i] = params[i];
  __syncthreads();
  const int64_t s = blockIdx.x * (int64_t)kGradRows + threadIdx.x;
  const int t = threadIdx.x;
  float l2 = 0.0f;
  if (s < nrows) {
    float f[F];
#pragma unroll
    for (int i = 0; i < F; ++i) f[i] = sF[t * F + i] = feat[s * F + i];
    Fwd o;
    mlp_fwd(P, f, o);
    const float e = o.y - target[s];
    l2 = e * e;
    const float dy = 2.0f * e / (float)nrows;
    sDy[t] = dy;
    float d2[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
      d2[h] = o.h2[h] > 0.0f ? dy * P[OFF_W3 + h] : 0.0f;
      sH1[t * H + h] = o.h1[h];
      sH2[t * H + h] = o.h2[h];
      sD2[t * H + h] = d2[h];
    }
#pragma unroll 4
    for (int g = 0; g < H; ++g) {
      float sacc = 0.0f;
#pragma unroll
      for (int h = 0; h < H; ++h) sacc = fmaf(P[OFF_W2 + h * H + g], d2[h], sacc);
      sD1[t * H + g] = o.h1[g] > 0.0f ? sacc : 0.0f;
    }
  } else {
    sDy[t] = 0.0f;
#pragma unroll
    for (int i = 0; i < F; ++i) sF[t * F + i] = 0.0f;
    for (int h = 0; h < H; ++h) sH1[t * H + h] = sH2[t * H + h] = sD1[t * H + h] = sD2[t * H + h] = 0.0f;
  }
  __syncthreads();
  const int rows = (int)((nrows - blockIdx.x * (int64_t)kGradRows) < kGradRows ? (nrows - blockIdx.x * (int64_t)kGradRows)
                                                                              : kGradRows);
  for (int p = threadIdx.x; p < NPARAM; p += blockDim.x) {
    float g = 0.0f;
    if (p < OFF_B1) {  // W1[h][i] = sum_s d1[s][h] f[s][i]
      const int h = p / F, i = p % F;
      for (int r = 0; r < rows; ++r) g = fmaf(sD1[r * H + h], sF[r * F + i], g);
    } else if (p < OFF_W2) {
      const int h = p - OFF_B1;
      for (int r = 0; r < rows; ++r) g += sD1[r * H + h];
    } else if (p < OFF_B2) {  // W2[h][q] = sum_s d2[s][h] h1[s][q]
      const int h = (p - OFF_W2) / H, q = (p - OFF_W2) % H;
      for (int r = 0; r < rows; ++r) g = fmaf(sD2[r * H + h], sH1[r * H + q], g);
    } else if (p < OFF_W3) {
      const int h = p - OFF_B2;
      for (int r = 0; r < rows; ++r) g += sD2[r * H + h];
    } else if (p < OFF_B3) {  // w3[h] = sum_s dy[s] h2[s][h]
      const int h = p - OFF_W3;
      for (int r = 0; r < rows; ++r) g = fmaf(sDy[r], sH2[r * H + h], g);
    } else {
      for (int r = 0; r < rows; ++r) g += sDy[r];
    }
    part[(size_t)blockIdx.x * kPartLd + p] = g;
  }
  l2 = warp_sum(l2);
  __shared__ float red[kGradRows / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l2;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tot = 0.0f;
    for (int w = 0; w < kGradRows / 32; ++w) tot += red[w];
    part[(size_t)blockIdx.x * kPartLd + NPARAM] = tot / (float)nrows;
  }
}

// grad[p] = sum over blocks of part[b][p] (in block order); loss likewise
__global__ void grad_reduce_kernel(const float* __restrict__ part, int nblocks, float* __restrict__ grad,
                                   float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > NPARAM) return;
  float acc = 0.0f;
  for (int b = 0; b < nblocks; ++b) acc += part[(size_t)b * kPartLd + p];
  if (p < NPARAM) grad[p] = acc;
  else *loss = acc;
}

__global__ void adam_kernel(float* __restrict__ params, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, int step, float lr, float b1, float b2, float eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  const float g = grad[p];
  const float mm = b1 * m[p] + (1.0f - b1) * g;
  const float vv = b2 * v[p] + (1.0f - b2) * g * g;
  m[p] = mm;
  v[p] = vv;
  const float mh = mm / (1.0f - powf(b1, (float)step));
  const float vh = vv / (1.0f - powf(b2, (float)step));
  params[p] -= lr * mh / (sqrtf(vh) + eps);
}

// ---------------------------------------------------------------- selection
__global__ void keep_count_kernel(int n, const int32_t* Ccp, int keep, int32_t* cnt, uint32_t* status) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int nc = Ccp[j + 1] - Ccp[j];
  cnt[j] = nc < keep ? nc : keep;
  if (nc > kCandMax) atomicOr(status, DEV_ST_CAPACITY);
}

// Warp per column: the diagonal always, then the candidates by decreasing
// score (ties to the lower row); the kept rows are written in increasing
// order.  Lane l ranks the candidates l, l + 32, l + 64, l + 96 against all
// of the column's candidates (staged in shared memory).
constexpr int kSelWarps = 8;
__global__ void __launch_bounds__(kSelWarps * 32)
    select_kernel(int n, const int32_t* __restrict__ Ccp, const int32_t* __restrict__ Cri,
                  const float* __restrict__ score, int keep, const int32_t* __restrict__ outcp,
                  int32_t* __restrict__ outri) {
  __shared__ int32_t sc_c[kSelWarps][kCandMax];
  __shared__ float sc_s[kSelWarps][kCandMax];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int j = blockIdx.x * kSelWarps + wib;
  if (j >= n) return;  // warp-uniform
  const int c0 = Ccp[j], nc = Ccp[j + 1] - c0;
  if (nc > kCandMax) return;  // reported by keep_count_kernel
  int cl[kCandPerLane];
  float sl[kCandPerLane];
#pragma unroll
  for (int u = 0; u < kCandPerLane; ++u) {
    const int i = lane + 32 * u;
    cl[u] = i < nc ? Cri[c0 + i] : INT_MAX;
    float sc = i < nc ? score[c0 + i] : -INFINITY;
    if (cl[u] == j) sc = INFINITY;
    if (!(sc == sc)) sc = -INFINITY;  // NaN scores rank last
    sl[u] = sc;
    sc_c[wib][i] = cl[u];
    sc_s[wib][i] = sc;
  }
  __syncwarp();
  const int kj = nc < keep ? nc : keep;
  int before = 0;  // kept candidates in the slots of earlier rounds
#pragma unroll
  for (int u = 0; u < kCandPerLane; ++u) {
    const int i = lane + 32 * u;
    int rank = 0;
    if (i < nc)
      for (int o = 0; o < nc; ++o) {
        const float so = sc_s[wib][o];
        const int co = sc_c[wib][o];
        if (so > sl[u] || (so == sl[u] && co < cl[u])) ++rank;
      }
    const bool kept = i < nc && rank < kj;
    const unsigned b = __ballot_sync(DIAF_FULL, kept);
    if (kept) outri[outcp[j] + before + __popc(b & ((1u << lane) - 1u))] = cl[u];
    before += __popc(b);
  }
}

// Per column: res_j / |V(j, j)| (infinity when V(j, j) is zero or absent).
template <class S>
__global__ void scaled_residuals_kernel(int n, const double* __restrict__ res, const int32_t* __restrict__ Vcp,
                                        const int32_t* __restrict__ Vri, const S* __restrict__ Vv,
                                        double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double d = 0.0;
  for (int p = Vcp[j]; p < Vcp[j + 1]; ++p)
    if (Vri[p] == j) d = sqrt((double)sc_abs2(Vv[p]));
  out[j] = d > 0.0 ? res[j] / d : INFINITY;
}

// The largest finite r_j^2 (one block; atomicMax on the bits of a
// non-negative double orders like the value).
__global__ void max_finite_sq_kernel(int n, const double* __restrict__ r, unsigned long long* out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double v = r[j] * r[j];
    if (isfinite(v) && v > m) m = v;
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    m = warp_max(m);
    if (threadIdx.x == 0) *out = (unsigned long long)__double_as_longlong(m);
  }
}

// Toggle target of candidate slot `slot` of every column (not the diagonal):
// with L(r) = log(min(max(r^2, floor), cap)) (non-finite r counts as cap),
// floor = 1e-30 max(M, 1e-300) and cap = 1e30 M for M the largest finite
// r0^2 (1 when no r0_j^2 is finite and positive), the value is
// L(rt_j) - L(r0_j) for a candidate in the base pattern (dropped) and
// L(r0_j) - L(rt_j) otherwise (added), clipped to [-clip, clip].
__global__ void toggle_targets_kernel(int n, const int32_t* __restrict__ Ccp, const int32_t* __restrict__ Cri,
                                      const uint8_t* __restrict__ in_base, const double* __restrict__ r0,
                                      const double* __restrict__ rt, int slot, double clip,
                                      const unsigned long long* __restrict__ mbits, double* __restrict__ value) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int e = Ccp[j] + slot;
  if (e >= Ccp[j + 1] || Cri[e] == j) return;
  double M = __longlong_as_double((long long)*mbits);
  if (!(M > 0.0)) M = 1.0;
  const double lo = fmax(M, 1e-300) * 1e-30, hi = 1e30 * M;
  auto L = [&](double r) {
    const double v = r * r;
    return log(isfinite(v) ? fmin(fmax(v, lo), hi) : hi);
  };
  const double d = L(rt[j]) - L(r0[j]);
  const double t = in_base[e] ? d : -d;
  value[e] = fmin(fmax(t, -clip), clip);
}

}  // namespace

extern "C" {

diaf_status diaf_propose_features(const diaf_csc* A, const diaf_pattern* CAND, float* d_feat, void* stream) {
  if (!A || !CAND || (CAND->nnz > 0 && !d_feat) || CAND->n != A->n) {
    diaf_set_last_error("A, CAND and feat must be given, of equal size");
    return DIAF_EINVAL;
  }
  const int n = A->n;
  if (n == 0) return DIAF_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t* st = nullptr;
  if (cudaMallocAsync(&st, sizeof(uint32_t), s) != cudaSuccess) return DIAF_ENOMEM;
  cudaMemsetAsync(st, 0, sizeof(uint32_t), s);
  const int blocks = ceil_div(n, kFeatWarps);
  if (A->dtype == DIAF_C128)
    features_kernel<Cx<double>><<<blocks, kFeatWarps * 32, 0, s>>>(n, A->colptr, A->rowidx, (const Cx<double>*)A->vals,
                                                                 CAND->colptr, CAND->rowidx, d_feat, st);
  else
    features_kernel<double><<<blocks, kFeatWarps * 32, 0, s>>>(n, A->colptr, A->rowidx, (const double*)A->vals,
                                                             CAND->colptr, CAND->rowidx, d_feat, st);
  DIAF_COUNT_LAUNCH();
  uint32_t h = 0;
  cudaMemcpyAsync(&h, st, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(st, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return DIAF_ECUDA;
  if (h & DEV_ST_BAD_INPUT) {
    diaf_set_last_error("a row index of A or CAND is out of range");
    return DIAF_EINVAL;
  }
  if (h & DEV_ST_CAPACITY) {
    diaf_set_last_error("a column has more than 128 candidates");
    return DIAF_EUNSUPPORTED;
  }
  return DIAF_OK;
}

diaf_status diaf_mlp_forward(const float* d_params, const float* d_feat, int64_t nrows, float* d_out, void* stream) {
  if (nrows < 0 || (nrows > 0 && (!d_params || !d_feat || !d_out))) return DIAF_EINVAL;
  if (nrows == 0) return DIAF_OK;
  int blocks = (int)((nrows + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  mlp_forward_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_params, d_feat, nrows, d_out);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError() == cudaSuccess ? DIAF_OK : DIAF_ECUDA;
}

diaf_status diaf_mlp_grad(const float* d_params, const float* d_feat, const float* d_target, int64_t nrows,
                          float* d_grad, float* d_loss, void* stream) {
  if (nrows <= 0 || !d_params || !d_feat || !d_target || !d_grad || !d_loss) return DIAF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t smem = sizeof(float) * (NPARAM + kGradRows * (F + 4 * H + 1));
  static bool configured = false;
  if (!configured) {
    if (cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return DIAF_ECUDA;
    configured = true;
  }
  const int64_t nb64 = (nrows + kGradRows - 1) / kGradRows;
  if (nb64 > INT_MAX) return DIAF_EINVAL;
  const int blocks = (int)nb64;
  float* part = nullptr;
  if (cudaMallocAsync(&part, sizeof(float) * (size_t)blocks * kPartLd, s) != cudaSuccess) return DIAF_ENOMEM;
  mlp_grad_kernel<<<blocks, kGradRows, smem, s>>>(d_params, d_feat, d_target, nrows, part);
  DIAF_COUNT_LAUNCH();
  grad_reduce_kernel<<<ceil_div(kPartLd, 256), 256, 0, s>>>(part, blocks, d_grad, d_loss);
  DIAF_COUNT_LAUNCH();
  cudaFreeAsync(part, s);
  return cudaGetLastError() == cudaSuccess ? DIAF_OK : DIAF_ECUDA;
}

diaf_status diaf_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, int32_t step, float lr,
                          void* stream) {
  if (!d_params || !d_grad || !d_m || !d_v || step < 1) return DIAF_EINVAL;
  adam_kernel<<<ceil_div(NPARAM, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(d_params, d_grad, d_m, d_v, step, lr,
                                                                                    0.9f, 0.999f, 1e-8f);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError() == cudaSuccess ? DIAF_OK : DIAF_ECUDA;
}

diaf_status diaf_propose_select(const diaf_pattern* CAND, const float* d_score, int32_t keep, int32_t* d_colptr,
                                int32_t* d_rowidx, void* stream) {
  if (!CAND || keep < 1 || !d_colptr || (CAND->nnz > 0 && (!d_score || !d_rowidx))) return DIAF_EINVAL;
  const int n = CAND->n;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n == 0) return cudaMemsetAsync(d_colptr, 0, sizeof(int32_t), s) == cudaSuccess ? DIAF_OK : DIAF_ECUDA;
  int32_t *cnt = nullptr, *bs = nullptr;
  uint32_t* st = nullptr;
  if (cudaMallocAsync(&cnt, sizeof(int32_t) * n, s) != cudaSuccess) return DIAF_ENOMEM;
  if (cudaMallocAsync(&bs, sizeof(int32_t) * scan_blocksums_size(n), s) != cudaSuccess) {
    cudaFreeAsync(cnt, s);
    return DIAF_ENOMEM;
  }
  if (cudaMallocAsync(&st, sizeof(uint32_t), s) != cudaSuccess) {
    cudaFreeAsync(cnt, s);
    cudaFreeAsync(bs, s);
    return DIAF_ENOMEM;
  }
  cudaError_t e = cudaMemsetAsync(st, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) {
    keep_count_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, CAND->colptr, keep, cnt, st);
    DIAF_COUNT_LAUNCH();
    e = exclusive_scan_i32(cnt, d_colptr, n, bs, s);
  }
  if (e == cudaSuccess) {
    select_kernel<<<ceil_div(n, kSelWarps), kSelWarps * 32, 0, s>>>(n, CAND->colptr, CAND->rowidx, d_score, keep,
                                                                     d_colptr, d_rowidx);
    DIAF_COUNT_LAUNCH();
    e = cudaGetLastError();
  }
  uint32_t h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(cnt, s);
  cudaFreeAsync(bs, s);
  cudaFreeAsync(st, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    diaf_set_last_error(cudaGetErrorString(e));
    return DIAF_ECUDA;
  }
  if (h & DEV_ST_CAPACITY) {
    diaf_set_last_error("a column has more than 128 candidates");
    return DIAF_EUNSUPPORTED;
  }
  return DIAF_OK;
}

diaf_status diaf_scaled_residuals(const diaf_factors* F, double* d_out, void* stream) {
  if (!F || (F->n > 0 && !d_out)) {
    diaf_set_last_error("NULL argument");
    return DIAF_EINVAL;
  }
  if (F->n == 0) return DIAF_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (F->dtype == DIAF_C128)
    scaled_residuals_kernel<Cx<double>><<<ceil_div(F->n, 256), 256, 0, s>>>(F->n, F->res, F->Vcp, F->Vri,
                                                                           (const Cx<double>*)F->Vv, d_out);
  else
    scaled_residuals_kernel<double><<<ceil_div(F->n, 256), 256, 0, s>>>(F->n, F->res, F->Vcp, F->Vri,
                                                                       (const double*)F->Vv, d_out);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError() == cudaSuccess ? DIAF_OK : DIAF_ECUDA;
}

diaf_status diaf_toggle_targets(const diaf_pattern* CAND, const uint8_t* d_in_base, const double* d_r0,
                                const double* d_rt, int32_t slot, double clip, double* d_value, void* stream) {
  if (!CAND || slot < 0 || !(clip > 0.0) || (CAND->n > 0 && (!d_in_base || !d_r0 || !d_rt || !d_value))) {
    diaf_set_last_error("NULL argument, negative slot or clip <= 0");
    return DIAF_EINVAL;
  }
  const int n = CAND->n;
  if (n == 0) return DIAF_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long* mbits = nullptr;
  if (cudaMallocAsync(&mbits, sizeof(unsigned long long), s) != cudaSuccess) return DIAF_ENOMEM;
  max_finite_sq_kernel<<<1, 1024, 0, s>>>(n, d_r0, mbits);
  DIAF_COUNT_LAUNCH();
  toggle_targets_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, CAND->colptr, CAND->rowidx, d_in_base, d_r0, d_rt, slot,
                                                         clip, mbits, d_value);
  DIAF_COUNT_LAUNCH();
  cudaFreeAsync(mbits, s);
  return cudaGetLastError() == cudaSuccess ? DIAF_OK : DIAF_ECUDA;
}

}  // extern "C"
