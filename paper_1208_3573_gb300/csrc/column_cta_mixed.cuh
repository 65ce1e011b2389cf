// Mixed-precision kernel for large tiles (size bucket 2: k_j <= 64,
// m_j <= 1024), real DIAF-S, one CTA per column -- the CTA-level form of the
// mixed warp kernel: the FP64 tile is gathered, its FP32 copy is factorised
// (Householder QR of T, FP32 leverage keys, QR of A-hat, one-sided Jacobi of
// R-hat), and the smallest right singular vector gets the second-order FP64
// correction in the FP32 singular basis (d = x^T H x / x^T x, r = H x - d x,
// x <- x - sum_{i != min} V_i (V_i^T r) / (s_i^2 - d), H = A-hat^T A-hat from
// the FP64 tile; twice when the gap is below 1e-2).  v_j = T(I_j,:) w_j and the
// residual are evaluated in FP64.
//
// A leverage decision within 2 delta of its threshold (delta = (m + k) eps_32
// kappa) makes the kernel recompute the column's keys in FP64 with the FP64
// CTA kernel's own QR and key computation and select with those.  A column
// goes back to the FP64 CTA kernel (flag FP64_FALLBACK) whenever the FP32
// result could differ from the FP64 one otherwise: column-scaled kappa(T) or
// kappa(A-hat) above 300, a singular gap below 1e-5, fewer rows outside I_j
// than k_j, or an empty W column.
#pragma once

#include "column_cta.cuh"

struct CtaMixedSmem {
  static constexpr int KP = kCtaKmax + 1;
  static constexpr size_t bytes(int mcap) {
    return sizeof(float) * (2 * KP * kCtaKmax + 3 * kCtaKmax) + sizeof(double) * (2 * kCtaKmax + 3 * mcap) +
           sizeof(double) * (2 * kCtaKmax + 2 * kCtaWarps) + sizeof(int32_t) * (5 * mcap + 2 * kCtaKmax + 8 + 2);
  }
};

// ---------------------------------------------------------------- tensor-core Gram path
// For a well-conditioned tile the two Householder QRs (of T for the keys, of
// A-hat for the SVD) are replaced by the Gram matrix on the tensor cores and
// Cholesky factorisations: G = T^T T by mma.m16n8k8 in TF32 with each FP32
// value split into a TF32 head and tail (head*head + head*tail + tail*head,
// FP32 accumulation: about FP32 accuracy); R_s = chol(D G D), D = diag(1 /
// ||T(:,c)||), so R = R_s D^-1 is T's R up to the signs of its rows; the keys
// h_r = ||T(r,:) R^-1||^2 = ||T(r,:) D R_s^-1||^2 by a second tensor-core
// product; the R of A-hat from G minus the I_j rows' outer products.  The
// error of a Gram-based factor grows with kappa^2 instead of kappa, so the
// path is taken only for column-scaled kappa <= kGramKappaMax (and the key
// decisions use the kappa^2 bound); other tiles keep the Householder QRs
// (kGramKappaMax).

__device__ __forceinline__ uint32_t tf32_head(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void mma_tf32_16x8x8(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// d += a b with a, b split into TF32 head and tail (the tail*tail term dropped)
__device__ __forceinline__ void mma_3xtf32(float (&d)[4], const float (&av)[4], const float (&bv)[2]) {
  uint32_t ah[4], at[4], bh[2], bt[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    ah[i] = tf32_head(av[i]);
    at[i] = tf32_head(av[i] - __uint_as_float(ah[i]));
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    bh[i] = tf32_head(bv[i]);
    bt[i] = tf32_head(bv[i] - __uint_as_float(bh[i]));
  }
  mma_tf32_16x8x8(d, at, bh);
  mma_tf32_16x8x8(d, ah, bt);
  mma_tf32_16x8x8(d, ah, bh);
}

// G (k x k, leading dimension ldg) = T^T T for the m x k FP32 tile T (leading
// dimension ld).  Output tiles of 16 x 8 over the CTA's warps; fragment
// layout of mma.m16n8k8: lane = 4 g + t holds A(g, t), A(g + 8, t),
// A(g, t + 4), A(g + 8, t + 4), B(t, g), B(t + 4, g) and D(g, 2t),
// D(g, 2t + 1), D(g + 8, 2t), D(g + 8, 2t + 1).
__device__ void cta_gram_tc(const float* T, int ld, int m, int k, float* G, int ldg) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int mt = (k + 15) / 16, nt = (k + 7) / 8;
  for (int tile = warp; tile < mt * nt; tile += kCtaWarps) {
    const int i0 = 16 * (tile / nt), j0 = 8 * (tile % nt);
    float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const int ca0 = i0 + g, ca1 = i0 + g + 8, cb = j0 + g;
    const float* pa0 = T + (size_t)(ca0 < k ? ca0 : 0) * ld;
    const float* pa1 = T + (size_t)(ca1 < k ? ca1 : 0) * ld;
    const float* pb = T + (size_t)(cb < k ? cb : 0) * ld;
    for (int r0 = 0; r0 < m; r0 += 8) {
      const int r = r0 + t, r4 = r0 + t + 4;
      const bool in = r < m, in4 = r4 < m;
      const float av[4] = {(in && ca0 < k) ? pa0[r] : 0.0f, (in && ca1 < k) ? pa1[r] : 0.0f,
                           (in4 && ca0 < k) ? pa0[r4] : 0.0f, (in4 && ca1 < k) ? pa1[r4] : 0.0f};
      const float bv[2] = {(in && cb < k) ? pb[r] : 0.0f, (in4 && cb < k) ? pb[r4] : 0.0f};
      mma_3xtf32(d, av, bv);
    }
    const int c0 = j0 + 2 * t;
    if (ca0 < k && c0 < k) G[ca0 + c0 * ldg] = d[0];
    if (ca0 < k && c0 + 1 < k) G[ca0 + (c0 + 1) * ldg] = d[1];
    if (ca1 < k && c0 < k) G[ca1 + c0 * ldg] = d[2];
    if (ca1 < k && c0 + 1 < k) G[ca1 + (c0 + 1) * ldg] = d[3];
  }
  __syncthreads();
}

// In place: the upper triangle of the k x k symmetric positive definite G
// (leading dimension ldg, scaled by D = diag(sc) on both sides first) becomes
// R_s with D G D = R_s^T R_s (right-looking, one column per step); the strict
// lower triangle is zeroed.  Returns false (uniformly) at a pivot <= 0.
__device__ bool cta_cholesky_scaled(float* G, int ldg, int k, const float* sc, float* redF) {
  const int tid = threadIdx.x;
  for (int i = tid; i < k * k; i += kCtaThreads) {
    const int p = i % k, q = i / k;
    G[p + q * ldg] = p <= q ? G[p + q * ldg] * sc[p] * sc[q] : 0.0f;
  }
  __syncthreads();
  for (int c = 0; c < k; ++c) {
    const float d = G[c + c * ldg];
    if (!(d > 0.0f)) return false;  // uniform: every thread read the same pivot
    const float rcc = sqrtf(d), rinv = 1.0f / rcc;
    __syncthreads();  // every thread has read the pivot
    for (int q = c + tid; q < k; q += kCtaThreads) G[c + q * ldg] = q == c ? rcc : G[c + q * ldg] * rinv;
    __syncthreads();
    const int w = k - c - 1;  // trailing block (c+1..k-1)^2, upper triangle
    for (int i = tid; i < w * w; i += kCtaThreads) {
      const int p = c + 1 + i % w, q = c + 1 + i / w;
      if (p <= q) G[p + q * ldg] -= G[c + p * ldg] * G[c + q * ldg];
    }
    __syncthreads();
  }
  (void)redF;
  return true;
}

// hk[r] = ||T(r,:) B||^2 for r < m, B (k x k, leading dimension ldb) in shared
// memory: tensor-core product of the tile with B (TF32 head/tail split),
// rows of 16 per warp task, squares summed from the accumulators.
__device__ void cta_row_norms_tc(const float* T, int ld, int m, int k, const float* B, int ldb, double* hk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int mt = (m + 15) / 16, nt = (k + 7) / 8, kt = (k + 7) / 8;
  for (int task = warp; task < mt; task += kCtaWarps) {
    const int r0 = 16 * task;
    const int ra = r0 + g, rb = r0 + g + 8;
    float h0 = 0.0f, h1 = 0.0f;
    for (int jn = 0; jn < nt; ++jn) {
      const int cb = 8 * jn + g;
      float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      for (int kk = 0; kk < kt; ++kk) {
        const int q = 8 * kk + t, q4 = 8 * kk + t + 4;
        const float av[4] = {(ra < m && q < k) ? T[ra + (size_t)q * ld] : 0.0f,
                             (rb < m && q < k) ? T[rb + (size_t)q * ld] : 0.0f,
                             (ra < m && q4 < k) ? T[ra + (size_t)q4 * ld] : 0.0f,
                             (rb < m && q4 < k) ? T[rb + (size_t)q4 * ld] : 0.0f};
        const float bv[2] = {(q < k && cb < k) ? B[q + cb * ldb] : 0.0f, (q4 < k && cb < k) ? B[q4 + cb * ldb] : 0.0f};
        mma_3xtf32(d, av, bv);
      }
      h0 += d[0] * d[0] + d[1] * d[1];
      h1 += d[2] * d[2] + d[3] * d[3];
    }
    h0 += __shfl_xor_sync(DIAF_FULL, h0, 1);
    h0 += __shfl_xor_sync(DIAF_FULL, h0, 2);
    h1 += __shfl_xor_sync(DIAF_FULL, h1, 1);
    h1 += __shfl_xor_sync(DIAF_FULL, h1, 2);
    if (t == 0) {
      if (ra < m) hk[ra] = (double)h0;
      if (rb < m) hk[rb] = (double)h1;
    }
  }
  __syncthreads();
}

// X (k x k, leading dimension ldx) = D R_s^-1 for the upper triangular R_s
// (leading dimension ldr): one column of the inverse per thread, back
// substitution, rows scaled by D = diag(sc).
__device__ void cta_upper_inverse_scaled(const float* Rsm, int ldr, int k, const float* sc, float* X, int ldx) {
  for (int jc = threadIdx.x; jc < k; jc += kCtaThreads) {
    for (int i = k - 1; i >= 0; --i) {
      float acc = i == jc ? 1.0f : 0.0f;
      if (i < jc)
        for (int p = i + 1; p <= jc; ++p) acc -= Rsm[i + p * ldr] * X[p + jc * ldx];
      X[i + jc * ldx] = i <= jc ? acc / Rsm[i + i * ldr] : 0.0f;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k * k; i += kCtaThreads) {
    const int p = i % k, q = i / k;
    X[p + q * ldx] *= sc[p];
  }
  __syncthreads();
}

// Greedy V rule of Sec. 3.1 on the keys hk (as select_rows_greedy, at CTA
// level): s picks among the admissible rows, ties within tau to the lower row.
// Returns the smallest distance of a non-leading candidate key from a
// threshold it was compared with (the FP32 decision margin).
__device__ inline double cta_select_rows(const int32_t* rs, const double* hk, int32_t* pick, int m, int rule, int j,
                                         int s, double tau, double* red, const int32_t* blk) {
  const int tid = threadIdx.x;
  double margin = DBL_MAX;
  for (int t = 0; t < s; ++t) {
    double hm = -DBL_MAX;
    for (int r = tid; r < m; r += kCtaThreads)
      if (!pick[r] && admissible_row(rule, rs[r], j, blk)) hm = dmax(hm, hk[r]);
    hm = block_max(hm, red);
    int rmax = INT_MAX;
    for (int r = tid; r < m; r += kCtaThreads)
      if (!pick[r] && admissible_row(rule, rs[r], j, blk) && hk[r] == hm) rmax = dmin(rmax, r);
    rmax = block_min(rmax, reinterpret_cast<int*>(red));
    const double thr = hm - tau;
    int best = INT_MAX;
    for (int r = tid; r < m; r += kCtaThreads)
      if (!pick[r] && admissible_row(rule, rs[r], j, blk)) {
        if (r != rmax) margin = dmin(margin, fabs(hk[r] - thr));
        if (hk[r] >= thr) best = dmin(best, r);
      }
    best = block_min(best, reinterpret_cast<int*>(red));
    if (best == INT_MAX) {  // no key reaches the threshold (non-finite keys): the lowest remaining admissible row
      for (int r = tid; r < m; r += kCtaThreads)
        if (!pick[r] && admissible_row(rule, rs[r], j, blk)) best = dmin(best, r);
      best = block_min(best, reinterpret_cast<int*>(red));
    }
    if (tid == 0 && best < m) pick[best] = 1;
    __syncthreads();
  }
  return block_min(margin, red);
}

// column norms of the m x k FP32 tile (warp per column)
__device__ inline void cta_col_norms_f(const float* T, int ld, int m, int k, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < k; c += kCtaWarps) {
    float s = 0.0f;
    for (int r = lane; r < m; r += 32) s += T[r + (size_t)c * ld] * T[r + (size_t)c * ld];
    s = warp_sum(s);
    if (lane == 0) out[c] = (double)sqrtf(s);
  }
  __syncthreads();
}

// g = H x = A-hat^T (A-hat x) in FP64 from the FP64 tile (rows of I_j
// excluded), z = A-hat x (m) as scratch.
__device__ inline void cta_hat_gram_apply(const double* Ts, int ld, int m, int k, const int32_t* inI, const double* x,
                                          double* z, double* g) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int r = tid; r < m; r += kCtaThreads) {
    double zr = 0.0;
    if (inI[r] < 0)
      for (int q = 0; q < k; ++q) zr += Ts[r + (size_t)q * ld] * x[q];
    z[r] = zr;
  }
  __syncthreads();
  for (int c = warp; c < k; c += kCtaWarps) {
    double gc = 0.0;
    for (int r = lane; r < m; r += 32) gc += Ts[r + (size_t)c * ld] * z[r];
    gc = warp_sum(gc);
    if (lane == 0) g[c] = gc;
  }
  __syncthreads();
}

// One second-order correction of x (FP64, k) with Rayleigh quotient d and
// g = H x in the FP32 singular basis V (columns i, leading dimension ldv,
// values sig): r = g - d x, x <- x - sum_i V_i (V_i^T r) / (sig_i^2 - d) over
// i other than e0 and e1 (projection in FP32; rf, cc: k floats of scratch).
// Returns this thread's largest |update|.
__device__ inline float cta_basis_correction(const float* V, int ldv, const double* sig, int k, uint64_t excl,
                                             double d, const double* g, double* x, float* rf, float* cc) {
  const int tid = threadIdx.x;
  for (int c = tid; c < k; c += kCtaThreads) rf[c] = (float)(g[c] - d * x[c]);
  __syncthreads();
  for (int i = tid; i < k; i += kCtaThreads) {
    float vr = 0.0f;
    for (int q = 0; q < k; ++q) vr += V[q + i * ldv] * rf[q];
    const float si = (float)sig[i];
    const float den = si * si - (float)d;
    cc[i] = ((excl >> i) & 1) ? 0.0f : -vr / den;
  }
  __syncthreads();
  float big = 0.0f;
  for (int c = tid; c < k; c += kCtaThreads) {
    float dx = 0.0f;
    for (int i = 0; i < k; ++i) dx += V[c + i * ldv] * cc[i];
    x[c] += (double)dx;
    big = fmaxf(big, fabsf(dx));
  }
  __syncthreads();
  return big;
}

constexpr int kClusterMax = 4;  // most singular values of a close cluster resolved in mixed precision

// Eigen-decomposition of the symmetric p x p matrix K (leading dimension
// kClusterMax, FP64) by cyclic Jacobi rotations, one thread: K becomes
// diagonal, Q (same layout) its eigenvectors, th the eigenvalues in
// ascending order (Q's columns sorted with them).
__device__ inline void small_sym_eig(double* K, double* Q, double* th, int p) {
  constexpr int P = kClusterMax;
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) Q[i + j * P] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int i = 0; i < p; ++i) {
      dia += K[i + i * P] * K[i + i * P];
      for (int j = i + 1; j < p; ++j) off += K[i + j * P] * K[i + j * P];
    }
    if (!(off > 1e-32 * dia)) break;
    for (int i = 0; i < p; ++i)
      for (int j = i + 1; j < p; ++j) {
        const double kij = K[i + j * P];
        if (kij == 0.0) continue;
        const double tau = (K[j + j * P] - K[i + i * P]) / (2.0 * kij);
        const double t = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
        for (int r = 0; r < p; ++r) {  // K <- K J (columns i, j)
          const double a = K[r + i * P], b = K[r + j * P];
          K[r + i * P] = cs * a - sn * b;
          K[r + j * P] = sn * a + cs * b;
        }
        for (int c = 0; c < p; ++c) {  // K <- J^T K (rows i, j)
          const double a = K[i + c * P], b = K[j + c * P];
          K[i + c * P] = cs * a - sn * b;
          K[j + c * P] = sn * a + cs * b;
        }
        for (int r = 0; r < p; ++r) {  // Q <- Q J
          const double a = Q[r + i * P], b = Q[r + j * P];
          Q[r + i * P] = cs * a - sn * b;
          Q[r + j * P] = sn * a + cs * b;
        }
      }
  }
  for (int i = 0; i < p; ++i) th[i] = K[i + i * P];
  for (int i = 0; i < p; ++i) {  // selection sort, ascending
    int lo = i;
    for (int j = i + 1; j < p; ++j)
      if (th[j] < th[lo]) lo = j;
    if (lo != i) {
      const double t = th[i];
      th[i] = th[lo];
      th[lo] = t;
      for (int r = 0; r < p; ++r) {
        const double q = Q[r + i * P];
        Q[r + i * P] = Q[r + lo * P];
        Q[r + lo * P] = q;
      }
    }
  }
}

// Rayleigh-Ritz step on the span of the p vectors X (k each, stride k) in
// FP64, with G = H X: X is orthonormalised by modified Gram-Schmidt (G
// follows linearly), the p x p matrix X^T H X diagonalised, and X, G become
// its Ritz vectors for the Ritz values th (ascending; K, Q, th: shared
// scratch of kClusterMax^2, kClusterMax^2 and kClusterMax doubles).
__device__ inline void cta_cluster_rayleigh_ritz(double* X, double* G, int p, int k, double* red, double* K,
                                                 double* Q, double* th) {
  constexpr int P = kClusterMax;
  const int tid = threadIdx.x;
  for (int a = 0; a < p; ++a) {
    double* xa = X + a * k;
    double* ga = G + a * k;
    for (int b = 0; b < a; ++b) {
      const double* xb = X + b * k;
      const double* gb = G + b * k;
      double part = 0.0;
      for (int c = tid; c < k; c += kCtaThreads) part += xb[c] * xa[c];
      const double coef = block_sum(part, red);
      for (int c = tid; c < k; c += kCtaThreads) {
        xa[c] -= coef * xb[c];
        ga[c] -= coef * gb[c];
      }
    }
    double part = 0.0;
    for (int c = tid; c < k; c += kCtaThreads) part += xa[c] * xa[c];
    const double inv = 1.0 / sqrt(block_sum(part, red));
    for (int c = tid; c < k; c += kCtaThreads) {
      xa[c] *= inv;
      ga[c] *= inv;
    }
  }
  for (int a = 0; a < p; ++a)
    for (int b = a; b < p; ++b) {
      double part = 0.0;
      for (int c = tid; c < k; c += kCtaThreads) part += 0.5 * (X[a * k + c] * G[b * k + c] + X[b * k + c] * G[a * k + c]);
      const double h = block_sum(part, red);
      if (tid == 0) K[a + b * P] = K[b + a * P] = h;
    }
  if (tid == 0) small_sym_eig(K, Q, th, p);
  __syncthreads();
  for (int c = tid; c < k; c += kCtaThreads) {
    double xs[P], gs[P];
#pragma unroll
    for (int a = 0; a < P; ++a) {
      xs[a] = a < p ? X[a * k + c] : 0.0;
      gs[a] = a < p ? G[a * k + c] : 0.0;
    }
#pragma unroll
    for (int a = 0; a < P; ++a)
      if (a < p) {
        double xn = 0.0, gn = 0.0;
#pragma unroll
        for (int b = 0; b < P; ++b)
          if (b < p) {
            xn += xs[b] * Q[b + a * P];
            gn += gs[b] * Q[b + a * P];
          }
        X[a * k + c] = xn;
        G[a * k + c] = gn;
      }
  }
  __syncthreads();
}

constexpr int kClusterMaxCorrections = 4;       // close cluster: corrections before the column goes to FP64
constexpr float kClusterCorrectionTol = 1e-10f;  // ... converged when no update exceeds this

#ifdef DIAF_PHASE_TIMING
#define CTA_FB(why)                                                         \
  do {                                                                      \
    if (threadIdx.x == 0 && a.phase) {                                      \
      atomicAdd(&a.phase[16 + (why)], 1ull);                                \
    }                                                                       \
  } while (0)
#else
#define CTA_FB(why) do {} while (0)
#endif
// Returns true when the column was finished here, false when it is handed back.
__device__ bool solve_column_cta_mixed(const ColArgs& a, const CtaScratch& sc, int j, unsigned char* smem) {
  using L = CtaMixedSmem;
  constexpr int KP = L::KP;
  const int tid = threadIdx.x;
  const int mcap = sc.ldm;
  float* Rs = reinterpret_cast<float*>(smem);  // R of T, then R-hat (KP x KMAX)
  float* Vj = Rs + KP * kCtaKmax;               // Jacobi V (Gram path: first D R_s^-1)
  float* rinv = Vj + KP * kCtaKmax;             // reciprocal diagonal (FP32)
  float* rf = rinv + kCtaKmax;                  // correction: r in FP32
  float* cc = rf + kCtaKmax;                    // correction coefficients
  double* wv = reinterpret_cast<double*>(cc + kCtaKmax);  // x, then w
  double* gg = wv + kCtaKmax;                   // H x
  double* vv = gg + kCtaKmax;                   // v (mcap)
  double* zz = vv + mcap;                       // A-hat x (mcap)
  double* hk = zz + mcap;                       // keys (mcap)
  double* sig = hk + mcap;                      // singular values (FP32 values)
  double* cn = sig + kCtaKmax;                  // column norms
  double* red = cn + kCtaKmax;                  // 2 x kCtaWarps
  int32_t* ibase = reinterpret_cast<int32_t*>(red + 2 * kCtaWarps);
  int32_t* rs = ibase;
  int32_t* inI = rs + mcap;
  int32_t* pick = inI + mcap;
  int32_t* Is = pick + mcap;
  int32_t* Iloc = Is + mcap;
  int32_t* cst = Iloc + mcap;
  int32_t* coff = cst + kCtaKmax;
  int32_t* misc = coff + kCtaKmax;  // [0] jpos, [1] count
  float* redF = reinterpret_cast<float*>(red);

  // the slab holds two tiles of the FP64 kernel's size: the FP64 tile, then
  // the FP32 one and (Gram path) G = T^T T (k x k, leading dimension kcap:
  // kcap^2 <= ldm kcap floats fit the tile's unused second half)
  double* Ts = reinterpret_cast<double*>(sc.slab) + (size_t)blockIdx.x * 2 * sc.ldm * sc.kcap;
  float* Tw = reinterpret_cast<float*>(Ts + (size_t)sc.ldm * sc.kcap);
  float* Gm = Tw + (size_t)sc.ldm * sc.kcap;
  const int ld = sc.ldm;

  const int k = a.Wcp[j + 1] - a.Wcp[j];
  const int m = a.m[j];
  const int l = a.l[j];
  const int me = m > k ? m : k;
  if (k == 0 || me > mcap) return false;  // the FP64 kernel has the conventions
  const int32_t* J = a.Wri + a.Wcp[j];
  const int32_t* Rj = a.rows + a.Eoff[j];
  const double* Av = reinterpret_cast<const double*>(a.Av);
  uint32_t flags = 0;

  DIAF_PHASE_START();
  // ---- gather (FP64) and the FP32 copy
  for (int r = tid; r < mcap; r += kCtaThreads) {
    rs[r] = r < m ? Rj[r] : INT_MAX;
    inI[r] = -1;
    pick[r] = 0;
  }
  for (size_t i = tid; i < (size_t)me * k; i += kCtaThreads) Ts[(i % me) + (i / me) * ld] = 0.0;
  cta_gather_offsets(a.Acp, J, k, cst, coff, misc + 1);
  __syncthreads();
  const int E = misc[1];
  for (int e = tid; e < E; e += kCtaThreads) {
    const int q = upper_bound_i32(coff, k, e) - 1;
    const int p = cst[q] + (e - coff[q]);
    const int r = lower_bound_i32(rs, m, a.Ari[p]);
    Ts[r + (size_t)q * ld] = Av[p];
  }
  __syncthreads();
  for (size_t i = tid; i < (size_t)me * k; i += kCtaThreads) {
    const size_t o = (i % me) + (i / me) * ld;
    Tw[o] = (float)Ts[o];
  }
  __syncthreads();
  cta_col_norms_f(Tw, ld, m, k, cn);

  DIAF_PHASE(0);
  // ---- tensor-core Gram path: G, R_s = chol(D G D), kappa, keys by a second product
  bool gram = false;      // the keys (and G) came from the Gram path
  bool tw_intact = true;  // Tw still holds the FP32 tile
  float kap = 0.0f;
  if (sc.gram && m >= k) {
    int zero = 0;
    for (int c = tid; c < k; c += kCtaThreads) {
      rf[c] = cn[c] > 0.0 ? (float)(1.0 / cn[c]) : 0.0f;
      zero |= !(cn[c] > 0.0);
    }
    if (!__syncthreads_or(zero)) {
      DIAF_PHASE(11);
      cta_gram_tc(Tw, ld, m, k, Gm, sc.kcap);
      DIAF_PHASE(12);
      for (int i = tid; i < k * k; i += kCtaThreads) Rs[(i % k) + (i / k) * KP] = Gm[(i % k) + (i / k) * sc.kcap];
      __syncthreads();
      if (cta_cholesky_scaled(Rs, KP, k, rf, redF)) {
        float kp = 0.0f;  // column-scaled kappa: ||T(:,c)|| / |R_cc| = 1 / |R_s,cc|
        for (int c = tid; c < k; c += kCtaThreads) kp = fmaxf(kp, 1.0f / fabsf(Rs[c + c * KP]));
        kap = block_max(kp, redF);
        gram = kap <= kGramKappaMax;
      }
      DIAF_PHASE(13);
    }
  }
  if (gram) {
#ifdef DIAF_PHASE_TIMING
    if (threadIdx.x == 0 && a.phase) atomicAdd(&a.phase[29], 1ull);
#endif
    if (a.rule != DIAF_RULE_FIXED) {
      cta_upper_inverse_scaled(Rs, KP, k, rf, Vj, KP);  // D R_s^-1 = R^-1
      DIAF_PHASE(14);
      cta_row_norms_tc(Tw, ld, m, k, Vj, KP, hk);       // h_r = ||T(r,:) R^-1||^2
      DIAF_PHASE(15);
    }
  } else {
    // ---- FP32 QR of T, kappa estimate, FP32 keys
    cta_householder_qr<float>(Tw, ld, me, k, redF, nullptr);
    for (int i = tid; i < k * k; i += kCtaThreads) {
      const int r = i % k, c = i / k;
      Rs[r + c * KP] = (r <= c) ? Tw[r + (size_t)c * ld] : 0.0f;
    }
    __syncthreads();
    float kp = 0.0f;
    for (int c = tid; c < k; c += kCtaThreads) {
      const float d = fabsf(Rs[c + c * KP]);
      kp = fmaxf(kp, d > 0.0f ? (float)cn[c] / d : INFINITY);
      rinv[c] = d > 0.0f ? 1.0f / Rs[c + c * KP] : 0.0f;
    }
    kap = block_max(kp, redF);
    if (!(kap <= kMixedKappaMax)) { CTA_FB(0); return false; }
    if (a.rule != DIAF_RULE_FIXED) {
      for (int r = tid; r < m; r += kCtaThreads) {  // Q = T R^-1 by rows (FP32), into Tw
        float h = 0.0f;
        for (int c = 0; c < k; ++c) {
          float acc = (float)Ts[r + (size_t)c * ld];
          for (int p2 = 0; p2 < c; ++p2) acc -= Tw[r + (size_t)p2 * ld] * Rs[p2 + c * KP];
          const float z = acc * rinv[c];
          Tw[r + (size_t)c * ld] = z;
          h += z * z;
        }
        hk[r] = (double)h;
      }
      __syncthreads();
    }
  }
  DIAF_PHASE(2);
  if (a.rule != DIAF_RULE_FIXED) {
    // (Is and Iloc, 2 mcap ints, are the sort's scratch until I_j is formed)
    const double margin = cta_select_rows_greedy(rs, hk, pick, m, a.rule, j, l - 1, a.tie_tol, a.blk, red, Is);
    // key error bound: the FP32 QR's backward error amplified by kappa, or
    // kappa^2 for keys from the Gram matrix
    const double delta = kMixedDeltaScale * (m + k) * (double)FLT_EPSILON * (double)kap * (gram ? (double)kap : 1.0);
    DIAF_PHASE(3);
    if (l > 1 && margin <= 2.0 * delta) {
      // the FP32 keys cannot decide this column: the FP64 CTA kernel's QR and
      // key computation on an FP64 copy of the tile (in the FP32 tile's slab
      // space, rewritten for A-hat below), then the selection with those keys,
      // so I_j is the FP64 kernel's choice
      double* Tq = reinterpret_cast<double*>(Tw);
      double* Rq = reinterpret_cast<double*>(Rs);  // KP x KMAX doubles over Rs and Vj (both free here)
      tw_intact = false;
#ifdef DIAF_PHASE_TIMING
      if (threadIdx.x == 0 && a.phase) atomicAdd(&a.phase[gram ? 31 : 28], 1ull);
#endif
      double* rq = wv;                              // reciprocal diagonal
      for (size_t i = tid; i < (size_t)me * k; i += kCtaThreads) Tq[(i % me) + (i / me) * ld] = Ts[(i % me) + (i / me) * ld];
      __syncthreads();
      cta_householder_qr<double>(Tq, ld, me, k, red, nullptr);
      for (int i = tid; i < k * k; i += kCtaThreads) {
        const int r = i % k, c = i / k;
        Rq[r + c * KP] = (r <= c) ? Tq[r + (size_t)c * ld] : 0.0;
      }
      __syncthreads();
      double part = 0.0;
      for (int c = tid; c < k; c += kCtaThreads) part = dmax(part, fabs(Rq[c + c * KP]));
      const double piv = 1e-14 * block_max(part, red);
      for (int c = tid; c < k; c += kCtaThreads) rq[c] = sc_recip_or_zero(Rq[c + c * KP], piv);
      for (int r = tid; r < mcap; r += kCtaThreads) pick[r] = 0;
      __syncthreads();
      for (int r = tid; r < m; r += kCtaThreads) {  // Q = T R^-1 by rows, into Tq
        double h = 0.0;
        for (int c = 0; c < k; ++c) {
          double acc = Ts[r + (size_t)c * ld];
          for (int p2 = 0; p2 < c; ++p2) acc -= Tq[r + (size_t)p2 * ld] * Rq[p2 + c * KP];
          const double z = acc * rq[c];
          Tq[r + (size_t)c * ld] = z;
          h += z * z;
        }
        hk[r] = h;
      }
      __syncthreads();
      cta_select_rows_greedy(rs, hk, pick, m, a.rule, j, l - 1, a.tie_tol, a.blk, red, Is);
      DIAF_PHASE(10);
    }
  }
  DIAF_PHASE(3);
  // I_j
  if (a.rule == DIAF_RULE_FIXED) {
    if (tid == 0) {
      misc[0] = -1;
      const int32_t* Vf = a.Vfri + a.Vfcp[j];
      for (int t = 0; t < l; ++t) {
        const int row = Vf[t];
        const int r = lower_bound_i32(rs, m, row);
        const int loc = (r < m && rs[r] == row) ? r : -1;
        Is[t] = row;
        Iloc[t] = loc;
        if (loc >= 0) inI[loc] = t;
        if (row == j) misc[0] = t;
      }
    }
  } else {
    cta_form_I_greedy(rs, pick, m, j, a.jin[j] != 0, Is, Iloc, inI, misc);
  }
  __syncthreads();
  const int jpos = misc[0];
  int inrows = 0;
  for (int t = 0; t < l; ++t) inrows += (Iloc[t] >= 0);
  if (m - inrows < k) { CTA_FB(1); return false; }  // A-hat has fewer rows than columns

  DIAF_PHASE(4);
  // ---- R-hat: from G on the Gram path (G minus the I_j rows' outer
  // products, Cholesky of its column-scaled form), else FP32 QR of A-hat
  bool gram_hat = false;
  if (gram && tw_intact) {
    int zc = 0;  // an exactly zero column of A-hat (all its entries in I_j rows) keeps the QR path
    for (int c = tid; c < k; c += kCtaThreads) {
      bool nz = false;
      for (int r = 0; r < m && !nz; ++r) nz = inI[r] < 0 && Tw[r + (size_t)c * ld] != 0.0f;
      zc |= !nz;
    }
    if (!__syncthreads_or(zc)) {
      for (int i = tid; i < k * k; i += kCtaThreads) {
        const int p = i % k, q = i / k;
        float gpq = Gm[p + q * sc.kcap];
        for (int t = 0; t < l; ++t) {
          const int r = Iloc[t];
          if (r >= 0) gpq -= Tw[r + (size_t)p * ld] * Tw[r + (size_t)q * ld];
        }
        Rs[p + q * KP] = gpq;
      }
      __syncthreads();
      for (int c = tid; c < k; c += kCtaThreads) {
        const float gc = Rs[c + c * KP];
        cn[c] = gc > 0.0f ? (double)sqrtf(gc) : 0.0;  // column norms of A-hat
        rf[c] = gc > 0.0f ? 1.0f / sqrtf(gc) : 0.0f;
      }
      __syncthreads();
      if (cta_cholesky_scaled(Rs, KP, k, rf, redF)) {
        float kp = 0.0f;
        for (int c = tid; c < k; c += kCtaThreads) kp = fmaxf(kp, 1.0f / fabsf(Rs[c + c * KP]));
        if (block_max(kp, redF) <= kGramKappaMax) {
          gram_hat = true;
#ifdef DIAF_PHASE_TIMING
          if (threadIdx.x == 0 && a.phase) atomicAdd(&a.phase[30], 1ull);
#endif
          for (int i = tid; i < k * k; i += kCtaThreads) Rs[(i % k) + (i / k) * KP] *= (float)cn[i / k];
          __syncthreads();
        }
      }
    }
  }
  if (!gram_hat) {
    // ---- FP32 QR of A-hat
    for (size_t i = tid; i < (size_t)me * k; i += kCtaThreads) {
      const int r = i % me, c = i / me;
      Tw[r + (size_t)c * ld] = (r < m && inI[r] >= 0) ? 0.0f : (float)Ts[r + (size_t)c * ld];
    }
    __syncthreads();
    cta_col_norms_f(Tw, ld, m, k, cn);
    cta_householder_qr<float>(Tw, ld, me, k, redF, nullptr);
    float kh = 0.0f;
    for (int c = tid; c < k; c += kCtaThreads) {  // exact zero columns of A-hat: exact zero singular values
      const float d = fabsf(Tw[c + (size_t)c * ld]);
      kh = fmaxf(kh, d > 0.0f ? (float)cn[c] / d : (cn[c] > 0.0 ? INFINITY : 0.0f));
    }
    if (!(block_max(kh, redF) <= kMixedKappaMax)) { CTA_FB(2); return false; }
    for (int i = tid; i < k * k; i += kCtaThreads) {
      const int r = i % k, c = i / k;
      Rs[r + c * KP] = (r <= c) ? Tw[r + (size_t)c * ld] : 0.0f;
    }
    __syncthreads();
  }
  DIAF_PHASE(6);
  if (cta_jacobi<float, KP, KP, true>(Rs, k, k, Vj, redF) < 0) flags |= DIAF_FLAG_JACOBI_NOCONV;
  DIAF_PHASE(7);
  for (int c = tid; c < k; c += kCtaThreads) {
    float s2 = 0.0f;
    for (int i = 0; i < k; ++i) s2 += Rs[i + c * KP] * Rs[i + c * KP];
    sig[c] = (double)sqrtf(s2);
  }
  __syncthreads();
  int imin = 0;
  double smin = sig[0], smax = sig[0];
  for (int c = 1; c < k; ++c) {
    if (sig[c] < smin) { smin = sig[c]; imin = c; }
    smax = dmax(smax, sig[c]);
  }
  double snext = INFINITY, gap = INFINITY;
  for (int c = 0; c < k; ++c)
    if (c != imin) {
      snext = dmin(snext, sig[c]);
      gap = dmin(gap, sig[c] * sig[c] - smin * smin);
    }
  if (k > 1 && (snext - smin) <= 1e-6 * smax) flags |= DIAF_FLAG_DEGENERATE;
  // A close cluster: sigma_min^2 and the next singular values, each within
  // 1e-5 smax^2 of the one before, up to kClusterMax of them (the rest at
  // least that far beyond).  Their FP32 vectors can be mixed (and even
  // ordered wrongly) at FP32 accuracy, so all of them are corrected against
  // the other singular vectors and the cluster is resolved by a
  // Rayleigh-Ritz step in FP64.  A longer chain goes to the FP64 kernel.
  int32_t* cl = cst;  // the cluster's singular indices (the gather's offsets are dead)
  uint64_t excl = 1ull << imin;
  int p = 1;
  if (k > 1 && gap <= 1e-5 * smax * smax) {
    double last = smin;
    for (;;) {
      int nx = -1;
      for (int c = 0; c < k; ++c)
        if (!((excl >> c) & 1) && (nx < 0 || sig[c] < sig[nx])) nx = c;
      if (nx < 0 || sig[nx] * sig[nx] - last * last > 1e-5 * smax * smax) break;
      if (p == kClusterMax) { CTA_FB(3); return false; }
      if (tid == 0) cl[p] = nx;
      excl |= 1ull << nx;
      last = sig[nx];
      ++p;
    }
    if (tid == 0) cl[0] = imin;
  }

  // ---- FP64 correction in the FP32 singular basis
  if (p == 1) {
    const int iters = (k > 1 && gap < 1e-2 * smax * smax) ? 2 : 1;
    for (int c = tid; c < k; c += kCtaThreads) wv[c] = (double)Vj[c + imin * KP];
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
      cta_hat_gram_apply(Ts, ld, m, k, inI, wv, zz, gg);
      double xg = 0.0, xx = 0.0;
      for (int c = tid; c < k; c += kCtaThreads) {
        xg += wv[c] * gg[c];
        xx += wv[c] * wv[c];
      }
      xg = block_sum(xg, red);
      xx = block_sum(xx, red);
      const double d = xg / xx;
      cta_basis_correction(Vj, KP, sig, k, excl, d, gg, wv, rf, cc);
    }
  } else {
    // the cluster's vectors X and G = H X (p x k each) in the slab's
    // working tile, dead here (2 kClusterMax k doubles <= ldm kcap floats);
    // the p x p Rayleigh-Ritz matrices over the column norms, dead here
    __syncthreads();  // cl
    double* Xc = reinterpret_cast<double*>(Tw);
    double* Gc = Xc + (size_t)kClusterMax * k;
    double* Km = cn;
    double* Qm = Km + kClusterMax * kClusterMax;
    double* th = Qm + kClusterMax * kClusterMax;
    for (int i = tid; i < p * k; i += kCtaThreads) Xc[i] = (double)Vj[(i % k) + cl[i / k] * KP];
    __syncthreads();
    bool conv = false;
    for (int it = 0;; ++it) {
      for (int c = 0; c < p; ++c) cta_hat_gram_apply(Ts, ld, m, k, inI, Xc + c * k, zz, Gc + c * k);
      cta_cluster_rayleigh_ritz(Xc, Gc, p, k, red, Km, Qm, th);
      if (conv) break;
      if (it == kClusterMaxCorrections) { CTA_FB(3); return false; }
      float big = 0.0f;
      for (int c = 0; c < p; ++c)
        big = fmaxf(big, cta_basis_correction(Vj, KP, sig, k, excl, th[c], Gc + c * k, Xc + c * k, rf, cc));
      conv = block_max(big, redF) <= kClusterCorrectionTol;
    }
    for (int c = tid; c < k; c += kCtaThreads) wv[c] = Xc[c];  // the smallest Ritz vector
    // the DEGENERATE decision on the FP64 Ritz values
    flags &= ~DIAF_FLAG_DEGENERATE;
    if (sqrt(dmax(th[1], 0.0)) - sqrt(dmax(th[0], 0.0)) <= 1e-6 * smax) flags |= DIAF_FLAG_DEGENERATE;
    __syncthreads();
  }
  double xn = 0.0;
  for (int c = tid; c < k; c += kCtaThreads) xn += wv[c] * wv[c];
  xn = block_sum(xn, red);
  const double inv = 1.0 / sqrt(xn);
  for (int c = tid; c < k; c += kCtaThreads) wv[c] *= inv;
  __syncthreads();
  DIAF_PHASE(8);
  // v = T(I_j,:) w in FP64
  for (int t = tid; t < l; t += kCtaThreads) {
    double s2 = 0.0;
    const int r = Iloc[t];
    if (r >= 0)
      for (int q = 0; q < k; ++q) s2 += Ts[r + (size_t)q * ld] * wv[q];
    vv[t] = s2;
  }
  __syncthreads();
  cta_finish<double>(a, j, k, m, l, jpos, Ts, ld, wv, vv, Is, Iloc, inI, flags, true, red, 1e-14 * smax);
  DIAF_PHASE(9);
  return true;
}

__global__ void __launch_bounds__(kCtaThreads, 3) column_cta_mixed_kernel(ColArgs a, CtaScratch sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int idx_s;
  const int count = *a.list_count;
  while (true) {
    if (threadIdx.x == 0) idx_s = atomicAdd(a.work_counter, 1);
    __syncthreads();
    const int idx = idx_s;
    __syncthreads();
    if (idx >= count) break;
    const int j = list_at(a, count, idx);
    if (!solve_column_cta_mixed(a, sc, j, smem_raw)) {
      if (threadIdx.x == 0) a.fb_list[atomicAdd(a.fb_count, 1)] = j;
    }
    __syncthreads();
  }
}
