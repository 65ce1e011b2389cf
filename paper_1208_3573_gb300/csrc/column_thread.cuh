// Four lanes per column: the mixed-precision DIAF-S (Sec. 2.2) for small real
// tiles (k_j <= 16, m_j <= 32, the size bucket of stencil operators).
//
// A quad of lanes runs the whole column -- gather, FP32 Householder QR of T,
// leverage keys, the V rule of Sec. 3.1, FP32 Householder QR of A-hat (T with
// the I_j rows removed), cyclic one-sided Jacobi SVD of its R, the FP64
// second-order correction of the smallest right singular vector in the FP32
// singular basis, v = T(I_j,:) w, phase, FP64 residual and scatter -- with the
// same arithmetic as the warp kernel of column_mixed.cuh (the same FP32
// factorisations, key-error bound, hand-back tests and FP64 correction).  A
// warp works on eight columns at once: lane s of a quad owns the rows
// r = s (mod 4) of every column-major array of its column, so the per-column
// dependency chains carry two-step quad reductions instead of warp-wide ones,
// and no lane idles on the short vectors of these tiles.
//
// Storage: the FP32 working matrix, keys and Jacobi norms in shared memory,
// element e of quad c at smem[32 (e / 4) + 8 (e mod 4) + c] (the 32 lanes of
// a warp reading four consecutive elements each hit 32 distinct banks); the
// FP64 tile in a global slab laid out the same way across all quads of the
// grid (coalesced); the k-vectors of the FP64 correction in registers.
//
// A column this kernel does not finish itself -- an empty or fixed-pattern
// column, a tile beyond its capacity or with fewer rows than columns, a tile
// too ill-conditioned for the FP32 factors, FP32 keys that cannot decide I_j,
// a singular gap too small for the correction -- goes to the defer list, which
// the warp kernel of column_mixed.cuh then runs (with its own FP64 keys and
// FP64 hand-back).
#pragma once

#include "column.cuh"

struct ThreadArgs {
  int M, K;              // capacity of this launch (rows, columns)
  int arena;             // shared-memory floats per column
  double* slab;          // FP64 per quad of the grid: the tile T (M * K) and z (M), thread_slab_doubles
  int nquads;            // quads of the grid (the slab's interleave)
  int32_t* defer_list;   // columns left to the warp kernel
  int32_t* defer_count;
};

constexpr int kThreadKMax = 16, kThreadMMax = 32;
constexpr int kQuad = 4;            // lanes per column
constexpr int kQuadCols = 8;        // columns per warp
constexpr int kQuadWarps = 1;       // warps per block

// Shared-memory floats per column for capacity (M, K): the working matrix
// max(M K, 2 K^2), keys (M), Jacobi norms (K); rounded up to whole rows of 4.
__host__ __device__ constexpr int thread_arena_floats(int M, int K) {
  return ((M * K > 2 * K * K ? M * K : 2 * K * K) + M + K + 3) / 4 * 4;
}
// FP64 shared-memory scratch per column: the refined vector x (K), rounded
// up to whole rows of 4.
__host__ __device__ constexpr int thread_arena_doubles(int M, int K) { return (void)M, (K + 3) / 4 * 4; }
// FP64 slab doubles per quad: the tile T (M K) and z = A-hat x (M), each
// rounded up to whole rows of 4.
__host__ __device__ constexpr int thread_slab_doubles(int M, int K) { return (M * K + 3) / 4 * 4 + (M + 3) / 4 * 4; }
// Shared-memory bytes of one warp (eight columns).
__host__ __device__ constexpr size_t thread_warp_smem(int M, int K) {
  return sizeof(float) * (size_t)thread_arena_floats(M, K) * 8 + sizeof(double) * (size_t)thread_arena_doubles(M, K) * 8;
}

// Element e of this quad's interleaved shared-memory array (base already
// offset by the quad's slot); element e + 4u lies at qptr(base, e)[32 u].
__device__ __forceinline__ float* qptr(float* base, int e) { return base + ((e >> 2) * 32 + (e & 3) * 8); }
__device__ __forceinline__ double* qptr(double* base, int e) { return base + ((e >> 2) * 32 + (e & 3) * 8); }
#define QS(base, e) (*qptr((base), (e)))

__device__ __forceinline__ float qsum(float v, unsigned qm) {
  v += __shfl_xor_sync(qm, v, 1);
  v += __shfl_xor_sync(qm, v, 2);
  return v;
}
__device__ __forceinline__ double qsum(double v, unsigned qm) {
  v += __shfl_xor_sync(qm, v, 1);
  v += __shfl_xor_sync(qm, v, 2);
  return v;
}

// Round-robin Jacobi schedule of the warp kernels for qq = 2, 4, ..., 16
// columns (k rounded up to even): kPairTab[qq/2 - 1][round][pair] = (a << 4) | b,
// with b >= k marking a bye; filled once on the host.
constexpr int kPairRounds = kThreadKMax - 1, kPairSlots = kThreadKMax / 2;
static __constant__ uint8_t kPairTab[kThreadKMax / 2][kPairRounds][kPairSlots];

constexpr int kQR = kThreadMMax / 4;  // most rows a lane owns in a column of the tile
#ifndef DIAF_QUAD_JACOBI_PAIRS
#define DIAF_QUAD_JACOBI_PAIRS 4
#endif
constexpr int kJP = DIAF_QUAD_JACOBI_PAIRS;  // disjoint pairs of a round rotated together
constexpr int kQK = kThreadKMax / 4;  // most rows a lane owns in a column of a k x k matrix

// Householder QR in place of the m x k column-major matrix at W (ld m,
// m >= k), FP32: reflector c maps W(c:m, c) to beta e_1 (the reflectors of
// warp_householder_qr).  Lane `sub` works on its rows (held in registers for
// the reflector's column); R ends in the upper triangle, visible to the whole
// quad on return.
__device__ __forceinline__ void quad_qr(float* W, int m, int k, int sub, unsigned qm) {
  for (int c = 0; c < k; ++c) {
    const int c0 = c * m;
    const int r0 = c + ((sub - c) & 3);  // first own row >= c
    float* pc = qptr(W, c0 + r0);
    float u[kQR];
    float s = 0.0f;
#pragma unroll
    for (int t = 0; t < kQR; ++t) {
      u[t] = r0 + 4 * t < m ? pc[32 * t] : 0.0f;
      s = fmaf(u[t], u[t], s);
    }
    s = qsum(s, qm);
    __syncwarp(qm);  // W(c, c), last written by its owner, is read by the whole quad
    const float alpha = QS(W, c0 + c);
    if (s == 0.0f) continue;
    const float ax = fabsf(alpha);
    const float nrm = sqrtf(s);
    const float ph = alpha < 0.0f ? -1.0f : 1.0f;
    const float two_uu = __fdividef(1.0f, nrm * (nrm + ax));
    if (r0 == c) u[0] = (ax + nrm) * ph;  // u_0 (the owner of row c)
    for (int q = c + 1; q < k; ++q) {
      float* pq = qptr(W, q * m + r0);
      float x[kQR];
      float f = 0.0f;
#pragma unroll
      for (int t = 0; t < kQR; ++t) {
        x[t] = r0 + 4 * t < m ? pq[32 * t] : 0.0f;
        f = fmaf(u[t], x[t], f);
      }
      f = qsum(f, qm) * two_uu;
#pragma unroll
      for (int t = 0; t < kQR; ++t)
        if (r0 + 4 * t < m) pq[32 * t] = fmaf(-f, u[t], x[t]);
    }
    if (r0 == c) pc[0] = -nrm * ph;  // beta
  }
  __syncwarp(qm);
}

template <int KMAX>
__device__ void solve_column_quad(const ColArgs& a, const ThreadArgs& ta, int j, float* S, double* D, double* G,
                                  int sub, unsigned qm) {
  static_assert(KMAX <= kThreadKMax, "tile capacity");
  const int k = a.Wcp[j + 1] - a.Wcp[j];
  const int m = a.m[j];
  const int l = a.l[j];
  auto defer = [&]() {
    if (sub == 0) {
      const int pos = atomicAdd(ta.defer_count, 1);
      ta.defer_list[pos] = j;
    }
  };
  if (k == 0 || k > ta.K || k > KMAX || m > ta.M || m > kThreadMMax || m < k || l > m + 1 ||
      a.rule == DIAF_RULE_FIXED) {
    defer();
    return;
  }
  const int M = ta.M, K = ta.K;
  const int wsz = M * K > 2 * K * K ? M * K : 2 * K * K;
  float* W = S;  // working matrix at element 0, keys at wsz, Jacobi norms at wsz + M
  const int HK = wsz, NR = wsz + M;
  // FP64 tile (ld m): element e of this quad at G[(e / 4) 4 nquads + (e mod 4)],
  // element e + 4u at gptr(e)[u gstride]
  const size_t gstride = (size_t)4 * ta.nquads;
  auto gptr = [&](int e) { return G + (size_t)(e >> 2) * gstride + (e & 3); };
  auto T = [&](int e) -> double& { return *gptr(e); };
  const int nown = (m - sub + 3) >> 2;  // own tile rows: sub, sub + 4, ...
  DIAF_PHASE_START();

  // ---- gather T = A(R_j, J_j): own rows zeroed, then each lane places every
  // fourth entry of the J_j columns by a binary search in R_j (a copy of R_j
  // in the keys' shared-memory slots, which are free until the keys)
  const int32_t* Rj = a.rows + a.Eoff[j];
  const int32_t* J = a.Wri + a.Wcp[j];
  const double* Av = reinterpret_cast<const double*>(a.Av);
  auto RS = [&](int r) -> int32_t& { return *reinterpret_cast<int32_t*>(qptr(W, HK + r)); };
  for (int r = sub; r < m; r += 4) RS(r) = Rj[r];
  // the entry range of A(:, J_j[q]) as an int pair in FP64 scratch slot q
  // (free until the correction)
  auto CR = [&](int q) -> int2& { return *reinterpret_cast<int2*>(qptr(D, q)); };
  for (int q = sub; q < k; q += 4) {
    const int c = J[q];
    CR(q) = make_int2(a.Acp[c], a.Acp[c + 1]);
  }
  for (int q = 0; q < k; ++q) {
    double* gq = gptr(q * m + sub);
    float* wq = qptr(W, q * m + sub);
#pragma unroll
    for (int t = 0; t < kQR; ++t)
      if (t < nown) {
        gq[t * gstride] = 0.0;
        wq[32 * t] = 0.0f;
      }
  }
  __syncwarp(qm);
  for (int q = 0; q < k; ++q) {
    const int2 be = CR(q);
    for (int p = be.x + sub; p < be.y; p += 4) {
      const int32_t row = a.Ari[p];
      int r = 0;  // first position of R_j holding a row >= row (row is in R_j)
      for (int len = m; len > 0;) {
        const int half = len >> 1;
        if (RS(r + half) < row) {
          r += half + 1;
          len -= half + 1;
        } else {
          len = half;
        }
      }
      const double v = Av[p];
      T(r + q * m) = v;
      QS(W, r + q * m) = (float)v;
    }
  }
  __syncwarp(qm);
  float cn[KMAX];
#pragma unroll
  for (int q = 0; q < KMAX; ++q) {
    float s2 = 0.0f;
    if (q < k) {
      const float* wq = qptr(W, q * m + sub);
#pragma unroll
      for (int t = 0; t < kQR; ++t)
        if (t < nown) s2 = fmaf(wq[32 * t], wq[32 * t], s2);
    }
    cn[q] = 0.0f;
    if (q < k) cn[q] = sqrtf(qsum(s2, qm));  // k is the same in the whole quad
  }

  // ---- FP32 QR of T and the conditioning estimate
  DIAF_PHASE(0);
  quad_qr(W, m, k, sub, qm);
  float kap = 0.0f;
  float rinv[KMAX];
#pragma unroll
  for (int q = 0; q < KMAX; ++q) {
    rinv[q] = 0.0f;
    if (q < k) {
      const float d = QS(W, q + q * m);
      kap = fmaxf(kap, fabsf(d) > 0.0f ? cn[q] / fabsf(d) : INFINITY);
      rinv[q] = __fdividef(1.0f, d);
    }
  }
  if (!(kap <= kMixedKappaMax)) { defer(); return; }

  // ---- leverage keys h_r = ||Q(r,:)||^2, Q = T R^-1 by rows (own rows; R's
  DIAF_PHASE(2);
  // column c read through four pointers, element c m + 4u + v at P[v][32 u])
  // two rows at a time: the loads of R are shared and the two solves are
  // independent chains
  for (int t = 0; t < nown; t += 2) {
    const int r = sub + 4 * t;
    const bool two = t + 1 < nown;
    float z[KMAX], y[KMAX];
    float h = 0.0f, h1 = 0.0f;
#pragma unroll
    for (int c = 0; c < KMAX; ++c) {
      z[c] = 0.0f;
      y[c] = 0.0f;
      if (c < k) {
        const float* P0 = qptr(W, c * m);
        const float* P1 = qptr(W, c * m + 1);
        const float* P2 = qptr(W, c * m + 2);
        const float* P3 = qptr(W, c * m + 3);
        float acc = (float)T(r + c * m);
        float acc1 = two ? (float)T(r + 4 + c * m) : 0.0f;
#pragma unroll
        for (int p2 = 0; p2 < c; ++p2) {
          const float* P = (p2 & 3) == 0 ? P0 : ((p2 & 3) == 1 ? P1 : ((p2 & 3) == 2 ? P2 : P3));
          const float rv = P[32 * (p2 >> 2)];
          acc = fmaf(-z[p2], rv, acc);
          acc1 = fmaf(-y[p2], rv, acc1);
        }
        z[c] = acc * rinv[c];
        y[c] = acc1 * rinv[c];
        h = fmaf(z[c], z[c], h);
        h1 = fmaf(y[c], y[c], h1);
      }
    }
    QS(W, HK + r) = h;
    if (two) QS(W, HK + r + 4) = h1;
  }
  __syncwarp(qm);

  // ---- I_j: the diagonal plus the l - 1 admissible rows of largest key
  DIAF_PHASE(3);
  // (ties within tau to the lower row), as select_rows_greedy; every lane of
  // the quad takes the same decisions (picks as bits)
  uint32_t adm = 0;
  for (int r = 0; r < m; ++r)
    if (admissible_row(a.rule, Rj[r], j, a.blk)) adm |= 1u << r;
  uint32_t picked = 0;
  float margin = FLT_MAX;
  const float tau = (float)a.tie_tol;
  for (int t = 0; t < l - 1; ++t) {
    const uint32_t cand = adm & ~picked;
    float hm = -FLT_MAX;
    for (uint32_t b = cand; b; b &= b - 1) hm = fmaxf(hm, QS(W, HK + __ffs(b) - 1));
    int rmax = INT_MAX;
    for (uint32_t b = cand; b && rmax == INT_MAX; b &= b - 1)
      if (QS(W, HK + __ffs(b) - 1) == hm) rmax = __ffs(b) - 1;
    const float thr = hm - tau;
    int best = INT_MAX;
    for (uint32_t b = cand; b; b &= b - 1) {
      const int r = __ffs(b) - 1;
      const float h = QS(W, HK + r);
      if (r != rmax) margin = fminf(margin, fabsf(h - thr));
      if (h >= thr && best == INT_MAX) best = r;
    }
    if (best == INT_MAX && cand) best = __ffs(cand) - 1;  // no key reaches the threshold (non-finite keys)
    if (best < m) picked |= 1u << best;
  }
  if (l > 1) {
    const double delta = kMixedDeltaScale * (m + k) * (double)FLT_EPSILON * (double)kap;
    if ((double)margin <= 2.0 * delta) { defer(); return; }  // FP32 keys cannot decide this column
  }
  // I_j = the picked tile rows, row j, and j itself when it is not a tile row
  // (inserted in order); tile row r in I_j has position pos_of(r)
  uint32_t inI = picked;
  int rj = -1;
  for (int r = 0; r < m; ++r)
    if (Rj[r] == j) rj = r;
  if (rj >= 0) inI |= 1u << rj;
  const bool jin = a.jin[j] != 0;
  int jbefore = m;  // tile rows from this index on come after an inserted j
  if (!jin) {
    jbefore = 0;
    while (jbefore < m && Rj[jbefore] < j) ++jbefore;
  }
  auto below = [](int r) { return r >= 32 ? 0xffffffffu : (1u << r) - 1u; };  // bits of the rows below r
  auto pos_of = [&](int r) { return __popc(inI & below(r)) + ((!jin && r >= jbefore) ? 1 : 0); };
  if (__popc(inI) + (jin ? 0 : 1) != l || (jin && rj < 0)) { defer(); return; }  // not reached
  const int v0 = a.Vcp[j];
  const int jpos = jin ? pos_of(rj) : __popc(inI & below(jbefore));
  if (sub == 0 && !jin) a.Vri[v0 + jpos] = j;
  for (int r = sub; r < m; r += 4)
    if ((inI >> r) & 1u) a.Vri[v0 + pos_of(r)] = Rj[r];

  // ---- FP32 QR of A-hat (the I_j rows zeroed), its conditioning
  DIAF_PHASE(4);
  float ch[KMAX];
  // own rows of every column first (independent loads), the column norms
  // from shared memory after
  for (int q = 0; q < k; ++q) {
    const double* gq = gptr(q * m + sub);
    float* wq = qptr(W, q * m + sub);
    float f[kQR];
#pragma unroll
    for (int t = 0; t < kQR; ++t) f[t] = (t < nown && !((inI >> (sub + 4 * t)) & 1u)) ? (float)gq[t * gstride] : 0.0f;
#pragma unroll
    for (int t = 0; t < kQR; ++t)
      if (t < nown) wq[32 * t] = f[t];
  }
#pragma unroll
  for (int q = 0; q < KMAX; ++q) {
    float s2 = 0.0f;
    if (q < k) {
      const float* wq = qptr(W, q * m + sub);
#pragma unroll
      for (int t = 0; t < kQR; ++t)
        if (t < nown) s2 = fmaf(wq[32 * t], wq[32 * t], s2);
    }
    ch[q] = 0.0f;
    if (q < k) ch[q] = sqrtf(qsum(s2, qm));
  }
  __syncwarp(qm);
  quad_qr(W, m, k, sub, qm);
  float kh = 0.0f;
  bool zdiag = false;  // R-hat singular (A-hat rank deficient): V is accumulated in the sweeps instead
#pragma unroll
  for (int q = 0; q < KMAX; ++q)
    if (q < k) {
      const float d = fabsf(QS(W, q + q * m));
      kh = fmaxf(kh, d > 0.0f ? ch[q] / d : (ch[q] > 0.0f ? INFINITY : 0.0f));
      zdiag |= d == 0.0f;
    }
  if (!(kh <= kMixedKappaMax)) { defer(); return; }

  // ---- R-hat to ld k at W[0, k^2) column by column (a column's new place
  DIAF_PHASE(6);
  // lies below every later column's old one), and a copy R0 of it at
  // W[k^2, 2k^2) for recovering V after the sweeps.  Lane `sub` owns rows
  // sub + 4u (u < nk) of every k x k column.
  const int nk = (k - sub + 3) >> 2;
  for (int c = 0; c < k; ++c) {
    const float* src = qptr(W, c * m + sub);
    float t4[kQK];
#pragma unroll
    for (int u = 0; u < kQK; ++u) t4[u] = (u < nk && sub + 4 * u <= c) ? src[32 * u] : 0.0f;
    __syncwarp(qm);
    float* dst = qptr(W, c * k + sub);
#pragma unroll
    for (int u = 0; u < kQK; ++u)
      if (u < nk) dst[32 * u] = t4[u];
    __syncwarp(qm);
  }
  const int VO = k * k;  // R0, or V = I when R-hat is singular
  for (int c = 0; c < k; ++c) {
    const float* src = qptr(W, c * k + sub);
    float* dst = qptr(W, VO + c * k + sub);
#pragma unroll
    for (int u = 0; u < kQK; ++u)
      if (u < nk) dst[32 * u] = zdiag ? (sub + 4 * u == c ? 1.0f : 0.0f) : src[32 * u];
  }

  // ---- one-sided Jacobi on R-hat in the warp kernels' round-robin order
  DIAF_PHASE(5);
  // (the rotations are applied to R-hat only: V is recovered afterwards from
  // R-hat V = B as R0^-1 B, which costs one triangular solve per column
  // instead of a second pair of column updates per rotation; a singular
  // R-hat has no R0^-1, and then V is accumulated in the rotations)
  // (in round rnd, position p >= 1 holds column 1 + ((p - 1 + rnd) mod L) and
  // positions p, qq - 1 - p pair up), with their rotation and stopping rules:
  // skip below tol = k eps_32, stop after a sweep without a rotation of
  // |gamma|^2 >= tol alpha beta; norms carried through rotations.  The pairs
  // of a round are disjoint: kJP of them are rotated together (independent
  // chains).
  // Every lane of the quad writes the same norms.
  uint32_t flags = 0;
  {
    float nf2 = 0.0f;
    for (int c = 0; c < k; ++c) {
      const float* pc = qptr(W, c * k + sub);
#pragma unroll
      for (int u = 0; u < kQK; ++u)
        if (u < nk) nf2 = fmaf(pc[32 * u], pc[32 * u], nf2);
    }
    nf2 = qsum(nf2, qm);
    const float tol = (float)k * FLT_EPSILON;
    const float tol2 = tol * tol;
    const float tiny = tol2 * nf2;
    const int qq = (k + 1) & ~1;
    const int npairs = qq / 2;
    const int L = qq - 1;
    const uint8_t* tab = &kPairTab[npairs - 1][0][0];
    auto pair_of = [&](int pr, int rnd) -> int2 {
      if (pr >= npairs) return make_int2(-1, -1);
      const int ab = tab[rnd * kPairSlots + pr];
      const int x = ab >> 4, y = ab & 15;
      return y < k ? make_int2(x, y) : make_int2(-1, -1);  // a bye for the padding column
    };
    int sweep = 1;
    for (; sweep <= kMaxSweeps; ++sweep) {
      for (int c = 0; c < k; ++c) {
        const float* pc = qptr(W, c * k + sub);
        float s2 = 0.0f;
#pragma unroll
        for (int u = 0; u < kQK; ++u)
          if (u < nk) s2 = fmaf(pc[32 * u], pc[32 * u], s2);
        QS(W, NR + c) = qsum(s2, qm);
      }
      bool large = false;
      if (k >= 2) {
        for (int rnd = 0; rnd < L; ++rnd) {
          for (int pr = 0; pr < npairs; pr += kJP) {
            int pa[kJP], pb[kJP];
#pragma unroll
            for (int h = 0; h < kJP; ++h) {
              const int2 ph = pair_of(pr + h, rnd);
              pa[h] = ph.x;
              pb[h] = ph.y;
            }
            float xa[kJP][kQK], xb[kJP][kQK], g[kJP];
            float *ga[kJP], *gb[kJP];
#pragma unroll
            for (int h = 0; h < kJP; ++h) {
              const bool act = pb[h] >= 0;
              ga[h] = qptr(W, (act ? pa[h] : 0) * k + sub);
              gb[h] = qptr(W, (act ? pb[h] : 0) * k + sub);
              g[h] = 0.0f;
#pragma unroll
              for (int u = 0; u < kQK; ++u) {
                xa[h][u] = (act && u < nk) ? ga[h][32 * u] : 0.0f;
                xb[h][u] = (act && u < nk) ? gb[h][32 * u] : 0.0f;
                g[h] = fmaf(xa[h][u], xb[h][u], g[h]);
              }
            }
#pragma unroll
            for (int h = 0; h < kJP; ++h) g[h] += __shfl_xor_sync(qm, g[h], 1);
#pragma unroll
            for (int h = 0; h < kJP; ++h) g[h] += __shfl_xor_sync(qm, g[h], 2);
#pragma unroll
            for (int h = 0; h < kJP; ++h) {
              if (pb[h] < 0) continue;
              const float al = QS(W, NR + pa[h]), be = QS(W, NR + pb[h]);
              const float g2 = g[h] * g[h];
              if (!(al > tiny && be > tiny && g2 > 0.0f && g2 > tol2 * (al * be))) continue;
              if (g2 >= tol * (al * be)) large = true;
              const float ag = fabsf(g[h]);
              const float d = be - al;
              const float t = __fdividef(copysignf(2.0f * ag, d), fabsf(d) + sqrtf(d * d + 4.0f * g2));
              const float cs = rsqrtf(1.0f + t * t), sn = cs * t;
              const float ssn = g[h] < 0.0f ? -sn : sn, scs = g[h] < 0.0f ? -cs : cs;  // y = sign(g) b
#pragma unroll
              for (int u = 0; u < kQK; ++u)
                if (u < nk) {
                  ga[h][32 * u] = fmaf(-ssn, xb[h][u], cs * xa[h][u]);
                  gb[h][32 * u] = fmaf(scs, xb[h][u], sn * xa[h][u]);
                }
              if (zdiag) {  // V accumulated: R0^-1 B does not exist
                float* va = qptr(W, VO + pa[h] * k + sub);
                float* vb = qptr(W, VO + pb[h] * k + sub);
#pragma unroll
                for (int u = 0; u < kQK; ++u)
                  if (u < nk) {
                    const float xv = va[32 * u], yv = vb[32 * u];
                    va[32 * u] = fmaf(-ssn, yv, cs * xv);
                    vb[32 * u] = fmaf(scs, yv, sn * xv);
                  }
              }
              QS(W, NR + pa[h]) = al - t * ag;
              QS(W, NR + pb[h]) = be + t * ag;
            }
          }
        }
      }
      if (!large) break;
    }
    if (sweep > kMaxSweeps) flags |= DIAF_FLAG_JACOBI_NOCONV;
  }
  __syncwarp(qm);

  // ---- singular values (column norms of R-hat V), the smallest and its gap
  DIAF_PHASE(7);
  for (int c = 0; c < k; ++c) {
    const float* pc = qptr(W, c * k + sub);
    float s2 = 0.0f;
#pragma unroll
    for (int u = 0; u < kQK; ++u)
      if (u < nk) s2 = fmaf(pc[32 * u], pc[32 * u], s2);
    QS(W, NR + c) = sqrtf(qsum(s2, qm));
  }
  int imin = 0;
  double smin = (double)QS(W, NR), smax = smin;
  for (int c = 1; c < k; ++c) {
    const double sv = (double)QS(W, NR + c);
    if (sv < smin) { smin = sv; imin = c; }
    smax = fmax(smax, sv);
  }
  double snext = INFINITY, gap = INFINITY;
  for (int c = 0; c < k; ++c)
    if (c != imin) {
      const double sv = (double)QS(W, NR + c);
      snext = fmin(snext, sv);
      gap = fmin(gap, sv * sv - smin * smin);
    }
  // V = R0^-1 B in place of B (R-hat regular): lane `sub` solves for the columns sub + 4v,
  // column-oriented back substitution (column jj of R0 read through four
  // pointers, element jj k + 4u + w at P[w][32 u])
  __syncwarp(qm);  // every lane has read B for the norms
  for (int c = zdiag ? k : sub; c < k; c += 4) {
    float bv[KMAX];
    const float* P0 = qptr(W, c * k);
    const float* P1 = qptr(W, c * k + 1);
    const float* P2 = qptr(W, c * k + 2);
    const float* P3 = qptr(W, c * k + 3);
#pragma unroll
    for (int i = 0; i < KMAX; ++i) {
      const float* P = (i & 3) == 0 ? P0 : ((i & 3) == 1 ? P1 : ((i & 3) == 2 ? P2 : P3));
      bv[i] = i < k ? P[32 * (i >> 2)] : 0.0f;
    }
#pragma unroll
    for (int jj = KMAX - 1; jj >= 0; --jj) {
      if (jj < k) {
        const float* R0 = qptr(W, VO + jj * k);
        const float* R1 = qptr(W, VO + jj * k + 1);
        const float* R2 = qptr(W, VO + jj * k + 2);
        const float* R3 = qptr(W, VO + jj * k + 3);
        const float* Rd = (jj & 3) == 0 ? R0 : ((jj & 3) == 1 ? R1 : ((jj & 3) == 2 ? R2 : R3));
        bv[jj] = bv[jj] / Rd[32 * (jj >> 2)];
#pragma unroll
        for (int i = 0; i < jj; ++i) {
          const float* R = (i & 3) == 0 ? R0 : ((i & 3) == 1 ? R1 : ((i & 3) == 2 ? R2 : R3));
          bv[i] = fmaf(-R[32 * (i >> 2)], bv[jj], bv[i]);
        }
      }
    }
    float* Q0 = qptr(W, c * k);
    float* Q1 = qptr(W, c * k + 1);
    float* Q2 = qptr(W, c * k + 2);
    float* Q3 = qptr(W, c * k + 3);
#pragma unroll
    for (int i = 0; i < KMAX; ++i) {
      float* Q = (i & 3) == 0 ? Q0 : ((i & 3) == 1 ? Q1 : ((i & 3) == 2 ? Q2 : Q3));
      if (i < k) Q[32 * (i >> 2)] = bv[i];
    }
  }
  __syncwarp(qm);
  if (k > 1 && (snext - smin) <= 1e-6 * smax) flags |= DIAF_FLAG_DEGENERATE;
  if (k > 1 && gap <= 1e-5 * smax * smax) { defer(); return; }
  const int iters = (k > 1 && gap < 1e-2 * smax * smax) ? 2 : 1;

  // ---- FP64 correction in the FP32 singular basis V: d = x^T H x / x^T x,
  // r = H x - d x (H = A-hat^T A-hat from the FP64 tile),
  // x <- x - sum_{i != imin} V_i (V_i^T r) / (sigma_i^2 - d).  x (k) in the
  // quad's FP64 shared scratch, z = A-hat x (m) in its slab: lane `sub` computes z
  // on its tile rows and (A-hat^T z)_q, r_q and the update of x_q on its rows
  // q of V.
  double* X = D;  // x, element q
  const int zo = (M * K + 3) / 4 * 4;  // z, element r: slab element zo + r
  {
    const float* vmin = qptr(W, (zdiag ? VO : 0) + imin * k + sub);
    double* xs = qptr(X, sub);
#pragma unroll
    for (int u = 0; u < kQK; ++u)
      if (u < nk) xs[32 * u] = (double)vmin[32 * u];
  }
  __syncwarp(qm);
  for (int it = 0; it < iters; ++it) {
    double zz = 0.0;
    for (int t = 0; t < nown; ++t) {
      const int r = sub + 4 * t;
      double z = 0.0;
      if (!((inI >> r) & 1u))
        for (int q = 0; q < k; ++q) z = fma(T(r + q * m), QS(X, q), z);
      T(zo + r) = z;
      zz = fma(z, z, zz);
    }
    double xx = 0.0;
    {
      const double* xs = qptr(X, sub);
#pragma unroll
      for (int u = 0; u < kQK; ++u)
        if (u < nk) xx = fma(xs[32 * u], xs[32 * u], xx);
    }
    const double d = qsum(zz, qm) / qsum(xx, qm);
    __syncwarp(qm);  // z complete
    float rfo[kQK];  // r on the lane's rows of V, in FP32
    double xo[kQK], gq[kQK];
#pragma unroll
    for (int u = 0; u < kQK; ++u) gq[u] = 0.0;
    for (int r = 0; r < m; ++r) {  // rows in I_j have z_r = 0
      const double zr = T(zo + r);
#pragma unroll
      for (int u = 0; u < kQK; ++u)
        if (u < nk) gq[u] = fma(T(r + (sub + 4 * u) * m), zr, gq[u]);
    }
#pragma unroll
    for (int u = 0; u < kQK; ++u) {
      const int q = sub + 4 * u;
      rfo[u] = 0.0f;
      xo[u] = 0.0;
      if (u < nk) {
        xo[u] = QS(X, q);
        rfo[u] = (float)(gq[u] - d * xo[u]);
      }
    }
    float dxo[kQK];
#pragma unroll
    for (int u = 0; u < kQK; ++u) dxo[u] = 0.0f;
    for (int i = 0; i < k; ++i) {
      const float* vi = qptr(W, (zdiag ? VO : 0) + i * k + sub);
      float vo[kQK];
      float vr = 0.0f;
#pragma unroll
      for (int u = 0; u < kQK; ++u) {
        vo[u] = u < nk ? vi[32 * u] : 0.0f;
        vr = fmaf(vo[u], rfo[u], vr);
      }
      vr = qsum(vr, qm);
      if (i == imin) continue;
      const float sl = QS(W, NR + i);
      const float ci = -vr / (sl * sl - (float)d);
#pragma unroll
      for (int u = 0; u < kQK; ++u) dxo[u] = fmaf(vo[u], ci, dxo[u]);
    }
    __syncwarp(qm);  // every lane has read x and z
    {
      double* xs = qptr(X, sub);
#pragma unroll
      for (int u = 0; u < kQK; ++u)
        if (u < nk) xs[32 * u] = xo[u] + (double)dxo[u];
    }
    __syncwarp(qm);
  }
  {
    double xn2 = 0.0;
    double* xs = qptr(X, sub);
#pragma unroll
    for (int u = 0; u < kQK; ++u)
      if (u < nk) xn2 = fma(xs[32 * u], xs[32 * u], xn2);
    const double inv = 1.0 / sqrt(qsum(xn2, qm));
    __syncwarp(qm);
#pragma unroll
    for (int u = 0; u < kQK; ++u)
      if (u < nk) xs[32 * u] *= inv;
    __syncwarp(qm);
  }

  // ---- v = T(I_j,:) w (into V's values by the row owners), phase v_jj >= 0,
  DIAF_PHASE(8);
  // FP64 residual
  double* Vout = reinterpret_cast<double*>(a.Vv) + v0;
  double vn2 = 0.0, vjj = 0.0, r2 = 0.0;
  if (sub == 0 && !jin) Vout[jpos] = 0.0;
  // rows in I_j: v_r = (T w)_r, so their term of ||T w - v|| is exactly zero;
  // the other rows contribute (T w)_r (the residual from its definition)
  for (int t = 0; t < nown; ++t) {
    const int r = sub + 4 * t;
    double sv = 0.0;
    for (int q = 0; q < k; ++q) sv = fma(T(r + q * m), QS(X, q), sv);
    if ((inI >> r) & 1u) {
      Vout[pos_of(r)] = sv;
      vn2 = fma(sv, sv, vn2);
      if (r == rj) vjj = sv;
    } else {
      r2 = fma(sv, sv, r2);
    }
  }
  vn2 = qsum(vn2, qm);
  vjj = qsum(vjj, qm);
  double ph = 1.0;
  const double zl = 64.0 * DBL_EPSILON;
  if (vjj * vjj > zl * zl * vn2) {
    ph = vjj < 0.0 ? -1.0 : 1.0;
  } else {
    flags |= DIAF_FLAG_VJJ_ZERO;
    double amx = 0.0, wsel = 1.0;
    for (int q = 0; q < k; ++q) {
      const double xq = QS(X, q);
      if (fabs(xq) > amx) { amx = fabs(xq); wsel = xq; }
    }
    ph = wsel < 0.0 ? -1.0 : 1.0;
  }
  bool finite = true;
  for (int t = 0; t < nown; ++t) {
    const int r = sub + 4 * t;
    if ((inI >> r) & 1u) {
      const int pos = pos_of(r);
      const double vt = Vout[pos];
      Vout[pos] = ph * vt;
      finite &= isfinite(vt);
    }
  }
  r2 = qsum(r2, qm);
  const double resj = sqrt(r2);
  if (resj <= 1e-14 * smax) flags |= DIAF_FLAG_RANK_DEFICIENT;
  finite &= isfinite(resj);
  double* Wout = reinterpret_cast<double*>(a.Wv) + a.Wcp[j];
  for (int q = sub; q < k; q += 4) {
    const double wq = ph * QS(X, q);
    finite &= isfinite(wq);
    Wout[q] = wq;
  }
  const unsigned fin = __ballot_sync(qm, finite) & qm;
  if (fin != qm) flags |= DIAF_FLAG_NONFINITE;
  if (sub == 0) {
    a.res[j] = resj;
    a.flags[j] = flags | a.extra_flags;
  }
  if (a.Hri) {  // the final I_j to the host (the rows as written above), then the column's word
    if (sub == 0 && !jin) a.Hri[v0 + jpos] = j;
    for (int r = sub; r < m; r += 4)
      if ((inI >> r) & 1u) a.Hri[v0 + pos_of(r)] = Rj[r];
    __threadfence_system();
    __syncwarp(qm);
    if (sub == 0) store_release_sys(a.Hgen + j, a.gen);
  }
  DIAF_PHASE(9);
}

// The persistent loop: each warp takes eight columns of the list at a time,
// one per quad.
template <int KMAX>
__global__ void __launch_bounds__(32 * kQuadWarps, 16) column_thread_kernel(ColArgs a, ThreadArgs ta) {
  extern __shared__ __align__(16) float tsmem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int sub = lane & 3, slot = lane >> 2;
  const unsigned qm = 0xFu << (lane & ~3);
  const int gq = (blockIdx.x * kQuadWarps + warp) * kQuadCols + slot;  // quad index in the grid
  const int M = ta.M, K = ta.K;
  unsigned char* wbase = reinterpret_cast<unsigned char*>(tsmem) + (size_t)warp * thread_warp_smem(M, K);
  float* S = reinterpret_cast<float*>(wbase) + slot;
  double* D = reinterpret_cast<double*>(wbase + sizeof(float) * (size_t)thread_arena_floats(M, K) * 8) + slot;
  double* G = ta.slab + (size_t)4 * gq;  // element e of the quad's tile at G[(e/4) 4 nquads + (e mod 4)]
  const int count = *a.list_count;
  while (true) {
    int base = 0;
    if (lane == 0) base = atomicAdd(a.work_counter, kQuadCols);
    base = __shfl_sync(DIAF_FULL, base, 0);
    if (base >= count) break;
    const int idx = base + slot;
    if (idx < count) solve_column_quad<KMAX>(a, ta, list_at(a, count, idx), S, D, G, sub, qm);
    __syncwarp();
  }
}

#undef QS
