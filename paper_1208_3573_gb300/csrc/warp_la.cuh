// Warp-cooperative dense linear algebra on small tiles in shared memory
// (column-major), shared by the FP64 and the mixed-precision column kernels:
// Householder QR, one-sided Jacobi SVD, leverage rows Q = T R^-1, and the
// two triangular solves with R^* and R.
//
// Cost model on GB300: FP64 warp instructions are the scarce resource, so the
// routines avoid divisions and square roots inside loops (reciprocals are
// formed once) and use |x| / sign(x) directly for real data.
#pragma once

#include <cfloat>
#include <climits>
#include <type_traits>

#include "common.cuh"

// Jacobi sweep limit (a test build lowers it to check the flag it sets).
#ifndef DIAF_MAX_SWEEPS
#define DIAF_MAX_SWEEPS 30
#endif
constexpr int kMaxSweeps = DIAF_MAX_SWEEPS;

template <class T> __device__ __forceinline__ T eps_of();
template <> __device__ __forceinline__ double eps_of<double>() { return DBL_EPSILON; }
template <> __device__ __forceinline__ float eps_of<float>() { return FLT_EPSILON; }

__device__ __forceinline__ double sc_abs(double a) { return fabs(a); }
__device__ __forceinline__ float sc_abs(float a) { return fabsf(a); }
template <class R> __device__ __forceinline__ R sc_abs(Cx<R> a) { return sqrt(sc_abs2(a)); }

__device__ __forceinline__ double rsqrt_r(double a) { return rsqrt(a); }
__device__ __forceinline__ float rsqrt_r(float a) { return rsqrtf(a); }

// a / b: IEEE in FP64; the fast approximate division in FP32 (about 2 ulp),
// whose results only seed the FP64 refinement of the mixed form
__device__ __forceinline__ double div_r(double a, double b) { return a / b; }
__device__ __forceinline__ float div_r(float a, float b) { return __fdividef(a, b); }

// a / |a| (1 for a == 0)
__device__ __forceinline__ double sc_unit(double a) { return a < 0.0 ? -1.0 : 1.0; }
__device__ __forceinline__ float sc_unit(float a) { return a < 0.0f ? -1.0f : 1.0f; }
template <class R> __device__ __forceinline__ Cx<R> sc_unit(Cx<R> a) {
  R n2 = sc_abs2(a);
  if (n2 == R(0)) return {R(1), R(0)};
  R inv = rsqrt_r(n2);
  return {a.re * inv, a.im * inv};
}

// 1 / d for a nonzero scalar, 0 when |d| <= piv
template <class S>
__device__ __forceinline__ S sc_recip_or_zero(S d, RealOf<S> piv) {
  using R = RealOf<S>;
  R a2 = sc_abs2(d);
  if (!(sc_abs(d) > piv)) return sc_zero<S>();
  return div_r(R(1), a2) * sc_conj(d);
}

__device__ __forceinline__ bool admissible_row(int rule, int i, int j, const int32_t* blk) {
  if (i == j) return false;
  if (rule == DIAF_RULE_UPPER) return i < j;
  if (rule == DIAF_RULE_LOWER) return i > j;
  if (rule == DIAF_RULE_BLOCK) return blk[i] == blk[j];
  return true;
}

// ------------------------------------------------------------------ QR
// Householder QR of the column-major m x k matrix T (leading dimension LD)
// in place: reflector c maps x = T(c:m, c) to beta e_1 with
// beta = -(x_0/|x_0|) ||x||, u = x - beta e_1, u^* u = 2 ||x|| (||x|| + |x_0|).
// On return rows 0..min(m,k)-1 hold R (zeros below the diagonal).
template <class S, int LD>
__device__ void warp_householder_qr(S* T, int m, int k, int lane) {
  using R = RealOf<S>;
  int p = m < k ? m : k;
  for (int c = 0; c < p; ++c) {
    S* tc = T + c * LD;
    R nrm2 = R(0);
    for (int r = c + lane; r < m; r += DIAF_WARP) nrm2 += sc_abs2(tc[r]);
    nrm2 = warp_sum(nrm2);
    S alpha = tc[c];
    __syncwarp();
    if (nrm2 == R(0)) continue;
    R ax = sc_abs(alpha);
    R nrm = sqrt(nrm2);
    S ph = sc_unit(alpha);
    S beta = -(nrm * ph);
    S u0 = (ax + nrm) * ph;
    R two_uu = div_r(R(1), nrm * (nrm + ax));
    for (int q = c + 1; q < k; ++q) {
      S* tq = T + q * LD;
      S part = sc_zero<S>();
      for (int r = c + lane; r < m; r += DIAF_WARP) part += sc_cmul(r == c ? u0 : tc[r], tq[r]);
      S f = two_uu * warp_sum(part);
      for (int r = c + lane; r < m; r += DIAF_WARP) tq[r] -= f * (r == c ? u0 : tc[r]);
    }
    __syncwarp();
    for (int r = c + lane; r < m; r += DIAF_WARP) tc[r] = (r == c) ? beta : sc_zero<S>();
    __syncwarp();
  }
}

// Butterfly reduce-scatter of NQ values (NQ a power of two, 2..32) across the
// warp: at each of the log2(NQ) steps a lane keeps one half of its values
// (the upper half when its lane bit is set) and adds the partner's copy of
// that half, received for the half it gives away; the lane bits left over
// finish with a plain butterfly sum.  On return lane L holds the warp-wide
// sum of value L >> (5 - log2 NQ), with log2(NQ) + 1 ... 5 dependent
// shuffles instead of 5 per value.
constexpr int ilog2_c(int x) { return x <= 1 ? 0 : 1 + ilog2_c(x / 2); }

template <class S, int NQ>
__device__ __forceinline__ S warp_reduce_scatter(S (&v)[NQ], int lane) {
  constexpr int LOG = ilog2_c(NQ);
  static_assert((1 << LOG) == NQ && NQ >= 2 && NQ <= 32, "NQ must be a power of two in [2, 32]");
#pragma unroll
  for (int t = 0; t < LOG; ++t) {
    const int mask = 16 >> t;
    const int half = NQ >> (t + 1);
    const bool upper = (lane & mask) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const S give = upper ? v[i] : v[i + half];
      const S keep = upper ? v[i + half] : v[i];
      v[i] = keep + shfl_xor(give, mask);
    }
  }
#pragma unroll
  for (int t = LOG; t < 5; ++t) v[0] += shfl_xor(v[0], 16 >> t);
  return v[0];
}

// Householder QR as warp_householder_qr (same reflectors), with all the
// trailing-column products of one reflector formed together: lane r owns rows
// r, r + 32, ... (MR rows, m <= 32 MR), the k <= NQ partial sums go through one
// reduce-scatter and come back by one broadcast each.
template <class S, int LD, int NQ, int MR>
__device__ void warp_householder_qr_rs(S* T, int m, int k, int lane) {
  using R = RealOf<S>;
  constexpr int LOG = ilog2_c(NQ);
  const int p = m < k ? m : k;
  for (int c = 0; c < p; ++c) {
    S* tc = T + c * LD;
    S ur[MR];
    R nrm2 = R(0);
#pragma unroll
    for (int i = 0; i < MR; ++i) {
      const int r = lane + DIAF_WARP * i;
      ur[i] = (r >= c && r < m) ? tc[r] : sc_zero<S>();
      nrm2 += sc_abs2(ur[i]);
    }
    nrm2 = warp_sum(nrm2);
    const S alpha = tc[c];
    __syncwarp();
    if (nrm2 == R(0)) continue;
    const R ax = sc_abs(alpha);
    const R nrm = sqrt(nrm2);
    const S ph = sc_unit(alpha);
    const S beta = -(nrm * ph);
    const S u0 = (ax + nrm) * ph;
    const R two_uu = div_r(R(1), nrm * (nrm + ax));
#pragma unroll
    for (int i = 0; i < MR; ++i)
      if (lane + DIAF_WARP * i == c) ur[i] = u0;
    if (c + 1 < k) {
      S v[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        S acc = sc_zero<S>();
        if (q > c && q < k) {
#pragma unroll
          for (int i = 0; i < MR; ++i) {
            const int r = lane + DIAF_WARP * i;
            if (r < m) acc += sc_cmul(ur[i], T[r + q * LD]);
          }
        }
        v[q] = acc;
      }
      const S fmine = two_uu * warp_reduce_scatter<S, NQ>(v, lane);
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        if (q > c && q < k) {  // warp-uniform
          const S fq = shfl_idx(fmine, q << (5 - LOG));
#pragma unroll
          for (int i = 0; i < MR; ++i) {
            const int r = lane + DIAF_WARP * i;
            if (r >= c && r < m) T[r + q * LD] -= fq * ur[i];
          }
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < MR; ++i) {
      const int r = lane + DIAF_WARP * i;
      if (r >= c && r < m) tc[r] = (r == c) ? beta : sc_zero<S>();
    }
    __syncwarp();
  }
}

// The same Householder QR for tiles of at most 32 rows and NQ <= 16
// columns with the tile in registers: lane r holds row r (converted from the
// tile T of type ST, leading dimension LDT; rows with mask[r] >= 0 read as
// zero when mask is given), so no trailing-column loads or stores go through
// shared memory.  Writes the k x k upper R to Rout (leading dimension LDR;
// it must not alias T)
// and the FP64 value of the column norms ||T(:,c)|| (of the masked tile) to
// cn[c].
template <class S, class ST, int LDT, int LDR, int NQ>
__device__ void warp_qr_rows(const ST* T, const int32_t* mask, int m, int k, S* Rout, double* cn, int lane) {
  using R = RealOf<S>;
  static_assert(NQ >= 2 && NQ <= 16, "row-register QR: at most 16 columns");
  constexpr int LOG = ilog2_c(NQ);
  S x[NQ];
  const bool live = lane < m && !(mask && mask[lane] >= 0);
#pragma unroll
  for (int q = 0; q < NQ; ++q) x[q] = (live && q < k) ? sc_cast<S>(T[lane + q * LDT]) : sc_zero<S>();
  {
    R v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = sc_abs2(x[q]);
    const R tot = warp_reduce_scatter<R, NQ>(v, lane);  // lane L: column L >> (5 - LOG)
    const int q = lane >> (5 - LOG);
    if ((lane & ((1 << (5 - LOG)) - 1)) == 0 && q < k) cn[q] = (double)sqrt(tot);
  }
  // R starts as zeros; row c is written by lane c once reflector c is applied
  for (int i = lane; i < k * k; i += DIAF_WARP) Rout[(i % k) + (i / k) * LDR] = sc_zero<S>();
  __syncwarp();
  // step c works on x[0] = column c: after it the row's entries shift down by
  // one, so every step runs the same code (no unrolling over c: small code)
  const int p = m < k ? m : k;
  for (int c = 0; c < p; ++c) {
    const R nrm2 = warp_sum(lane >= c ? sc_abs2(x[0]) : R(0));
    const S alpha = shfl_idx(x[0], c);
    if (nrm2 != R(0)) {
      const R ax = sc_abs(alpha);
      const R nrm = sqrt(nrm2);
      const S ph = sc_unit(alpha);
      const S beta = -(nrm * ph);
      const S u0 = (ax + nrm) * ph;
      const R two_uu = div_r(R(1), nrm * (nrm + ax));
      const S u = lane > c ? x[0] : (lane == c ? u0 : sc_zero<S>());
      const int rest = k - c;  // columns c .. k-1 are x[0 .. rest-1]
      if (rest > 1) {
        S v[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] = (q >= 1 && q < rest) ? sc_cmul(u, x[q]) : sc_zero<S>();
        const S fmine = two_uu * warp_reduce_scatter<S, NQ>(v, lane);
#pragma unroll
        for (int q = 1; q < NQ; ++q) {
          if (q < rest) {  // warp-uniform
            const S fq = shfl_idx(fmine, q << (5 - LOG));
            x[q] -= fq * u;
          }
        }
      }
      if (lane == c) x[0] = beta;
    }
    if (lane == c) {
#pragma unroll
      for (int q = 0; q < NQ; ++q)
        if (q < k - c) Rout[c + (c + q) * LDR] = x[q];
    }
#pragma unroll
    for (int q = 0; q + 1 < NQ; ++q) x[q] = x[q + 1];
    x[NQ - 1] = sc_zero<S>();
  }
  __syncwarp();
}

// ------------------------------------------------------------------ Jacobi
// Parallel one-sided (Hestenes) Jacobi on the p x q matrix G (leading
// dimension LDG): G V has orthogonal columns, V (q x q, leading dimension
// LDV) unitary.  Round-robin ordering: in each of the qq-1 rounds of a sweep
// (qq = q rounded up to even) the columns split into qq/2 disjoint pairs, one
// group of LPP lanes per pair.  A pair (a, b) with alpha = |g_a|^2,
// beta = |g_b|^2, gamma = g_a^* g_b is rotated when |gamma| > tol
// sqrt(alpha beta), tol = p eps, and neither column is below p eps ||G||_F:
// b' = e^{-i arg gamma} b, then [a b'] [[c, s], [-s, c]] with t = s / c the
// smaller root of t^2 + 2 zeta t - 1 = 0, zeta = (beta - alpha) / (2|gamma|),
// i.e. t = sign(d) 2|gamma| / (|d| + sqrt(d^2 + 4|gamma|^2)), d = beta - alpha.
// Returns sweeps used, or -1 at the sweep limit.
// PREDICT (reduced-precision callers whose result is refined afterwards):
// the sweep that would only confirm convergence is skipped -- once every
// rotation of a sweep had |gamma| < sqrt(tol) sqrt(alpha beta), Jacobi's
// quadratic convergence leaves the next sweep's ratios near tol.
template <class S, int LDG, int LDV, int QMAX, bool PREDICT = false>
__device__ int warp_jacobi(S* G, int p, int q, S* V, int lane) {
  using R = RealOf<S>;
  constexpr int kPairsMax = QMAX / 2;
  constexpr int kGroups = kPairsMax >= 32 ? 32 : (kPairsMax >= 16 ? 16 : (kPairsMax >= 8 ? 8 : (kPairsMax >= 4 ? 4 : 2)));
  constexpr int LPP = DIAF_WARP / kGroups;
  for (int i = lane; i < q * q; i += DIAF_WARP) {
    int r = i % q, c = i / q;
    V[r + c * LDV] = (r == c) ? sc_real_s<S>(R(1)) : sc_zero<S>();
  }
  R nf2 = R(0);
  for (int i = lane; i < p * q; i += DIAF_WARP) nf2 += sc_abs2(G[(i % p) + (i / p) * LDG]);
  nf2 = warp_sum(nf2);
  const R tol = R(p > 1 ? p : 1) * eps_of<R>();
  const R tol2 = tol * tol;
  const R tiny = tol2 * nf2;
  __syncwarp();
  if (q < 2) return 1;
  const int qq = (q + 1) & ~1;
  const int npairs = qq / 2;
  const int grp = lane / LPP, sub = lane % LPP;
  const int L = qq - 1;
  for (int sweep = 1; sweep <= kMaxSweeps; ++sweep) {
    bool rotated = false;
    bool large = false;  // PREDICT: a rotation with |gamma|^2 >= tol alpha beta
    for (int rnd = 0; rnd < L; ++rnd) {
      for (int pr0 = 0; pr0 < npairs; pr0 += kGroups) {
        int pr = pr0 + grp;
        int a = -1, b = -1;
        if (pr < npairs) {
          // position p >= 1 holds column 1 + ((p - 1 + rnd) mod L)
          int pb = qq - 1 - pr;
          int ea = pr - 1 + rnd, eb = pb - 1 + rnd;
          if (ea >= L) ea -= L;
          if (eb >= L) eb -= L;
          a = pr == 0 ? 0 : 1 + ea;
          b = 1 + eb;
          if (a > b) { int t = a; a = b; b = t; }
          if (b >= q) a = -1;  // bye for the padding column
        }
        bool act = a >= 0;
        R al = R(0), be = R(0);
        S ga = sc_zero<S>();
        if (act) {
          const S* ca = G + a * LDG;
          const S* cb = G + b * LDG;
          for (int i = sub; i < p; i += LPP) {
            S x = ca[i], y = cb[i];
            al += sc_abs2(x);
            be += sc_abs2(y);
            ga += sc_cmul(x, y);
          }
        }
        al = group_sum<LPP>(al);
        be = group_sum<LPP>(be);
        ga = group_sum<LPP>(ga);
        const R ag2 = sc_abs2(ga);
        bool rot = act && al > tiny && be > tiny && ag2 > R(0) && ag2 > tol2 * (al * be);
        if (rot) {
          rotated = true;
          if (PREDICT && ag2 >= tol * (al * be)) large = true;
          R ag;
          S eph;
          if constexpr (ScalarInfo<S>::cplx) {
            R rinv = rsqrt_r(ag2);
            ag = ag2 * rinv;
            eph = rinv * sc_conj(ga);
          } else {
            ag = sc_abs(ga);
            eph = sc_unit(ga);
          }
          const R d = be - al;
          const R t = div_r(copysign(R(2) * ag, d), fabs(d) + sqrt(d * d + R(4) * ag2));
          const R cs = rsqrt_r(R(1) + t * t), sn = cs * t;
          S* ca = G + a * LDG;
          S* cb = G + b * LDG;
          for (int i = sub; i < p; i += LPP) {
            S x = ca[i], y = eph * cb[i];
            ca[i] = cs * x - sn * y;
            cb[i] = sn * x + cs * y;
          }
          S* va = V + a * LDV;
          S* vb = V + b * LDV;
          for (int i = sub; i < q; i += LPP) {
            S x = va[i], y = eph * vb[i];
            va[i] = cs * x - sn * y;
            vb[i] = sn * x + cs * y;
          }
        }
        __syncwarp();
      }
    }
    if (!__any_sync(DIAF_FULL, rotated)) return sweep;
    if (PREDICT && !__any_sync(DIAF_FULL, large)) return sweep;
  }
  return -1;
}

// The same Jacobi for reduced-precision callers whose result is refined
// afterwards (PREDICT behaviour), tuned for small tiles: p <= PMAX rows, so a
// lane keeps its share of the pair's two columns in registers between the
// inner product and the rotation, and the squared column norms live in nrm
// (q scratch values of the real type): exact at the start of every sweep,
// then updated per rotation by alpha' = alpha - t |gamma|,
// beta' = beta + t |gamma| (the rotated pair's norms in exact arithmetic), so
// a pair needs only gamma = g_a^* g_b.
template <class S, int LDG, int LDV, int QMAX, int PMAX>
__device__ int warp_jacobi_reg(S* G, int p, int q, S* V, RealOf<S>* nrm, int lane) {
  using R = RealOf<S>;
  constexpr int kPairsMax = QMAX / 2;
  constexpr int kGroups = kPairsMax >= 32 ? 32 : (kPairsMax >= 16 ? 16 : (kPairsMax >= 8 ? 8 : (kPairsMax >= 4 ? 4 : 2)));
  constexpr int LPP = DIAF_WARP / kGroups;
  constexpr int PER = (PMAX + LPP - 1) / LPP;
  constexpr int VPER = (QMAX + LPP - 1) / LPP;
  for (int i = lane; i < q * q; i += DIAF_WARP) {
    int r = i % q, c = i / q;
    V[r + c * LDV] = (r == c) ? sc_real_s<S>(R(1)) : sc_zero<S>();
  }
  R nf2 = R(0);
  for (int i = lane; i < p * q; i += DIAF_WARP) nf2 += sc_abs2(G[(i % p) + (i / p) * LDG]);
  nf2 = warp_sum(nf2);
  const R tol = R(p > 1 ? p : 1) * eps_of<R>();
  const R tol2 = tol * tol;
  const R tiny = tol2 * nf2;
  __syncwarp();
  if (q < 2) return 1;
  const int qq = (q + 1) & ~1;
  const int npairs = qq / 2;
  const int grp = lane / LPP, sub = lane % LPP;
  const int L = qq - 1;
  for (int sweep = 1; sweep <= kMaxSweeps; ++sweep) {
    for (int c = lane; c < q; c += DIAF_WARP) {
      R s2 = R(0);
      for (int i = 0; i < p; ++i) s2 += sc_abs2(G[i + c * LDG]);
      nrm[c] = s2;
    }
    __syncwarp();
    bool rotated = false, large = false;
    for (int rnd = 0; rnd < L; ++rnd) {
      for (int pr0 = 0; pr0 < npairs; pr0 += kGroups) {
        const int pr = pr0 + grp;
        int a = -1, b = -1;
        if (pr < npairs) {
          int pb = qq - 1 - pr;
          int ea = pr - 1 + rnd, eb = pb - 1 + rnd;
          if (ea >= L) ea -= L;
          if (eb >= L) eb -= L;
          a = pr == 0 ? 0 : 1 + ea;
          b = 1 + eb;
          if (a > b) { int t = a; a = b; b = t; }
          if (b >= q) a = -1;
        }
        const bool act = a >= 0;
        S xa[PER], xb[PER];
        S ga = sc_zero<S>();
        S* ca = G + (act ? a : 0) * LDG;
        S* cb = G + (act ? b : 0) * LDG;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int i = sub + u * LPP;
          xa[u] = sc_zero<S>();
          xb[u] = sc_zero<S>();
          if (act && i < p) {
            xa[u] = ca[i];
            xb[u] = cb[i];
            ga += sc_cmul(xa[u], xb[u]);
          }
        }
        ga = group_sum<LPP>(ga);
        const R al = act ? nrm[a] : R(0), be = act ? nrm[b] : R(0);
        const R ag2 = sc_abs2(ga);
        const bool rot = act && al > tiny && be > tiny && ag2 > R(0) && ag2 > tol2 * (al * be);
        __syncwarp();
        if (rot) {
          rotated = true;
          if (ag2 >= tol * (al * be)) large = true;
          R ag;
          S eph;
          if constexpr (ScalarInfo<S>::cplx) {
            R ri = rsqrt_r(ag2);
            ag = ag2 * ri;
            eph = ri * sc_conj(ga);
          } else {
            ag = sc_abs(ga);
            eph = sc_unit(ga);
          }
          const R d = be - al;
          const R t = div_r(copysign(R(2) * ag, d), fabs(d) + sqrt(d * d + R(4) * ag2));
          const R cs = rsqrt_r(R(1) + t * t), sn = cs * t;
#pragma unroll
          for (int u = 0; u < PER; ++u) {
            const int i = sub + u * LPP;
            if (i < p) {
              const S x = xa[u], y = eph * xb[u];
              ca[i] = cs * x - sn * y;
              cb[i] = sn * x + cs * y;
            }
          }
          S* va = V + a * LDV;
          S* vb = V + b * LDV;
#pragma unroll
          for (int u = 0; u < VPER; ++u) {
            const int i = sub + u * LPP;
            if (i < q) {
              const S x = va[i], y = eph * vb[i];
              va[i] = cs * x - sn * y;
              vb[i] = sn * x + cs * y;
            }
          }
          if (sub == 0) {
            nrm[a] = al - t * ag;
            nrm[b] = be + t * ag;
          }
        }
        __syncwarp();
      }
    }
    if (!__any_sync(DIAF_FULL, rotated)) return sweep;
    if (!__any_sync(DIAF_FULL, large)) return sweep;
  }
  return -1;
}

// column norms of G (p x q) into sigma[c], kept in the factor's own real type
// (reduced-precision callers scan and compare them without FP64 instructions)
template <class S, int LDG>
__device__ void warp_col_norms_r(const S* G, int p, int q, RealOf<S>* sigma, int lane) {
  using R = RealOf<S>;
  for (int c = lane; c < q; c += DIAF_WARP) {
    R s = R(0);
    for (int i = 0; i < p; ++i) s += sc_abs2(G[i + c * LDG]);
    sigma[c] = sqrt(s);
  }
  __syncwarp();
}

// column norms of G (p x q) into sigma[c] (double)
template <class S, int LDG>
__device__ void warp_col_norms(const S* G, int p, int q, double* sigma, int lane) {
  using R = RealOf<S>;
  for (int c = lane; c < q; c += DIAF_WARP) {
    R s = R(0);
    for (int i = 0; i < p; ++i) s += sc_abs2(G[i + c * LDG]);
    sigma[c] = (double)sqrt(s);  // in the factor's own precision
  }
  __syncwarp();
}

// ------------------------------------------------------------------ leverage
// Q = T R^-1 row by row (lane r owns tile row r) and h_r = ||Q(r,:)||^2.
// T: tile of type ST (leading dimension LDT), Rm: k x k upper R (type S,
// leading dimension LDR), Qout: rows of Q (type S, leading dimension LDT),
// rinv: KMAX scratch for the reciprocal diagonal (pivots below piv give 0).
template <class S, class ST, int LDT, int LDR, class K>
__device__ void warp_leverage_rows(const ST* T, const S* Rm, S* Qout, K* hk, S* rinv, int m, int k,
                                   RealOf<S> piv, int lane) {
  using R = RealOf<S>;
  for (int c = lane; c < k; c += DIAF_WARP) rinv[c] = sc_recip_or_zero(Rm[c + c * LDR], piv);
  __syncwarp();
  for (int r = lane; r < m; r += DIAF_WARP) {
    R h = R(0);
    for (int c = 0; c < k; ++c) {
      S acc = sc_cast<S>(T[r + c * LDT]);
      for (int p2 = 0; p2 < c; ++p2) acc -= Qout[r + p2 * LDT] * Rm[p2 + c * LDR];
      S z = acc * rinv[c];
      Qout[r + c * LDT] = z;
      h += sc_abs2(z);
    }
    hk[r] = (K)h;
  }
  __syncwarp();
}

// ------------------------------------------------------------------ triangular solves
// x := R^-1 R^-* x for the k x k upper triangular R (type S, leading dimension
// LDR), in precision SD.  x is held one entry per lane (lane q < k owns x_q);
// rinv: the reciprocal diagonal in SD (lane c reads rinv[c]).  Returns the
// lane's entry.
template <class SD, class S, int LDR>
__device__ SD warp_solve_RhR(const S* Rm, const SD* rinv, SD x, int k, int lane) {
  // forward: R^* u = x  (u_c = (x_c - sum_{p<c} conj(R_pc) u_p) / conj(R_cc))
  for (int c = 0; c < k; ++c) {
    SD uc = shfl_idx(x * sc_conj(rinv[c]), c);
    if (lane > c && lane < k) x -= sc_conj(sc_cast<SD>(Rm[c + lane * LDR])) * uc;
    if (lane == c) x = uc;
  }
  // backward: R y = u
  for (int c = k - 1; c >= 0; --c) {
    SD yc = shfl_idx(x * rinv[c], c);
    if (lane < c) x -= sc_cast<SD>(Rm[lane + c * LDR]) * yc;
    if (lane == c) x = yc;
  }
  return x;
}
