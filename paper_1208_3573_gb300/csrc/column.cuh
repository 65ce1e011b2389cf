// Fused per-column kernel of the columnwise setup, one warp per column, the
// tile in shared memory.  For column j:
//   gather  T = A(R_j, J_j)                       (A_j of eq. spaqr on its nonzero rows)
//   QR      T = Q R, Householder                  (eq. spaqr)
//   keys    h_i = ||Q(i,:)||^2, Q = T R^-1 by rows (norms of the columns of Q_j^*, Sec. 3.1)
//   I_j     diagonal + l_j - 1 admissible rows of largest h (Sec. 3.1), or fixed
//   DIAF-S  QR of T with the I_j rows zeroed, one-sided Jacobi SVD of its R,
//           w = right singular vector of sigma_min, v = T(I_j,:) w     (Sec. 2.2)
//   DIAF-Q  one-sided Jacobi on Q_I = Q(I_j,:): u, sigma = top right singular
//           pair, v = Q_I u / sigma (eq. nocond), w = sigma R^-1 u, the
//           least-squares solution of eq. condwj
//   phase   v_jj real >= 0 (scaling invariance, Sec. 2.1)
//   res     ||A w - v||_2 from its definition; scatter into CSC W and V.
#pragma once

#include <cfloat>
#include <climits>

#include "common.cuh"

struct ColArgs {
  int n;
  const int32_t* Acp;
  const int32_t* Ari;
  const void* Av;
  const int32_t* Wcp;
  const int32_t* Wri;
  const int64_t* Eoff;
  const int32_t* rows;
  const int32_t* m;
  const int32_t* l;
  const int32_t* jin;
  int rule;
  const int32_t* Vfcp;
  const int32_t* Vfri;
  const int32_t* Vcp;
  double tie_tol;
  const int32_t* list;        // bucket's columns
  const int32_t* list_count;  // device count of the list
  int32_t* work_counter;      // zeroed before launch
  void* Wv;
  int32_t* Vri;
  void* Vv;
  double* res;
  uint32_t* flags;
  uint32_t* status;
};

constexpr int kMaxSweeps = 30;

__device__ __forceinline__ bool admissible_row(int rule, int i, int j) {
  if (i == j) return false;
  if (rule == DIAF_RULE_UPPER) return i < j;
  if (rule == DIAF_RULE_LOWER) return i > j;
  return true;
}

template <class T> __device__ __forceinline__ T eps_of();
template <> __device__ __forceinline__ double eps_of<double>() { return DBL_EPSILON; }
template <> __device__ __forceinline__ float eps_of<float>() { return FLT_EPSILON; }

// ------------------------------------------------------------------ QR
// Householder QR of the column-major m x k matrix T (leading dimension LD)
// in place: reflector c maps x = T(c:m, c) to beta e_1 with
// beta = -(x_0/|x_0|) ||x||, u = x - beta e_1.  On return rows 0..k-1 hold R.
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
    R ax = sqrt(sc_abs2(alpha));
    S ph = ax > R(0) ? (R(1) / ax) * alpha : sc_real_s<S>(R(1));
    S beta = -(sqrt(nrm2) * ph);
    S u0 = alpha - beta;
    R uu = nrm2 - sc_abs2(alpha) + sc_abs2(u0);
    R two_uu = R(2) / uu;
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

// ------------------------------------------------------------------ Jacobi
// Parallel one-sided (Hestenes) Jacobi on the p x q matrix G (leading
// dimension LDG): G V has orthogonal columns, V (q x q, leading dimension
// LDV) unitary.  Round-robin ordering: in each of the qq-1 rounds of a sweep
// (qq = q rounded up to even) the columns split into qq/2 disjoint pairs, one
// group of LPP lanes per pair.  A pair is rotated when |g_a^* g_b| > tol
// sqrt(|g_a|^2 |g_b|^2), tol = p eps, and neither column is below
// p eps ||G||_F.  Returns sweeps used, or -1 at the sweep limit.
template <class S, int LDG, int LDV, int QMAX>
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
  const R tiny = tol * tol * nf2;
  __syncwarp();
  if (q < 2) return 1;
  const int qq = (q + 1) & ~1;
  const int npairs = qq / 2;
  const int grp = lane / LPP, sub = lane % LPP;
  for (int sweep = 1; sweep <= kMaxSweeps; ++sweep) {
    bool rotated = false;
    for (int rnd = 0; rnd < qq - 1; ++rnd) {
      for (int pr0 = 0; pr0 < npairs; pr0 += kGroups) {
        int pr = pr0 + grp;
        int a = -1, b = -1;
        if (pr < npairs) {
          int pa = pr, pb = qq - 1 - pr;
          a = pa == 0 ? 0 : 1 + (pa - 1 + rnd) % (qq - 1);
          b = 1 + (pb - 1 + rnd) % (qq - 1);
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
        R ag = sqrt(sc_abs2(ga));
        bool rot = act && al > tiny && be > tiny && ag != R(0) && ag > tol * sqrt(al * be);
        if (rot) {
          rotated = true;
          S eph = (R(1) / ag) * sc_conj(ga);
          R zeta = (be - al) / (R(2) * ag);
          R t = (zeta >= R(0) ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
          R cs = R(1) / sqrt(R(1) + t * t), sn = cs * t;
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
  }
  return -1;
}

// column norms of G (p x q): sigma[c]
template <class S, int LDG>
__device__ void warp_col_norms(const S* G, int p, int q, RealOf<S>* sigma, int lane) {
  using R = RealOf<S>;
  for (int c = lane; c < q; c += DIAF_WARP) {
    R s = R(0);
    for (int i = 0; i < p; ++i) s += sc_abs2(G[i + c * LDG]);
    sigma[c] = sqrt(s);
  }
  __syncwarp();
}

// ------------------------------------------------------------------ kernel
template <class S, int KMAX, int MMAX>
struct WarpLayout {
  static constexpr int kTile = MMAX * KMAX;
  static constexpr size_t raw() {
    return sizeof(S) * (2 * kTile + 2 * KMAX * KMAX + KMAX + MMAX) + sizeof(double) * (MMAX + KMAX) +
           sizeof(int32_t) * (5 * MMAX + 2 * KMAX + 8);
  }
  static constexpr size_t bytes() { return (raw() + 15) / 16 * 16; }  // keeps every warp's slice 16-byte aligned
};

template <class S, int KMAX, int MMAX, int ALG>
__device__ void solve_column_warp(const ColArgs& a, int j, unsigned char* smem, int lane) {
  using R = RealOf<S>;
  using L = WarpLayout<S, KMAX, MMAX>;
  S* Ts = reinterpret_cast<S*>(smem);           // original tile, MMAX x KMAX
  S* Tw = Ts + L::kTile;                          // working tile / Q rows / Q_I
  S* Rs = Tw + L::kTile;                          // R of T, later R-hat (KMAX x KMAX)
  S* Vj = Rs + KMAX * KMAX;                       // Jacobi V
  S* wv = Vj + KMAX * KMAX;                       // w (KMAX)
  S* vv = wv + KMAX;                              // v (MMAX)
  double* hk = reinterpret_cast<double*>(vv + MMAX);  // leverage keys (MMAX)
  R* sig = reinterpret_cast<R*>(hk + MMAX);       // singular values (KMAX)
  int32_t* rs = reinterpret_cast<int32_t*>(hk + MMAX + KMAX);
  int32_t* inI = rs + MMAX;      // per tile row: position in I or -1
  int32_t* pick = inI + MMAX;    // per tile row: picked by the rule
  int32_t* Is = pick + MMAX;     // I_j rows (sorted)
  int32_t* Iloc = Is + MMAX;     // tile row of Is[t] or -1
  int32_t* cst = Iloc + MMAX;    // column starts of J_j in A
  int32_t* coff = cst + KMAX;    // exclusive offsets of the gathered entries
  int32_t* misc = coff + KMAX;   // [0] = jpos

  const int k = a.Wcp[j + 1] - a.Wcp[j];
  const int32_t* J = a.Wri + a.Wcp[j];
  const int m = a.m[j];
  const int l = a.l[j];
  const int me = m > k ? m : k;  // rows of the working tile (zero padded)
  const int32_t* Rj = a.rows + a.Eoff[j];
  const S* Av = reinterpret_cast<const S*>(a.Av);
  uint32_t flags = 0;

  // ---- row set and gather
  for (int r = lane; r < MMAX; r += DIAF_WARP) {
    rs[r] = r < m ? Rj[r] : INT_MAX;
    inI[r] = -1;
    pick[r] = 0;
  }
  for (int i = lane; i < me * k; i += DIAF_WARP) Ts[(i % me) + (i / me) * MMAX] = sc_zero<S>();
  int len = 0;
  if (lane < k) {
    int c = J[lane];
    cst[lane] = a.Acp[c];
    len = a.Acp[c + 1] - a.Acp[c];
  }
  int incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(DIAF_FULL, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane < k) coff[lane] = incl - len;
  const int E = __shfl_sync(DIAF_FULL, incl, 31);
  __syncwarp();
  for (int e = lane; e < E; e += DIAF_WARP) {
    int q = 0;
    while (q + 1 < k && coff[q + 1] <= e) ++q;
    int p = cst[q] + (e - coff[q]);
    int r = lower_bound_i32(rs, m, a.Ari[p]);
    Ts[r + q * MMAX] = Av[p];
  }
  __syncwarp();

  // ---- I_j
  int jpos = -1;
  if (k > 0) {
    // QR of T (copy) -> R
    for (int i = lane; i < me * k; i += DIAF_WARP) Tw[(i % me) + (i / me) * MMAX] = Ts[(i % me) + (i / me) * MMAX];
    __syncwarp();
    warp_householder_qr<S, MMAX>(Tw, me, k, lane);
    for (int i = lane; i < k * k; i += DIAF_WARP) {
      int r = i % k, c = i / k;
      Rs[r + c * KMAX] = (r <= c) ? Tw[r + c * MMAX] : sc_zero<S>();
    }
    __syncwarp();
  }
  // pivot threshold for R (rank guard, 1e-14 of the largest |R_ii|)
  R rdmax = R(0);
  for (int c = lane; c < k; c += DIAF_WARP) rdmax = dmax(rdmax, (R)sqrt(sc_abs2(Rs[c + c * KMAX])));
  rdmax = warp_max(rdmax);
  const R piv = R(1e-14) * rdmax;
  if (k > 0 && (a.rule != DIAF_RULE_FIXED || ALG == DIAF_ALG_Q)) {
    // Q = T R^-1 row by row (lane r owns tile row r); h_r = ||Q(r,:)||^2
    for (int r = lane; r < m; r += DIAF_WARP) {
      R h = R(0);
      for (int c = 0; c < k; ++c) {
        S acc = Ts[r + c * MMAX];
        for (int p2 = 0; p2 < c; ++p2) acc -= Tw[r + p2 * MMAX] * Rs[p2 + c * KMAX];
        S d = Rs[c + c * KMAX];
        R ad2 = sc_abs2(d);
        S z = sc_zero<S>();
        if (sqrt(ad2) > piv) z = (R(1) / ad2) * (acc * sc_conj(d));
        Tw[r + c * MMAX] = z;
        h += sc_abs2(z);
      }
      hk[r] = (double)h;
    }
    __syncwarp();
  }
  if (a.rule == DIAF_RULE_FIXED) {
    const int32_t* Vf = a.Vfri + a.Vfcp[j];
    for (int t = lane; t < l; t += DIAF_WARP) {
      int row = Vf[t];
      int r = lower_bound_i32(rs, m, row);
      int loc = (r < m && rs[r] == row) ? r : -1;
      Is[t] = row;
      Iloc[t] = loc;
      if (loc >= 0) inI[loc] = t;
      if (row == j) misc[0] = t;
    }
    if (lane == 0) {
      bool has = false;
      for (int t = 0; t < l; ++t) has |= (Vf[t] == j);
      if (!has) misc[0] = -1;
    }
    __syncwarp();
    jpos = misc[0];
  } else {
    const int s = l - 1;
    for (int t = 0; t < s; ++t) {
      double hm = -DBL_MAX;
      for (int r = lane; r < m; r += DIAF_WARP)
        if (!pick[r] && admissible_row(a.rule, rs[r], j)) hm = dmax(hm, hk[r]);
      hm = warp_max(hm);
      const double thr = hm - a.tie_tol;
      int best = INT_MAX;
      for (int r = lane; r < m; r += DIAF_WARP)
        if (!pick[r] && admissible_row(a.rule, rs[r], j) && hk[r] >= thr) best = dmin(best, r);
      best = warp_min(best);
      if (lane == 0 && best < m) pick[best] = 1;
      __syncwarp();
    }
    // compaction of {picked} U {j} in row order
    int cnt = 0;
    for (int r0 = 0; r0 < m; r0 += DIAF_WARP) {
      int r = r0 + lane;
      bool f = r < m && (pick[r] || rs[r] == j);
      unsigned b = __ballot_sync(DIAF_FULL, f);
      if (f) {
        int pos = cnt + __popc(b & ((1u << lane) - 1u));
        Is[pos] = rs[r];
        Iloc[pos] = r;
      }
      cnt += __popc(b);
    }
    __syncwarp();
    if (!a.jin[j]) {  // j is not a tile row: insert it (its tile row is zero)
      if (lane == 0) {
        int pos = 0;
        while (pos < cnt && Is[pos] < j) ++pos;
        for (int t = cnt; t > pos; --t) { Is[t] = Is[t - 1]; Iloc[t] = Iloc[t - 1]; }
        Is[pos] = j;
        Iloc[pos] = -1;
      }
      __syncwarp();
    }
    for (int t = lane; t < l; t += DIAF_WARP) {
      if (Iloc[t] >= 0) inI[Iloc[t]] = t;
      if (Is[t] == j) misc[0] = t;
    }
    __syncwarp();
    jpos = misc[0];
  }

  for (int t = lane; t < l; t += DIAF_WARP) vv[t] = sc_zero<S>();
  for (int q = lane; q < k; q += DIAF_WARP) wv[q] = sc_zero<S>();
  __syncwarp();

  if (k == 0) {
    flags |= DIAF_FLAG_EMPTY;
    if (ALG == DIAF_ALG_Q) {
      if (lane == 0) vv[jpos >= 0 ? jpos : 0] = sc_real_s<S>(R(1));
      flags |= DIAF_FLAG_DEGENERATE;
    } else {
      flags |= DIAF_FLAG_RANK_DEFICIENT;
    }
    __syncwarp();
  } else if (ALG == DIAF_ALG_S) {
    // ---- DIAF-S: QR of the tile without the I_j rows, Jacobi SVD of R-hat
    for (int i = lane; i < me * k; i += DIAF_WARP) {
      int r = i % me, c = i / me;
      Tw[r + c * MMAX] = (r < m && inI[r] >= 0) ? sc_zero<S>() : Ts[r + c * MMAX];
    }
    __syncwarp();
    warp_householder_qr<S, MMAX>(Tw, me, k, lane);
    for (int i = lane; i < k * k; i += DIAF_WARP) {
      int r = i % k, c = i / k;
      Rs[r + c * KMAX] = (r <= c) ? Tw[r + c * MMAX] : sc_zero<S>();
    }
    __syncwarp();
    int sw = warp_jacobi<S, KMAX, KMAX, KMAX>(Rs, k, k, Vj, lane);
    if (sw < 0) flags |= DIAF_FLAG_JACOBI_NOCONV;
    warp_col_norms<S, KMAX>(Rs, k, k, sig, lane);
    int imin = 0;
    R smin = sig[0], smax = sig[0];
    for (int c = 1; c < k; ++c) {
      if (sig[c] < smin) { smin = sig[c]; imin = c; }
      smax = dmax(smax, sig[c]);
    }
    R snext = R(INFINITY);
    for (int c = 0; c < k; ++c) if (c != imin) snext = dmin(snext, sig[c]);
    int inrows = 0;
    for (int t = 0; t < l; ++t) inrows += (Iloc[t] >= 0);
    if (smin <= R(1e-14) * smax || m - inrows < k) flags |= DIAF_FLAG_RANK_DEFICIENT;
    if (k > 1 && (snext - smin) <= R(1e-6) * smax) flags |= DIAF_FLAG_DEGENERATE;
    for (int q = lane; q < k; q += DIAF_WARP) wv[q] = Vj[q + imin * KMAX];
    __syncwarp();
    for (int t = lane; t < l; t += DIAF_WARP) {
      S s = sc_zero<S>();
      int r = Iloc[t];
      if (r >= 0)
        for (int q = 0; q < k; ++q) s += Ts[r + q * MMAX] * wv[q];
      vv[t] = s;
    }
    __syncwarp();
  } else {
    // ---- DIAF-Q: Q_I = rows I_j of Q (compacted in place to the top of Tw)
    for (int c = 0; c < k; ++c) {
      S tmp[MMAX / DIAF_WARP + 1];
      int nn = 0;
      for (int t = lane; t < l; t += DIAF_WARP) {
        int r = Iloc[t];
        tmp[nn++] = r >= 0 ? Tw[r + c * MMAX] : sc_zero<S>();
      }
      __syncwarp();
      nn = 0;
      for (int t = lane; t < l; t += DIAF_WARP) Tw[t + c * MMAX] = tmp[nn++];
      __syncwarp();
    }
    int sw = warp_jacobi<S, MMAX, KMAX, KMAX>(Tw, l, k, Vj, lane);
    if (sw < 0) flags |= DIAF_FLAG_JACOBI_NOCONV;
    warp_col_norms<S, MMAX>(Tw, l, k, sig, lane);
    int imax = 0;
    R smax = sig[0];
    for (int c = 1; c < k; ++c) if (sig[c] > smax) { smax = sig[c]; imax = c; }
    R snext = R(0);
    for (int c = 0; c < k; ++c) if (c != imax) snext = dmax(snext, sig[c]);
    if (smax == R(0) || (k > 1 && (smax - snext) <= R(1e-6) * smax)) flags |= DIAF_FLAG_DEGENERATE;
    if (smax > R(0)) {
      for (int t = lane; t < l; t += DIAF_WARP) vv[t] = (R(1) / smax) * Tw[t + imax * MMAX];
    } else if (lane == 0) {
      vv[jpos >= 0 ? jpos : 0] = sc_real_s<S>(R(1));
    }
    __syncwarp();
    // w = sigma R^-1 u  (R w = Q^* v, eq. condwj)
    if (lane == 0) {
      bool rd = false;
      for (int c = k - 1; c >= 0; --c) {
        S s = smax * Vj[c + imax * KMAX];
        for (int t = c + 1; t < k; ++t) s -= Rs[c + t * KMAX] * wv[t];
        S d = Rs[c + c * KMAX];
        R ad2 = sc_abs2(d);
        if (sqrt(ad2) <= piv) { rd = true; wv[c] = sc_zero<S>(); }
        else wv[c] = (R(1) / ad2) * (s * sc_conj(d));
      }
      if (rd) misc[1] = 1; else misc[1] = 0;
    }
    __syncwarp();
    if (misc[1]) flags |= DIAF_FLAG_RANK_DEFICIENT;
  }

  // ---- phase: v_jj real and >= 0
  if (k > 0 || ALG == DIAF_ALG_Q) {
    S ph = sc_real_s<S>(R(1));
    R vjj = jpos >= 0 ? (R)sqrt(sc_abs2(vv[jpos])) : R(0);
    R vn2 = R(0);
    for (int t = 0; t < l; ++t) vn2 += sc_abs2(vv[t]);
    // v_jj counts as zero below the rounding level of the column
    if (jpos >= 0 && vjj > R(64) * eps_of<R>() * sqrt(vn2)) {
      ph = (R(1) / vjj) * sc_conj(vv[jpos]);
    } else {
      flags |= DIAF_FLAG_VJJ_ZERO;
      R amx = R(0);
      int imx = -1;
      for (int q = 0; q < k; ++q) {
        R aq = sqrt(sc_abs2(wv[q]));
        if (aq > amx) { amx = aq; imx = q; }
      }
      if (imx >= 0) ph = (R(1) / amx) * sc_conj(wv[imx]);
    }
    __syncwarp();
    for (int q = lane; q < k; q += DIAF_WARP) wv[q] = ph * wv[q];
    for (int t = lane; t < l; t += DIAF_WARP) vv[t] = ph * vv[t];
    __syncwarp();
  }

  // ---- residual ||A_j w - v||
  R r2 = R(0);
  for (int r = lane; r < m; r += DIAF_WARP) {
    S s = sc_zero<S>();
    for (int q = 0; q < k; ++q) s += Ts[r + q * MMAX] * wv[q];
    if (inI[r] >= 0) s -= vv[inI[r]];
    r2 += sc_abs2(s);
  }
  for (int t = lane; t < l; t += DIAF_WARP)
    if (Iloc[t] < 0) r2 += sc_abs2(vv[t]);
  r2 = warp_sum(r2);
  const double resj = sqrt((double)r2);

  bool finite = isfinite(resj);
  for (int q = lane; q < k; q += DIAF_WARP) finite &= isfinite(sc_real(wv[q])) && isfinite(sc_imag(wv[q]));
  for (int t = lane; t < l; t += DIAF_WARP) finite &= isfinite(sc_real(vv[t])) && isfinite(sc_imag(vv[t]));
  finite = __all_sync(DIAF_FULL, finite);
  if (!finite) flags |= DIAF_FLAG_NONFINITE;

  // ---- scatter
  S* Wout = reinterpret_cast<S*>(a.Wv) + a.Wcp[j];
  for (int q = lane; q < k; q += DIAF_WARP) Wout[q] = wv[q];
  const int v0 = a.Vcp[j];
  S* Vout = reinterpret_cast<S*>(a.Vv) + v0;
  for (int t = lane; t < l; t += DIAF_WARP) {
    a.Vri[v0 + t] = Is[t];
    Vout[t] = vv[t];
  }
  if (lane == 0) {
    a.res[j] = resj;
    a.flags[j] = flags;
  }
  __syncwarp();
}

template <class S, int KMAX, int MMAX, int ALG>
__global__ void column_warp_kernel(ColArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* smem = smem_raw + warp * WarpLayout<S, KMAX, MMAX>::bytes();
  const int count = *a.list_count;
  while (true) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(a.work_counter, 1);
    idx = __shfl_sync(DIAF_FULL, idx, 0);
    if (idx >= count) break;
    solve_column_warp<S, KMAX, MMAX, ALG>(a, a.list[idx], smem, lane);
  }
}
