// Fused per-column kernel of the columnwise setup, FP64 (or complex128)
// throughout, one warp per column, the tile in shared memory.  For column j:
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
// The same kernel finishes the columns the mixed-precision kernel hands back.
#pragma once

#include <limits>

#include "warp_la.cuh"

// Column-scaled conditioning estimate of an upper R whose columns came from a
// tile with column norms cn: max_c cn_c / |R_cc| (1 for orthogonal columns).
constexpr float kMixedKappaMax = 300.0f;
// Bound on an FP32 leverage key's error: delta = kMixedDeltaScale (m + k) eps_32 kappa
// (the backward error of the FP32 QR and row solves, amplified by the column-scaled
// conditioning); a decision within 2 delta of its threshold is left to the FP64 kernel.
#ifndef DIAF_MIXED_DELTA_SCALE
#define DIAF_MIXED_DELTA_SCALE 1.0
#endif
constexpr double kMixedDeltaScale = DIAF_MIXED_DELTA_SCALE;
// A factor taken from a Gram matrix in FP32 carries kappa^2 instead of kappa:
// the Gram paths of the mixed kernels are used only up to this column-scaled
// kappa (the Householder QR otherwise).
constexpr float kGramKappaMax = 30.0f;

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
  const int32_t* blk;         // DIAF_RULE_BLOCK: block of every row
  double stab_tol;            // stabilised DIAF-Q: trigger |v_jj| < stab_tol (0: off)
  double stab_r;              // stabilised DIAF-Q: imposed v_jj before scaling to unit norm
  const int32_t* list;        // bucket's columns
  const int32_t* list_count;  // device count of the list
  int32_t* work_counter;      // zeroed before launch
  uint32_t extra_flags;       // OR-ed into every column's flags (FP64 fallback of the mixed form)
  int32_t* fb_list;           // mixed form: columns handed to the FP64 kernel
  int32_t* fb_count;
  void* Wv;
  int32_t* Vri;
  void* Vv;
  double* res;
  uint32_t* flags;
  uint32_t* status;
  unsigned long long* phase;  // profiling builds only: per-phase cycle counters (or null)
  void* tile_scratch;         // mixed warp kernels: one FP64 tile per resident warp (global memory)
  // V's structure streamed to the host during the numeric pass (or all null / 0):
  int list_desc;              // 1: the lists are taken from their end (descending columns, upper V)
  int32_t* Hri;               // host-mapped copy of Vri, written as each column becomes final
  uint32_t* Hgen;             // host-mapped word per column: set to gen after the column's rows
  uint32_t gen;
};

// Column of the idx-th list entry taken by a persistent kernel: from the
// list's end when the host walks V's columns in descending order.
__device__ __forceinline__ int list_at(const ColArgs& a, int count, int idx) {
  return a.list[a.list_desc ? count - 1 - idx : idx];
}

// ------------------------------------------------------------------ shared steps
// Per-warp index scratch for the parts common to both kernels.
struct ColumnIdx {
  int32_t* rs;    // R_j (MMAX), INT_MAX past m
  int32_t* inI;   // per tile row: position in I_j or -1
  int32_t* pick;  // per tile row: picked by the rule
  int32_t* Is;    // I_j rows (sorted)
  int32_t* Iloc;  // tile row of Is[t] or -1
  int32_t* cst;   // column starts of J_j in A (KMAX)
  int32_t* coff;  // exclusive offsets of the gathered entries (KMAX)
  int32_t* misc;  // [0] = position of j in I_j
};
template <int KMAX, int MMAX>
constexpr size_t idx_bytes() { return sizeof(int32_t) * (5 * MMAX + 2 * KMAX + 8); }

template <int KMAX, int MMAX>
__device__ ColumnIdx carve_idx(int32_t* base) {
  ColumnIdx ix;
  ix.rs = base;
  ix.inI = ix.rs + MMAX;
  ix.pick = ix.inI + MMAX;
  ix.Is = ix.pick + MMAX;
  ix.Iloc = ix.Is + MMAX;
  ix.cst = ix.Iloc + MMAX;
  ix.coff = ix.cst + KMAX;
  ix.misc = ix.coff + KMAX;
  return ix;
}

// Loads R_j and gathers T = A(R_j, J_j) (zero padded to me rows) into Ts.
template <class SD, int KMAX, int MMAX, int LDT>
__device__ void gather_tile(const ColArgs& a, int j, int k, int m, int me, SD* Ts, const ColumnIdx& ix, int lane) {
  const int32_t* Rj = a.rows + a.Eoff[j];
  const int32_t* J = a.Wri + a.Wcp[j];
  const SD* Av = reinterpret_cast<const SD*>(a.Av);
  for (int r = lane; r < MMAX; r += DIAF_WARP) {
    ix.rs[r] = r < m ? Rj[r] : INT_MAX;
    ix.inI[r] = -1;
    ix.pick[r] = 0;
  }
  for (int i = lane; i < me * k; i += DIAF_WARP) Ts[(i % me) + (i / me) * LDT] = sc_zero<SD>();
  int len = 0;
  if (lane < k) {
    int c = J[lane];
    ix.cst[lane] = a.Acp[c];
    len = a.Acp[c + 1] - a.Acp[c];
  }
  int incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(DIAF_FULL, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane < k) ix.coff[lane] = incl - len;
  const int E = __shfl_sync(DIAF_FULL, incl, 31);
  __syncwarp();
  for (int e = lane; e < E; e += DIAF_WARP) {
    int q = 0;
    while (q + 1 < k && ix.coff[q + 1] <= e) ++q;
    int p = ix.cst[q] + (e - ix.coff[q]);
    int r = lower_bound_i32(ix.rs, m, a.Ari[p]);
    Ts[r + q * LDT] = Av[p];
  }
  __syncwarp();
}

// Greedy selection of s admissible rows by key hk (Sec. 3.1 with ties within
// tau to the lower row).  Returns the smallest distance of any remaining
// candidate's key to a pick threshold, the candidate holding the maximum
// excluded (it passes the threshold by construction): how close a decision
// came to flipping when the keys carry an error.
// K: the key type (double in the FP64 kernels; float in the mixed ones, whose
// keys are FP32 values and are compared as such).
template <class K>
__device__ inline double select_rows_greedy(const int32_t* rs, const K* hk, int32_t* pick, int m, int rule,
                                            int j, int s, double tau, int lane, const int32_t* blk) {
  K margin = std::numeric_limits<K>::max();
  for (int r = lane; r < m; r += DIAF_WARP) pick[r] = 0;
  __syncwarp();
  for (int t = 0; t < s; ++t) {
    K hm = -std::numeric_limits<K>::max();
    for (int r = lane; r < m; r += DIAF_WARP)
      if (!pick[r] && admissible_row(rule, rs[r], j, blk)) hm = dmax(hm, hk[r]);
    hm = warp_max(hm);
    int rmax = INT_MAX;
    for (int r = lane; r < m; r += DIAF_WARP)
      if (!pick[r] && admissible_row(rule, rs[r], j, blk) && hk[r] == hm) rmax = dmin(rmax, r);
    rmax = warp_min(rmax);
    const K thr = hm - K(tau);
    int best = INT_MAX;
    for (int r = lane; r < m; r += DIAF_WARP)
      if (!pick[r] && admissible_row(rule, rs[r], j, blk)) {
        if (r != rmax) margin = dmin(margin, (K)fabs(hk[r] - thr));
        if (hk[r] >= thr) best = dmin(best, r);
      }
    best = warp_min(best);
    if (best == INT_MAX) {  // no key reaches the threshold (non-finite keys): the lowest remaining admissible row
      for (int r = lane; r < m; r += DIAF_WARP)
        if (!pick[r] && admissible_row(rule, rs[r], j, blk)) best = dmin(best, r);
      best = warp_min(best);
    }
    if (lane == 0 && best < m) pick[best] = 1;
    __syncwarp();
  }
  return (double)warp_min(margin);
}

// I_j from the picks (rule) or the fixed pattern; fills Is, Iloc, inI; returns
// the position of j in I_j (-1 if absent).
__device__ inline int build_I(const ColArgs& a, int j, int m, int l, const ColumnIdx& ix, int lane) {
  if (lane == 0) ix.misc[0] = -1;
  __syncwarp();
  if (a.rule == DIAF_RULE_FIXED) {
    const int32_t* Vf = a.Vfri + a.Vfcp[j];
    for (int t = lane; t < l; t += DIAF_WARP) {
      int row = Vf[t];
      int r = lower_bound_i32(ix.rs, m, row);
      int loc = (r < m && ix.rs[r] == row) ? r : -1;
      ix.Is[t] = row;
      ix.Iloc[t] = loc;
      if (loc >= 0) ix.inI[loc] = t;
      if (row == j) ix.misc[0] = t;
    }
    __syncwarp();
    return ix.misc[0];
  }
  int cnt = 0;
  for (int r0 = 0; r0 < m; r0 += DIAF_WARP) {
    int r = r0 + lane;
    bool f = r < m && (ix.pick[r] || ix.rs[r] == j);
    unsigned b = __ballot_sync(DIAF_FULL, f);
    if (f) {
      int pos = cnt + __popc(b & ((1u << lane) - 1u));
      ix.Is[pos] = ix.rs[r];
      ix.Iloc[pos] = r;
    }
    cnt += __popc(b);
  }
  __syncwarp();
  if (!a.jin[j]) {  // j is not a tile row: insert it (its tile row is zero)
    if (lane == 0) {
      int pos = 0;
      while (pos < cnt && ix.Is[pos] < j) ++pos;
      for (int t = cnt; t > pos; --t) { ix.Is[t] = ix.Is[t - 1]; ix.Iloc[t] = ix.Iloc[t - 1]; }
      ix.Is[pos] = j;
      ix.Iloc[pos] = -1;
    }
    __syncwarp();
  }
  for (int t = lane; t < l; t += DIAF_WARP) {
    if (ix.Iloc[t] >= 0) ix.inI[ix.Iloc[t]] = t;
    if (ix.Is[t] == j) ix.misc[0] = t;
  }
  __syncwarp();
  return ix.misc[0];
}

// Phase (v_jj real >= 0, else the largest |w_q| real), residual
// ||A_j w - v||, finiteness, and the scatter of column j.
template <class SD, int LDT>
__device__ void finish_column(const ColArgs& a, int j, int k, int m, int l, int jpos, const SD* Ts, SD* wv, SD* vv,
                              const ColumnIdx& ix, uint32_t flags, bool do_phase, int lane,
                              double rank_thr = -1.0) {
  using R = RealOf<SD>;
  if (do_phase) {
    SD ph = sc_real_s<SD>(R(1));
    const R vjj2 = jpos >= 0 ? sc_abs2(vv[jpos]) : R(0);
    R vn2 = R(0);
    for (int t = 0; t < l; ++t) vn2 += sc_abs2(vv[t]);
    // v_jj counts as zero below the rounding level of the column (|v_jj| <= 64 eps ||v||)
    const R zl = R(64) * eps_of<R>();
    if (jpos >= 0 && vjj2 > zl * zl * vn2) {
      if constexpr (ScalarInfo<SD>::cplx) ph = (R(1) / sqrt(vjj2)) * sc_conj(vv[jpos]);
      else ph = vv[jpos] < R(0) ? sc_real_s<SD>(R(-1)) : sc_real_s<SD>(R(1));  // v_jj / |v_jj|, exactly
    } else {
      flags |= DIAF_FLAG_VJJ_ZERO;
      R amx = R(0);
      int imx = -1;
      for (int q = 0; q < k; ++q) {
        R aq = sc_abs(wv[q]);
        if (aq > amx) { amx = aq; imx = q; }
      }
      if (imx >= 0) ph = (R(1) / amx) * sc_conj(wv[imx]);
    }
    __syncwarp();
    for (int q = lane; q < k; q += DIAF_WARP) wv[q] = ph * wv[q];
    for (int t = lane; t < l; t += DIAF_WARP) vv[t] = ph * vv[t];
    __syncwarp();
  }
  R r2 = R(0);
  for (int r = lane; r < m; r += DIAF_WARP) {
    SD s = sc_zero<SD>();
    for (int q = 0; q < k; ++q) s += Ts[r + q * LDT] * wv[q];
    if (ix.inI[r] >= 0) s -= vv[ix.inI[r]];
    r2 += sc_abs2(s);
  }
  for (int t = lane; t < l; t += DIAF_WARP)
    if (ix.Iloc[t] < 0) r2 += sc_abs2(vv[t]);
  r2 = warp_sum(r2);
  const double resj = sqrt((double)r2);
  if (resj <= rank_thr) flags |= DIAF_FLAG_RANK_DEFICIENT;  // DIAF-S: res = ||A-hat w|| = sigma_min
  bool finite = isfinite(resj);
  for (int q = lane; q < k; q += DIAF_WARP) finite &= isfinite(sc_real(wv[q])) && isfinite(sc_imag(wv[q]));
  for (int t = lane; t < l; t += DIAF_WARP) finite &= isfinite(sc_real(vv[t])) && isfinite(sc_imag(vv[t]));
  finite = __all_sync(DIAF_FULL, finite);
  if (!finite) flags |= DIAF_FLAG_NONFINITE;
  SD* Wout = reinterpret_cast<SD*>(a.Wv) + a.Wcp[j];
  for (int q = lane; q < k; q += DIAF_WARP) Wout[q] = wv[q];
  const int v0 = a.Vcp[j];
  SD* Vout = reinterpret_cast<SD*>(a.Vv) + v0;
  for (int t = lane; t < l; t += DIAF_WARP) {
    a.Vri[v0 + t] = ix.Is[t];
    Vout[t] = vv[t];
  }
  if (lane == 0) {
    a.res[j] = resj;
    a.flags[j] = flags | a.extra_flags;
  }
  if (a.Hri) {  // the final I_j to the host: rows, then the column's word
    for (int t = lane; t < l; t += DIAF_WARP) a.Hri[v0 + t] = ix.Is[t];
    __threadfence_system();
    __syncwarp();
    if (lane == 0) store_release_sys(a.Hgen + j, a.gen);
  }
  __syncwarp();
}

// Compacts rows Iloc[0..l) of the columns 0..k-1 of Tw (leading dimension LD)
// to its top l rows (a missing row gives zeros).  Iloc is increasing, so
// reading every value of a column before writing it is enough.
template <class S, int LD>
__device__ void compact_rows(S* Tw, const int32_t* Iloc, int l, int k, int lane) {
  for (int c = 0; c < k; ++c) {
    S tmp[LD / DIAF_WARP + 1];
    int nn = 0;
    for (int t = lane; t < l; t += DIAF_WARP) {
      int r = Iloc[t];
      tmp[nn++] = r >= 0 ? Tw[r + c * LD] : sc_zero<S>();
    }
    __syncwarp();
    nn = 0;
    for (int t = lane; t < l; t += DIAF_WARP) Tw[t + c * LD] = tmp[nn++];
    __syncwarp();
  }
}

// ------------------------------------------------------------------ FP64 kernel
template <class S, int KMAX, int MMAX>
struct WarpLayout {
  static constexpr int LDT = MMAX + 1;  // odd leading dimensions: no bank conflicts between columns
  static constexpr int KP = KMAX + 1;
  static constexpr int kTile = LDT * KMAX;
  static constexpr size_t raw() {
    return sizeof(S) * (2 * kTile + 2 * KP * KMAX + 2 * KMAX + MMAX) + sizeof(double) * (MMAX + KMAX) +
           idx_bytes<KMAX, MMAX>();
  }
  static constexpr size_t bytes() { return (raw() + 15) / 16 * 16; }  // keeps every warp's slice 16-byte aligned
};

// Stabilised DIAF-Q (Sec. 3.2).  On entry Tw holds Q_I V1 (the rows I_j of Q
// after the first Jacobi, l x k) and vv the unit v_j of eq. nocond with
// |v_jj| < stab_tol.  The j-th component is imposed as r and the rest is the
// top singular vector z of M_hat = Q_I'^* (I' = I_j without j) with the phase
// e^{i theta}, theta = arg of the first component of U_hat^* p, p = Q(j,:)^*.
// Rotating Q_I by V1 changes neither z nor U_hat^* p: B = Q_I' V1 = Z S Y^*
// gives M_hat = (V1 Y) S Z^*, so z = B Y(:,1)/s_1 and U_hat(:,1)^* p =
// conj(sum_c Y(c,1) q_c) with q = row j of Q_I V1.  v_j = (r e_j + e^{i theta}
// z) / sqrt(r^2 + 1); the lane's entry of Q_I^* v_j = R^-* T_I^* v_j is
// returned, ready for the back substitution of eq. condwj.
template <class S, int LDT, int KP, int KMAX>
__device__ S stabilise_q_warp(const ColArgs& a, const S* Ts, S* Tw, const S* Rs, const S* rinv, S* Vj, S* wv,
                              S* vv, double* sig, const ColumnIdx& ix, int k, int l, int jpos, uint32_t& flags,
                              int lane) {
  using R = RealOf<S>;
  for (int q = lane; q < k; q += DIAF_WARP) wv[q] = Tw[jpos + q * LDT];  // q = row j of Q_I V1
  __syncwarp();
  for (int c = 0; c < k; ++c) {  // drop row jpos: rows below move up by one
    S tmp[(LDT + DIAF_WARP - 1) / DIAF_WARP];
    int nn = 0;
    for (int t = jpos + lane; t < l - 1; t += DIAF_WARP) tmp[nn++] = Tw[t + 1 + c * LDT];
    __syncwarp();
    nn = 0;
    for (int t = jpos + lane; t < l - 1; t += DIAF_WARP) Tw[t + c * LDT] = tmp[nn++];
    __syncwarp();
  }
  const int lh = l - 1;
  if (warp_jacobi<S, LDT, KP, KMAX>(Tw, lh, k, Vj, lane) < 0) flags |= DIAF_FLAG_JACOBI_NOCONV;
  warp_col_norms<S, LDT>(Tw, lh, k, sig, lane);
  int i1 = 0;
  double s1 = sig[0];
  for (int c = 1; c < k; ++c) if (sig[c] > s1) { s1 = sig[c]; i1 = c; }
  double s2 = 0.0;
  for (int c = 0; c < k; ++c) if (c != i1) s2 = dmax(s2, sig[c]);
  flags &= ~DIAF_FLAG_DEGENERATE;  // now describes the stabilised problem
  if (s1 == 0.0 || (lh > 1 && k > 1 && (s1 - s2) <= 1e-6 * s1)) flags |= DIAF_FLAG_DEGENERATE;
  S pt = sc_zero<S>();
  R pn = R(0);
  for (int q = lane; q < k; q += DIAF_WARP) {
    pt += Vj[q + i1 * KP] * wv[q];
    pn += sc_abs2(wv[q]);
  }
  pt = sc_conj(warp_sum(pt));
  pn = warp_sum(pn);
  const R apt = sc_abs(pt);
  if (!(apt > R(1e-10) * sqrt(pn))) flags |= DIAF_FLAG_DEGENERATE;  // any theta will do; theta = 0
  const S eth = apt > R(0) ? (R(1) / apt) * pt : sc_real_s<S>(R(1));
  const R r = a.stab_r > 0.0 ? R(a.stab_r) : R(2);
  const R scl = R(1) / sqrt(r * r + R(1));
  const R zs = s1 > 0.0 ? scl / R(s1) : R(0);
  for (int u = lane; u < lh; u += DIAF_WARP) vv[u < jpos ? u : u + 1] = (zs * eth) * Tw[u + i1 * LDT];
  if (lane == 0) vv[jpos] = sc_real_s<S>(r * scl);
  __syncwarp();
  // Q_I^* v = R^-* T_I^* v
  S y = sc_zero<S>();
  if (lane < k)
    for (int t = 0; t < l; ++t) {
      const int rr = ix.Iloc[t];
      if (rr >= 0) y += sc_conj(Ts[rr + lane * LDT]) * vv[t];
    }
  for (int c = 0; c < k; ++c) {  // forward substitution R^* x = y
    S uc = shfl_idx(y * sc_conj(rinv[c]), c);
    if (lane > c && lane < k) y -= sc_conj(Rs[c + lane * KP]) * uc;
    if (lane == c) y = uc;
  }
  flags |= DIAF_FLAG_STABILISED;
  return y;
}

template <class S, int KMAX, int MMAX, int ALG>
__device__ void solve_column_warp(const ColArgs& a, int j, unsigned char* smem, int lane) {
  using R = RealOf<S>;
  using L = WarpLayout<S, KMAX, MMAX>;
  constexpr int LDT = L::LDT, KP = L::KP;
  S* Ts = reinterpret_cast<S*>(smem);  // original tile, LDT x KMAX
  S* Tw = Ts + L::kTile;               // working tile / Q rows / Q_I
  S* Rs = Tw + L::kTile;               // R of T, later R-hat (KP x KMAX)
  S* Vj = Rs + KP * KMAX;              // Jacobi V
  S* wv = Vj + KP * KMAX;              // w (KMAX)
  S* rinv = wv + KMAX;                 // reciprocal diagonal (KMAX)
  S* vv = rinv + KMAX;                 // v (MMAX)
  double* hk = reinterpret_cast<double*>(vv + MMAX);  // keys (MMAX)
  double* sig = hk + MMAX;                            // singular values (KMAX)
  ColumnIdx ix = carve_idx<KMAX, MMAX>(reinterpret_cast<int32_t*>(sig + KMAX));

  const int k = a.Wcp[j + 1] - a.Wcp[j];
  const int m = a.m[j];
  const int l = a.l[j];
  const int me = m > k ? m : k;  // rows of the working tile (zero padded)
  uint32_t flags = 0;

  gather_tile<S, KMAX, MMAX, LDT>(a, j, k, m, me, Ts, ix, lane);

  // ---- QR of T, keys, I_j
  if (k > 0) {
    for (int i = lane; i < me * k; i += DIAF_WARP) Tw[(i % me) + (i / me) * LDT] = Ts[(i % me) + (i / me) * LDT];
    __syncwarp();
    warp_householder_qr_rs<S, LDT, KMAX, MMAX / DIAF_WARP>(Tw, me, k, lane);
    for (int i = lane; i < k * k; i += DIAF_WARP) {
      int r = i % k, c = i / k;
      Rs[r + c * KP] = (r <= c) ? Tw[r + c * LDT] : sc_zero<S>();
    }
    __syncwarp();
  }
  R rdmax = R(0);
  for (int c = lane; c < k; c += DIAF_WARP) rdmax = dmax(rdmax, sc_abs(Rs[c + c * KP]));
  rdmax = warp_max(rdmax);
  const R piv = R(1e-14) * rdmax;
  if (k > 0 && (a.rule != DIAF_RULE_FIXED || ALG == DIAF_ALG_Q))
    warp_leverage_rows<S, S, LDT, KP>(Ts, Rs, Tw, hk, rinv, m, k, piv, lane);
  if (a.rule != DIAF_RULE_FIXED) select_rows_greedy(ix.rs, hk, ix.pick, m, a.rule, j, l - 1, a.tie_tol, lane, a.blk);
  const int jpos = build_I(a, j, m, l, ix, lane);

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
      Tw[r + c * LDT] = (r < m && ix.inI[r] >= 0) ? sc_zero<S>() : Ts[r + c * LDT];
    }
    __syncwarp();
    warp_householder_qr_rs<S, LDT, KMAX, MMAX / DIAF_WARP>(Tw, me, k, lane);
    for (int i = lane; i < k * k; i += DIAF_WARP) {
      int r = i % k, c = i / k;
      Rs[r + c * KP] = (r <= c) ? Tw[r + c * LDT] : sc_zero<S>();
    }
    __syncwarp();
    int sw = warp_jacobi<S, KP, KP, KMAX>(Rs, k, k, Vj, lane);
    if (sw < 0) flags |= DIAF_FLAG_JACOBI_NOCONV;
    warp_col_norms<S, KP>(Rs, k, k, sig, lane);
    int imin = 0;
    double smin = sig[0], smax = sig[0];
    for (int c = 1; c < k; ++c) {
      if (sig[c] < smin) { smin = sig[c]; imin = c; }
      smax = dmax(smax, sig[c]);
    }
    double snext = INFINITY;
    for (int c = 0; c < k; ++c) if (c != imin) snext = dmin(snext, sig[c]);
    int inrows = 0;
    for (int t = 0; t < l; ++t) inrows += (ix.Iloc[t] >= 0);
    if (smin <= 1e-14 * smax || m - inrows < k) flags |= DIAF_FLAG_RANK_DEFICIENT;
    if (k > 1 && (snext - smin) <= 1e-6 * smax) flags |= DIAF_FLAG_DEGENERATE;
    for (int q = lane; q < k; q += DIAF_WARP) wv[q] = Vj[q + imin * KP];
    __syncwarp();
    for (int t = lane; t < l; t += DIAF_WARP) {
      S s = sc_zero<S>();
      int r = ix.Iloc[t];
      if (r >= 0)
        for (int q = 0; q < k; ++q) s += Ts[r + q * LDT] * wv[q];
      vv[t] = s;
    }
    __syncwarp();
  } else {
    // ---- DIAF-Q: Q_I = rows I_j of Q (compacted to the top of Tw)
    compact_rows<S, LDT>(Tw, ix.Iloc, l, k, lane);
    int sw = warp_jacobi<S, LDT, KP, KMAX>(Tw, l, k, Vj, lane);
    if (sw < 0) flags |= DIAF_FLAG_JACOBI_NOCONV;
    warp_col_norms<S, LDT>(Tw, l, k, sig, lane);
    int imax = 0;
    double smax = sig[0];
    for (int c = 1; c < k; ++c) if (sig[c] > smax) { smax = sig[c]; imax = c; }
    double snext = 0.0;
    for (int c = 0; c < k; ++c) if (c != imax) snext = dmax(snext, sig[c]);
    if (smax == 0.0 || (k > 1 && (smax - snext) <= 1e-6 * smax)) flags |= DIAF_FLAG_DEGENERATE;
    if (smax > 0.0) {
      const R inv = R(1) / R(smax);
      for (int t = lane; t < l; t += DIAF_WARP) vv[t] = inv * Tw[t + imax * LDT];
    } else if (lane == 0) {
      vv[jpos >= 0 ? jpos : 0] = sc_real_s<S>(R(1));
    }
    __syncwarp();
    // w = sigma R^-1 u  (R w = Q^* v, eq. condwj); rinv holds R's reciprocal diagonal
    bool rd = false;
    for (int c = lane; c < k; c += DIAF_WARP) rd |= !(sc_abs(Rs[c + c * KP]) > piv);
    rd = __any_sync(DIAF_FULL, rd);
    if (rd) flags |= DIAF_FLAG_RANK_DEFICIENT;
    S x = lane < k ? R(smax) * Vj[lane + imax * KP] : sc_zero<S>();
    if (a.stab_tol > 0.0 && jpos >= 0 && l > 1 && (double)sc_abs(vv[jpos]) < a.stab_tol)
      x = stabilise_q_warp<S, LDT, KP, KMAX>(a, Ts, Tw, Rs, rinv, Vj, wv, vv, sig, ix, k, l, jpos, flags, lane);
    for (int c = k - 1; c >= 0; --c) {
      S yc = shfl_idx(x * rinv[c], c);
      if (lane < c) x -= Rs[lane + c * KP] * yc;
      if (lane == c) x = yc;
    }
    if (lane < k) wv[lane] = x;
    __syncwarp();
  }
  finish_column<S, LDT>(a, j, k, m, l, jpos, Ts, wv, vv, ix, flags, k > 0 || ALG == DIAF_ALG_Q, lane);
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
    solve_column_warp<S, KMAX, MMAX, ALG>(a, list_at(a, count, idx), smem, lane);
  }
}
