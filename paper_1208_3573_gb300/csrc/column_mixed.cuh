// Mixed-precision per-column kernel: the tile is gathered in FP64 (complex128)
// into the warp's slab in global memory and factorised in FP32 (complex64):
// Householder QR (tile rows in registers for tiles of up to 32 x 16, in
// shared memory otherwise), leverage keys and the one-sided Jacobi SVD; then
// (w_j, v_j) are refined in FP64 against the FP64 tile and the residual
// ||A w - v|| is evaluated in FP64.
//
//   DIAF-S: the FP32 Jacobi gives R-hat V = U diag(sigma); x0 = V e_min.
//     With H = A-hat^* A-hat taken from the FP64 tile, V^* H V is diagonal to
//     FP32 accuracy, so one correction in that basis,
//       d = x^* H x / x^* x,  r = H x - d x,
//       x <- x - sum_{i != min} V_i (V_i^* r) / (sigma_i^2 - d),
//     makes x the smallest right singular vector to second order (repeated
//     once when the relative gap is below 1e-2; columns with a gap below 1e-5
//     go to the FP64 kernel).  w = x / ||x||, v = T(I_j,:) w.
//   DIAF-Q: the optimal v of eq. nocond is the top eigenvector of
//     C = Q_I Q_I^* = T_I (T^* T)^-1 T_I^* (C = M_j^* M_j).  The FP32 Jacobi on
//     Q_I gives C's eigenvectors U_c and values s_c^2 and v0 = U_max.  C v is
//     applied in FP64 without forming C: y = (T^* T)^-1 T_I^* v by the FP32 R
//     and corrections with the FP64 residual, C v = T_I y.  (When l < k the
//     Jacobi runs on the smaller Q_I^*.)  With
//     mu = v^* C v / v^* v and r = C v - mu v the same second-order correction
//     as for DIAF-S, v <- v - sum_{c != max} U_c (U_c^* r) / (s_c^2 - mu)
//     + r_perp / mu (r_perp: the part of r in C's null space), repeated until
//     the predicted error is below 1e-11 (at most four times, else the column
//     goes to FP64); w = (T^* T)^-1 T_I^* v, the least-squares solution of
//     eq. condwj, is the y that follows v through the updates.
//
// When a leverage-selection decision is closer to its threshold than the FP32
// key error bound (so I_j could differ from the FP64 choice), the kernel
// recomputes that column's keys in FP64 with the FP64 kernel's own QR and
// leverage routines and selects with those.  A column goes to the FP64 kernel
// instead (appended to fb_list) when the tile is too ill-conditioned for FP32
// factors to drive the refinement, or the refinement cannot converge.
#pragma once

#include "column.cuh"

template <class S> struct DoubleOf;
template <> struct DoubleOf<float> { using T = double; };
template <> struct DoubleOf<Cx<float>> { using T = Cx<double>; };

constexpr int kQRefineMax = 4;  // DIAF-Q: most corrections before the column goes to FP64
constexpr int kRRMax = 8;  // DIAF-Q: sizes of the refinement's scratch (KP x 8 and 2 x 64 scalars)

// R of the real m x k FP32 tile W (leading dimension LDT, one warp) from
// its Gram matrix: lane q accumulates column q of G = W^T W (the other
// columns read as broadcasts), cn receives the column norms, R_s =
// chol(D G D) with D = diag(1 / cn) is formed in place in Rs (leading
// dimension KP, upper triangle; strict lower triangle zeroed), and R = R_s
// D^-1 is kept when the column-scaled kappa max_c 1 / R_s,cc is at most
// kGramKappaMax.  Returns false (uniformly; Rs then undefined, cn the
// column norms) for a zero column, a non-positive pivot or a larger kappa.
template <int KMAX, int LDT, int KP>
__device__ bool warp_gram_cholesky(const float* W, int m, int k, float* Rs, double* cn, int lane) {
  float acc[KMAX];
#pragma unroll
  for (int p = 0; p < KMAX; ++p) acc[p] = 0.0f;
  if (lane < k) {
    const float* wq = W + lane * LDT;
    for (int r = 0; r < m; ++r) {
      const float x = wq[r];
#pragma unroll
      for (int p = 0; p < KMAX; ++p)
        if (p < k) acc[p] = fmaf(x, W[r + p * LDT], acc[p]);
    }
  }
  // the diagonal: lane q holds acc[q]
  float gqq = 0.0f;
#pragma unroll
  for (int p = 0; p < KMAX; ++p)
    if (p == lane) gqq = acc[p];
  const float nq = sqrtf(gqq);
  if (lane < k) cn[lane] = (double)nq;
  const int zero = __any_sync(DIAF_FULL, lane < k && !(nq > 0.0f));
  if (zero) return false;
  const float dq = lane < k ? 1.0f / nq : 0.0f;
  // D G D (upper triangle) into Rs: element (p, q) = acc[p] d_p d_q
#pragma unroll
  for (int p = 0; p < KMAX; ++p) {
    const float dp = __shfl_sync(DIAF_FULL, dq, p);
    if (lane < k && p < k) Rs[p + lane * KP] = p <= lane ? acc[p] * dp * dq : 0.0f;
  }
  __syncwarp();
  // right-looking Cholesky, lane q owns column q
  float kap = 0.0f;
  for (int c = 0; c < k; ++c) {
    const float d = Rs[c + c * KP];
    if (!(d > 0.0f)) return false;  // uniform: every lane read the same pivot
    const float rcc = sqrtf(d), rinv = 1.0f / rcc;
    kap = fmaxf(kap, rinv);
    __syncwarp();
    const float rcq = lane > c && lane < k ? Rs[c + lane * KP] * rinv : 0.0f;
    if (lane == c) Rs[c + c * KP] = rcc;
    if (lane > c && lane < k) Rs[c + lane * KP] = rcq;
    __syncwarp();
    if (lane > c && lane < k)
      for (int p = c + 1; p <= lane; ++p) Rs[p + lane * KP] -= Rs[c + p * KP] * rcq;
    __syncwarp();
  }
  if (!(kap <= kGramKappaMax)) return false;
  // R = R_s D^-1: column q times cn_q
  if (lane < k)
    for (int p = 0; p <= lane; ++p) Rs[p + lane * KP] *= nq;
  __syncwarp();
  return true;
}

template <class S, int KMAX, int MMAX, int ALG>
struct MixedLayout {
  using SD = typename DoubleOf<S>::T;
  static constexpr int LDT = MMAX + 1;  // odd leading dimensions: no bank conflicts between columns
  static constexpr int KP = KMAX + 1;
  static constexpr int kTile = LDT * KMAX;
  static constexpr int kRR = ALG == DIAF_ALG_Q ? kRRMax : 0;  // DIAF-Q only: scratch for C v, r, coefficients
  // The FP64 tile lives in global memory (ColArgs::tile_scratch, one slab
  // per resident warp, mostly L1/L2 hits): shared memory holds only the FP32
  // working set and the vectors, which raises the warps resident per SM
  // (measured: 11 -> 18 for complex 16-column tiles, 6 -> 11 for real
  // 32-column ones, 21 -> 28 by shared memory for real 16-column ones).  A
  // slab holds the tile and two tiles of scratch for the FP64 keys of the
  // columns whose FP32 keys cannot decide.
  static constexpr size_t tile_bytes() { return 3 * sizeof(SD) * kTile; }
  // The FP64 keys of the columns whose FP32 keys cannot decide: in shared
  // memory (over the FP32 keys, which then take 2 MMAX floats), except for
  // the real 32-column tiles, where shared memory sets the warps per SM and
  // such columns are few: there they go to the slab after the FP64 R
  // (12 -> 13 warps per SM).  On the complex Helmholtz tiles the slab
  // placement measured 11 % slower, so it is limited to the real wide ones.
  static constexpr bool kKeysInSlab = KMAX > 16 && !ScalarInfo<S>::cplx;
  static_assert(KP * KMAX * sizeof(SD) + MMAX * sizeof(double) <= kTile * sizeof(SD), "FP64 keys after R in the slab");
  // Householder QR with the tile in registers (one row per lane): tiles of
  // up to 32 rows and 16 columns
  static constexpr bool kRegQR = KMAX <= 16 && MMAX <= 32;
  // DIAF-S keeps the Jacobi's V in the working tile, which is dead once
  // R-hat has been copied out of it (kTile >= KP KMAX since MMAX >= KMAX):
  // one k x k factor less per warp (real 32-column tiles: 10 -> 12 warps
  // per SM)
  static constexpr int kFactors = ALG == DIAF_ALG_S ? 1 : 2;
  static_assert(MMAX >= KMAX, "the working tile holds V");
  static constexpr size_t raw() {
    return sizeof(SD) * (3 * KMAX + 2 * MMAX + kRR * KP + 2 * kRR * kRR) +
           sizeof(S) * (kTile + kFactors * KP * KMAX + KMAX) + sizeof(float) * MMAX * (kKeysInSlab ? 1 : 2) +
           sizeof(double) * (2 * KMAX) + idx_bytes<KMAX, MMAX>();
  }
  static constexpr size_t bytes() { return (raw() + 15) / 16 * 16; }
};

// lane c < k: (T^* z)_c in FP64 over the m tile rows.  Tiles of up to 16
// columns split the rows between the two half-warps (alternate rows, one
// shuffle to combine), halving the FP64 instructions of the product.
template <class SD, int LDT, int KMAX>
__device__ __forceinline__ SD tile_adj_mul(const SD* Ts, const SD* zz, int m, int k, int lane) {
  SD g = sc_zero<SD>();
  if constexpr (KMAX <= 16) {
    const int c = lane & 15;
    if (c < k)
      for (int r = lane >> 4; r < m; r += 2) g += sc_cmul(Ts[r + c * LDT], zz[r]);
    g += shfl_xor(g, 16);
  } else {
    if (lane < k)
      for (int r = 0; r < m; ++r) g += sc_cmul(Ts[r + lane * LDT], zz[r]);
  }
  return g;
}

template <class S, int KMAX, int MMAX, int ALG>
__device__ void solve_column_mixed(const ColArgs& a, int j, unsigned char* smem,
                                   typename DoubleOf<S>::T* Ts, typename DoubleOf<S>::T* Tx, int lane) {
  using SD = typename DoubleOf<S>::T;
  using R = RealOf<S>;
  using L = MixedLayout<S, KMAX, MMAX, ALG>;
  constexpr int LDT = L::LDT, KP = L::KP, kRR = L::kRR;
  // Ts: the FP64 tile (LDT x KMAX) and Tx: two tiles of scratch, in the slab
  SD* rinvD = reinterpret_cast<SD*>(smem);  // KMAX FP64 scratch: FP64-key reciprocal diagonal, DIAF-S coefficients
  SD* wv = rinvD + KMAX;                 // w
  SD* gg = wv + KMAX;                    // k-vector scratch
  SD* vv = gg + KMAX;                    // v (MMAX)
  SD* zz = vv + MMAX;                    // m-vector scratch
  SD* Xs = zz + MMAX;                    // DIAF-Q scratch: C v (KP x kRR >= MMAX)
  SD* Cs = Xs + kRR * KP;                // DIAF-Q scratch: correction coefficients (as FP32)
  SD* Ms = Cs + kRR * kRR;               // DIAF-Q scratch: r = C v - mu v (as FP32)
  S* Tw = reinterpret_cast<S*>(Ms + kRR * kRR);  // FP32 working tile
  S* Rs = Tw + L::kTile;                 // FP32 R of T, then R-hat (Jacobi works on it)
  S* Vj = ALG == DIAF_ALG_S ? Tw : Rs + KP * KMAX;  // FP32 Jacobi V (DIAF-S: over the dead working tile)
  S* rinv = Rs + L::kFactors * KP * KMAX;  // FP32 reciprocal diagonal
  float* hk = reinterpret_cast<float*>(rinv + KMAX);  // FP32 keys (MMAX; 2 MMAX floats unless kKeysInSlab)
  double* sig = reinterpret_cast<double*>(hk + MMAX * (L::kKeysInSlab ? 1 : 2));
  R* sg = reinterpret_cast<R*>(sig);     // singular values / column norms in the FP32 type (KMAX)
  double* cn = sig + KMAX;               // column norms of the tile
  ColumnIdx ix = carve_idx<KMAX, MMAX>(reinterpret_cast<int32_t*>(cn + KMAX));

  const int k = a.Wcp[j + 1] - a.Wcp[j];
  const int m = a.m[j];
  const int l = a.l[j];
  const int me = m > k ? m : k;
  uint32_t flags = 0;

  auto hand_back = [&](int why) {
#ifdef DIAF_PHASE_TIMING
    if (lane == 0 && a.phase) atomicAdd(&a.phase[24 + why], 1ull);
#endif
    (void)why;
    if (lane == 0) {
      int pos = atomicAdd(a.fb_count, 1);
      a.fb_list[pos] = j;
    }
    __syncwarp();
  };
  if (k == 0) {  // trivial columns: the FP64 kernel has the conventions
    hand_back(0);
    return;
  }

  DIAF_PHASE_START();
  gather_tile<SD, KMAX, MMAX, LDT>(a, j, k, m, me, Ts, ix, lane);
  DIAF_PHASE(0);

  // ---- FP32 QR of T and the keys
  if constexpr (L::kRegQR) {
    // the tile in registers, one row per lane: R and the column norms directly
    DIAF_PHASE(1);
    warp_qr_rows<S, SD, LDT, KP, KMAX>(Ts, nullptr, m, k, Rs, cn, lane);
  } else {
    for (int i = lane; i < me * k; i += DIAF_WARP) {
      int r = i % me, c = i / me;
      Tw[r + c * LDT] = sc_cast<S>(Ts[r + c * LDT]);
    }
    __syncwarp();
    for (int c = lane; c < k; c += DIAF_WARP) {  // column norms for the kappa estimate: FP32 is enough
      R s2 = R(0);
      for (int r = 0; r < m; ++r) s2 += sc_abs2(Tw[r + c * LDT]);
      cn[c] = (double)sqrt(s2);
    }
    __syncwarp();
    DIAF_PHASE(1);
    warp_householder_qr_rs<S, LDT, KMAX, MMAX / DIAF_WARP>(Tw, me, k, lane);
    for (int i = lane; i < k * k; i += DIAF_WARP) {
      int r = i % k, c = i / k;
      Rs[r + c * KP] = (r <= c) ? Tw[r + c * LDT] : sc_zero<S>();
    }
    __syncwarp();
  }
  DIAF_PHASE(2);
  float kap = 0.0f;
  for (int c = lane; c < k; c += DIAF_WARP) {
    float d = (float)sc_abs(Rs[c + c * KP]);
    kap = fmaxf(kap, d > 0.0f ? (float)cn[c] / d : INFINITY);
  }
  kap = warp_max(kap);
  if (!(kap <= kMixedKappaMax)) { hand_back(1); return; }
  warp_leverage_rows<S, SD, LDT, KP>(Ts, Rs, Tw, hk, rinv, m, k, R(0), lane);
  DIAF_PHASE(3);
  if (a.rule != DIAF_RULE_FIXED) {
    const double margin = select_rows_greedy(ix.rs, hk, ix.pick, m, a.rule, j, l - 1, a.tie_tol, lane, a.blk);
    // bound on the FP32 key error: backward error of the FP32 QR and of the
    // row solves, amplified by the (column-scaled) conditioning of T
    const double delta = kMixedDeltaScale * (m + k) * (double)FLT_EPSILON * (double)kap;
    if (l > 1 && margin <= 2.0 * delta) {
      // the FP32 keys cannot decide this column: recompute them the way the
      // FP64 kernel does -- its Householder QR and leverage routines, in FP64,
      // on a copy of the tile in the slab -- and select with those, so I_j is
      // the FP64 kernel's choice; the rest of the column stays mixed
      SD* Tq = Tx;             // QR workspace, then the FP64 rows of Q (LDT x KMAX)
      SD* Rq = Tx + L::kTile;  // the FP64 R (KP x KMAX)
      double* hd = L::kKeysInSlab ? reinterpret_cast<double*>(Rq + KP * KMAX)  // FP64 keys (MMAX)
                                  : reinterpret_cast<double*>(hk);
      for (int i = lane; i < me * k; i += DIAF_WARP) Tq[(i % me) + (i / me) * LDT] = Ts[(i % me) + (i / me) * LDT];
      __syncwarp();
      warp_householder_qr_rs<SD, LDT, KMAX, MMAX / DIAF_WARP>(Tq, me, k, lane);
      for (int i = lane; i < k * k; i += DIAF_WARP) {
        const int r = i % k, c = i / k;
        Rq[r + c * KP] = (r <= c) ? Tq[r + c * LDT] : sc_zero<SD>();
      }
      __syncwarp();
      RealOf<SD> rdmax = RealOf<SD>(0);
      for (int c = lane; c < k; c += DIAF_WARP) rdmax = dmax(rdmax, sc_abs(Rq[c + c * KP]));
      rdmax = warp_max(rdmax);
      warp_leverage_rows<SD, SD, LDT, KP>(Ts, Rq, Tq, hd, rinvD, m, k, RealOf<SD>(1e-14) * rdmax, lane);
      select_rows_greedy(ix.rs, hd, ix.pick, m, a.rule, j, l - 1, a.tie_tol, lane, a.blk);
#ifdef DIAF_PHASE_TIMING
      if (lane == 0 && a.phase) atomicAdd(&a.phase[24 + 2], 1ull);
#endif
    }
  }
  const int jpos = build_I(a, j, m, l, ix, lane);
  double rank_thr = -1.0;
  for (int t = lane; t < l; t += DIAF_WARP) vv[t] = sc_zero<SD>();
  __syncwarp();
  DIAF_PHASE(4);

  if (ALG == DIAF_ALG_S) {
    // ---- FP32 QR of A-hat (I_j rows zeroed) into Rs; then the Jacobi SVD of R-hat
    if constexpr (L::kRegQR) {
      DIAF_PHASE(5);
      warp_qr_rows<S, SD, LDT, KP, KMAX>(Ts, ix.inI, m, k, Rs, cn, lane);
    } else {
      for (int i = lane; i < me * k; i += DIAF_WARP) {
        int r = i % me, c = i / me;
        Tw[r + c * LDT] = (r < m && ix.inI[r] >= 0) ? sc_zero<S>() : sc_cast<S>(Ts[r + c * LDT]);
      }
      __syncwarp();
      bool gram_hat = false;
      if constexpr (!ScalarInfo<S>::cplx) {
        // R-hat from the Gram matrix of A-hat's own rows (no downdating, so no
        // cancellation): lane q forms column q of G-hat = A-hat^T A-hat in
        // FP32, then a scaled Cholesky factor; kept when the column-scaled
        // kappa is at most kGramKappaMax (the Householder QR otherwise, and for
        // an exactly zero column of A-hat)
        gram_hat = warp_gram_cholesky<KMAX, LDT, KP>(Tw, m, k, Rs, cn, lane);
      }
      DIAF_PHASE(5);
      if (!gram_hat) {
        if constexpr (ScalarInfo<S>::cplx) {  // (the Gram path gave the real tiles' norms)
          for (int c = lane; c < k; c += DIAF_WARP) {
            R s2 = R(0);
            for (int r = 0; r < m; ++r) s2 += sc_abs2(Tw[r + c * LDT]);
            cn[c] = (double)sqrt(s2);
          }
          __syncwarp();
        }
        warp_householder_qr_rs<S, LDT, KMAX, MMAX / DIAF_WARP>(Tw, me, k, lane);
        for (int i = lane; i < k * k; i += DIAF_WARP) {
          int r = i % k, c = i / k;
          Rs[r + c * KP] = (r <= c) ? Tw[r + c * LDT] : sc_zero<S>();
        }
        __syncwarp();
      }
    }
    DIAF_PHASE(6);
    // an exactly zero column of A-hat (all its tile entries in I_j) is no
    // conditioning problem: it is an exact zero singular value, which the FP32
    // Jacobi keeps exact (w = e_c, residual 0, flagged from the residual)
    float kh = 0.0f;
    for (int c = lane; c < k; c += DIAF_WARP) {
      const float d = (float)sc_abs(Rs[c + c * KP]);
      kh = fmaxf(kh, d > 0.0f ? (float)cn[c] / d : (cn[c] > 0.0 ? INFINITY : 0.0f));
    }
    kh = warp_max(kh);
    if (!(kh <= kMixedKappaMax)) { hand_back(3); return; }
    // register-resident pairs for the warp-per-column tiles of up to 16
    // columns; the wider tiles (fewer warps per SM) keep the plain form
    int sw;
    if constexpr (KMAX <= 16)
      sw = warp_jacobi_reg<S, KP, KP, KMAX, KMAX>(Rs, k, k, Vj, reinterpret_cast<R*>(sig), lane);
    else
      sw = warp_jacobi<S, KP, KP, KMAX, true>(Rs, k, k, Vj, lane);
    if (sw < 0) flags |= DIAF_FLAG_JACOBI_NOCONV;
#ifdef DIAF_PHASE_TIMING
    if (lane == 0 && a.phase) atomicAdd(&a.phase[20], (unsigned long long)(sw < 0 ? kMaxSweeps : sw));
#endif
    DIAF_PHASE(7);
    // (FP32 scans here measured slower: they raised this branch's registers,
    // 80 -> 86 on the real 16-column tile, which cost more warps per SM than
    // the FP64 instructions they saved)
    warp_col_norms<S, KP>(Rs, k, k, sig, lane);
    int imin = 0;
    double smin = sig[0], smax = sig[0];
    for (int c = 1; c < k; ++c) {
      if (sig[c] < smin) { smin = sig[c]; imin = c; }
      smax = dmax(smax, sig[c]);
    }
    double snext = INFINITY;
    for (int c = 0; c < k; ++c) if (c != imin) snext = dmin(snext, sig[c]);
    if (k > 1 && (snext - smin) <= 1e-6 * smax) flags |= DIAF_FLAG_DEGENERATE;
    // ---- FP64 correction in the FP32 singular basis V (columns of Vj)
    double gap = INFINITY;
    for (int c = 0; c < k; ++c) if (c != imin) gap = dmin(gap, sig[c] * sig[c] - smin * smin);
    if (k > 1 && gap <= 1e-5 * smax * smax) { hand_back(4); return; }
    const int iters = (k > 1 && gap < 1e-2 * smax * smax) ? 2 : 1;
    // the correction itself is small: its projection runs in FP32 (relative
    // error ~1e-7 of a correction of relative size <~1e-5), the Rayleigh
    // quotient and the residual r = H x - d x in FP64
    S* cc = reinterpret_cast<S*>(rinvD);  // correction coefficients (KMAX)
    S* rf = reinterpret_cast<S*>(wv);     // r in FP32 (KMAX)
    SD x = lane < k ? sc_cast<SD>(Vj[lane + imin * KP]) : sc_zero<SD>();
    for (int it = 0; it < iters; ++it) {
      if (lane < k) gg[lane] = x;
      __syncwarp();
      for (int r = lane; r < m; r += DIAF_WARP) {
        SD z = sc_zero<SD>();
        if (ix.inI[r] < 0)
          for (int q = 0; q < k; ++q) z += Ts[r + q * LDT] * gg[q];
        zz[r] = z;
      }
      __syncwarp();
      const SD g = tile_adj_mul<SD, LDT, KMAX>(Ts, zz, m, k, lane);  // (H x)_q = (A-hat^* (A-hat x))_q
      const double xg = warp_sum(lane < k ? (double)sc_real(sc_cmul(x, g)) : 0.0);
      const double xx = warp_sum(lane < k ? (double)sc_abs2(x) : 0.0);
      const double d = xg / xx;
      if (lane < k) rf[lane] = sc_cast<S>(g - RealOf<SD>(d) * x);  // r = H x - d x
      __syncwarp();
      if (lane < k) {
        S vr = sc_zero<S>();
        for (int q = 0; q < k; ++q) vr += sc_cmul(Vj[q + lane * KP], rf[q]);
        const R sl = R(sig[lane]);
        const R den = sl * sl - R(d);
        cc[lane] = (lane == imin) ? sc_zero<S>() : (R(-1) / den) * vr;
      }
      __syncwarp();
      if (lane < k) {
        S dx = sc_zero<S>();
        for (int i = 0; i < k; ++i) dx += Vj[lane + i * KP] * cc[i];
        x += sc_cast<SD>(dx);
      }
      __syncwarp();
    }
    const double xn2 = warp_sum(lane < k ? (double)sc_abs2(x) : 0.0);
    if (lane < k) wv[lane] = RealOf<SD>(1.0 / sqrt(xn2)) * x;
    __syncwarp();
    DIAF_PHASE(8);
    // v = T(I_j,:) w and the rank test on the FP64 value of ||A-hat w||
    for (int t = lane; t < l; t += DIAF_WARP) {
      SD s = sc_zero<SD>();
      int r = ix.Iloc[t];
      if (r >= 0)
        for (int q = 0; q < k; ++q) s += Ts[r + q * LDT] * wv[q];
      vv[t] = s;
    }
    rank_thr = 1e-14 * smax;  // tested on res = ||A-hat w|| in finish_column
    __syncwarp();
  } else {
    // ---- eigenpairs of C = Q_I Q_I^* by an FP32 one-sided Jacobi (the rows of
    // Q = T R^-1 are in Tw).  l >= k: on Q_I itself, Q_I V = U S.  l < k: on
    // the smaller M = Q_I^* (k x l), whose right singular vectors are C's
    // eigenvectors.  Either way column c < kc of Tw ends as U_c s_c.
    int kc = k, sw;
    if (l < k && l <= kRRMax) {
      S* M = reinterpret_cast<S*>(Xs);  // k x l, leading dimension KP
      for (int i = lane; i < k * l; i += DIAF_WARP) {
        const int c = i % k, t = i / k, r = ix.Iloc[t];
        M[c + t * KP] = r >= 0 ? sc_conj(Tw[r + c * LDT]) : sc_zero<S>();
      }
      __syncwarp();
      sw = warp_jacobi_reg<S, KP, KP, kRRMax, KMAX>(M, k, l, Vj, reinterpret_cast<R*>(sig), lane);
      warp_col_norms_r<S, KP>(M, k, l, sg, lane);
      for (int i = lane; i < l * l; i += DIAF_WARP) {
        const int t = i % l, c = i / l;
        Tw[t + c * LDT] = sg[c] * Vj[t + c * KP];
      }
      __syncwarp();
      kc = l;
    } else {
      compact_rows<S, LDT>(Tw, ix.Iloc, l, k, lane);
      sw = warp_jacobi<S, LDT, KP, KMAX, true>(Tw, l, k, Vj, lane);
      warp_col_norms_r<S, LDT>(Tw, l, k, sg, lane);
    }
    if (sw < 0) flags |= DIAF_FLAG_JACOBI_NOCONV;
    DIAF_PHASE(7);
    int imax = 0;
    R smaxf = sg[0];
    for (int c = 1; c < kc; ++c) if (sg[c] > smaxf) { smaxf = sg[c]; imax = c; }
    R snextf = R(0);
    for (int c = 0; c < kc; ++c) if (c != imax) snextf = fmaxf(snextf, sg[c]);
    if (!(smaxf > R(0))) { hand_back(6); return; }
    if (kc > 1 && (smaxf - snextf) <= R(1e-6) * smaxf) flags |= DIAF_FLAG_DEGENERATE;
    const double smax = smaxf, snext = snextf;
    // the correction below converges from v0's FP32 error (about eps_32 / relative
    // gap) only when that error is small against the gap: closer gaps go to FP64
    const double gap2 = smax * smax - snext * snext;
    if (kc > 1 && gap2 < 1e-3 * smax * smax) { hand_back(4); return; }
    // the FP32 factors perturb C (norm <= 1) by about eps_32 kappa(T), so each
    // correction shrinks v's error by about rho = eps_32 kappa(T) / gap (a Newton
    // step with an FP32 Jacobian): iterate until the predicted error rho ||dv||
    // is below 1e-11 ||v||, at most kQRefineMax times
    const double rho = 8.0 * 1.1920929e-7 * (double)kap / gap2;
    {
      const RealOf<SD> inv = RealOf<SD>(1) / RealOf<SD>(smax);
      for (int t = lane; t < l; t += DIAF_WARP) vv[t] = inv * sc_cast<SD>(Tw[t + imax * LDT]);
    }
    __syncwarp();
    // lane c < k: (T^* T)^-1 T_I^* x for an l-vector x, with the FP32 factor
    // in FP32 arithmetic (a first guess, or the image of a small update)
    auto solve32 = [&](const SD* x) -> SD {
      SD b = sc_zero<SD>();
      if (lane < k)
        for (int t = 0; t < l; ++t) {
          const int rI = ix.Iloc[t];
          if (rI >= 0) b += sc_cmul(Ts[rI + lane * LDT], x[t]);
        }
      return sc_cast<SD>(warp_solve_RhR<S, S, KP>(Rs, rinv, sc_cast<S>(b), k, lane));
    };
    // one correction of y for the current v: the residual T^* (v_I - T y) on
    // the FP64 tile (v_I: v on the rows of I_j, zero elsewhere), solved with
    // the FP32 factor; it shrinks y's error by about eps_32 kappa(T)^2
    auto correct = [&](SD y) -> SD {
      if (lane < k) gg[lane] = y;
      __syncwarp();
      for (int r = lane; r < m; r += DIAF_WARP) {
        const int t = ix.inI[r];
        SD z = t >= 0 ? vv[t] : sc_zero<SD>();
        for (int q = 0; q < k; ++q) z -= Ts[r + q * LDT] * gg[q];
        zz[r] = z;
      }
      __syncwarp();
      const SD rn = tile_adj_mul<SD, LDT, KMAX>(Ts, zz, m, k, lane);
      y += sc_cast<SD>(warp_solve_RhR<S, S, KP>(Rs, rinv, sc_cast<S>(rn), k, lane));
      __syncwarp();
      return y;
    };
    // y = (T^* T)^-1 T_I^* v (lane c holds y_c): C v = T_I y, and for the final
    // v this y is the least-squares w of eq. condwj.  From scratch once (FP32
    // solve + two corrections); afterwards y follows each update dv of v by the
    // FP32 solve for dv (dv is small) plus one correction.
    SD y = solve32(vv);
    y = correct(y);
    y = correct(y);
    SD* cvv = Xs;                              // C v, then the update dv (l)
    S* rl = reinterpret_cast<S*>(Ms);          // r = C v - mu v in FP32 (l)
    S* ac = reinterpret_cast<S*>(Cs);          // U_c^* r / (s_c^2 - mu) (kc)
    S* bc = ac + KMAX;                         // U_c^* r (kc)
    bool converged = false;
    int it = 0;
    while (true) {
      if (lane < k) gg[lane] = y;
      __syncwarp();
      RealOf<SD> vcv = 0, vvn = 0;
      for (int t = lane; t < l; t += DIAF_WARP) {
        SD cv = sc_zero<SD>();
        const int rI = ix.Iloc[t];
        if (rI >= 0)
          for (int q = 0; q < k; ++q) cv += Ts[rI + q * LDT] * gg[q];
        cvv[t] = cv;
        vcv += sc_real(sc_cmul(vv[t], cv));
        vvn += sc_abs2(vv[t]);
      }
      vcv = warp_sum(vcv);
      vvn = warp_sum(vvn);
      const double mu = (double)vcv / (double)vvn;
      for (int t = lane; t < l; t += DIAF_WARP) rl[t] = sc_cast<S>(cvv[t] - RealOf<SD>(mu) * vv[t]);
      __syncwarp();
      for (int c = lane; c < kc; c += DIAF_WARP) {  // projections on U_c = Tw(:,c) / s_c
        const R sc = sg[c];
        S p = sc_zero<S>();
        if (sc > R(0))
          for (int t = 0; t < l; ++t) p += sc_cmul(Tw[t + c * LDT], rl[t]);
        p = sc > R(0) ? (R(1) / sc) * p : sc_zero<S>();
        bc[c] = p;
        ac[c] = (c == imax || !(sc > R(0))) ? sc_zero<S>() : (R(1) / (sc * sc - R(mu))) * p;
      }
      __syncwarp();
      // v <- v - sum_{c != max} U_c a_c + r_perp / mu  (r_perp: the part of r outside
      // the span of the U_c, C's null space when Q_I has rank below l)
      R dn = 0;
      for (int t = lane; t < l; t += DIAF_WARP) {
        S dv = sc_zero<S>(), rin = sc_zero<S>();
        for (int c = 0; c < kc; ++c) {
          const R sc = sg[c];
          if (!(sc > R(0))) continue;
          const S u = (R(1) / sc) * Tw[t + c * LDT];
          dv += u * ac[c];
          rin += u * bc[c];
        }
        const S rperp = rl[t] - rin;
        const S step = (R(1) / R(mu)) * rperp - dv;
        dn += sc_abs2(step);
        const SD stepd = sc_cast<SD>(step);
        vv[t] += stepd;
        cvv[t] = stepd;
      }
      dn = warp_sum(dn);
      converged = rho * rho * (double)dn <= 1e-22 * (double)vvn;
      __syncwarp();
      y += solve32(cvv);
      ++it;
      if (converged || it == kQRefineMax) break;
      y = correct(y);
    }
#ifdef DIAF_PHASE_TIMING
    if (lane == 0 && a.phase) atomicAdd(&a.phase[20], (unsigned long long)it);
#endif
    DIAF_PHASE(8);
    if (!converged) { hand_back(5); return; }
    RealOf<SD> vn = 0;
    for (int t = lane; t < l; t += DIAF_WARP) vn += sc_abs2(vv[t]);
    vn = warp_sum(vn);
    {
      const RealOf<SD> inv = RealOf<SD>(1) / sqrt(vn);
      for (int t = lane; t < l; t += DIAF_WARP) vv[t] = inv * vv[t];
      if (lane < k) wv[lane] = inv * y;  // w: eq. condwj for the normalised v
    }
    __syncwarp();
    // stabilised DIAF-Q (Sec. 3.2): the FP64 kernel takes every column at or
    // near the trigger, so the decision is the FP64 one
    if (a.stab_tol > 0.0 && jpos >= 0 && l > 1 && (double)sc_abs(vv[jpos]) < a.stab_tol * (1.0 + 1e-6)) {
      hand_back(7);
      return;
    }
  }
  DIAF_PHASE(9);
  finish_column<SD, LDT>(a, j, k, m, l, jpos, Ts, wv, vv, ix, flags, true, lane, rank_thr);
  DIAF_PHASE(10);
}

// The persistent loop: one warp per column, columns taken from the work
// counter.
template <class S, int KMAX, int MMAX, int ALG>
__device__ __forceinline__ void column_mixed_loop(const ColArgs& a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  using L = MixedLayout<S, KMAX, MMAX, ALG>;
  unsigned char* smem = smem_raw + warp * L::bytes();
  typename L::SD* Ts = reinterpret_cast<typename L::SD*>(a.tile_scratch) +
                       (size_t)(blockIdx.x * (blockDim.x >> 5) + warp) * 3 * L::kTile;
  const int count = *a.list_count;
  while (true) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(a.work_counter, 1);
    idx = __shfl_sync(DIAF_FULL, idx, 0);
    if (idx >= count) break;
    solve_column_mixed<S, KMAX, MMAX, ALG>(a, list_at(a, count, idx), smem, Ts, Ts + L::kTile, lane);
  }
}

template <class S, int KMAX, int MMAX, int ALG>
__global__ void column_mixed_kernel(ColArgs a) {
  column_mixed_loop<S, KMAX, MMAX, ALG>(a);
}

// The same kernel with a register cap CAP: the real 16-column DIAF-Q tiles
// run 5 % faster at 72 (27 instead of 24 warps per SM, no spills).  The
// DIAF-S one did not gain from a cap; an explicit cap on the others raised
// their register counts (the compiler's own choice is the better one there).
template <class S, int KMAX, int MMAX, int ALG, int CAP>
__global__ void __maxnreg__((CAP)) column_mixed_kernel_cap(ColArgs a) {
  column_mixed_loop<S, KMAX, MMAX, ALG>(a);
}

// 0: no cap (a cap of 112 on the complex 16-column tiles, 18 instead of 16
// warps per SM, measured no faster)
template <class S, int KMAX, int ALG>
constexpr int mixed_reg_cap() {
  return (sizeof(S) == 4 && KMAX <= 16 && ALG == DIAF_ALG_Q) ? 72 : 0;
}
