// Mixed-precision per-column kernel: the tile is gathered in FP64 (complex128)
// and copied to FP32 (complex64); QR, leverage keys and the Jacobi SVD run in
// FP32; then (w_j, v_j) get one FP64 refinement step against the FP64 tile
// and the residual ||A w - v|| is evaluated in FP64.
//
//   DIAF-S: the FP32 Jacobi gives R-hat V = U diag(sigma); x0 = V e_min.
//     With H = A-hat^* A-hat taken from the FP64 tile, V^* H V is diagonal to
//     FP32 accuracy, so one correction in that basis,
//       d = x^* H x / x^* x,  r = H x - d x,
//       x <- x - sum_{i != min} V_i (V_i^* r) / (sigma_i^2 - d),
//     makes x the smallest right singular vector to second order (repeated
//     once when the relative gap is below 1e-2; columns with a gap below 1e-5
//     go to the FP64 kernel).  w = x / ||x||, v = T(I_j,:) w.
//   DIAF-Q: v0 = Q_I u / sigma from the FP32 Jacobi.  In FP64:
//     X = (T^* T)^-1 T_I^* column by column (normal equations with the FP32 R
//     as the solver plus one correction with the FP64 residual), the l x l
//     matrix C = T_I X whose top eigenvector is the optimal v of eq. nocond
//     (C = M_j^* M_j), one Rayleigh-quotient-iteration step from v0
//     (mu = v0^* C v0, v = (C - mu)^-1 v0 normalised), and w = X v, the
//     least-squares solution of eq. condwj.  Columns with l_j > 8 go to the
//     FP64 kernel.
//
// A column goes to the FP64 kernel instead (appended to fb_list) when a
// leverage-selection decision is closer to its threshold than the FP32 key
// error bound (so I_j could differ from the FP64 choice), or when the tile is
// too ill-conditioned for FP32 factors to drive the refinement.
#pragma once

#include "column.cuh"

template <class S> struct DoubleOf;
template <> struct DoubleOf<float> { using T = double; };
template <> struct DoubleOf<Cx<float>> { using T = Cx<double>; };

constexpr int kRRMax = 8;  // DIAF-Q: largest l_j refined through the explicit l x l matrix C

template <class S, int KMAX, int MMAX, int ALG>
struct MixedLayout {
  using SD = typename DoubleOf<S>::T;
  static constexpr int LDT = MMAX + 1;  // odd leading dimensions: no bank conflicts between columns
  static constexpr int KP = KMAX + 1;
  static constexpr int kTile = LDT * KMAX;
  static constexpr int kRR = ALG == DIAF_ALG_Q ? kRRMax : 0;  // DIAF-Q only: X, C, C - mu I
  static constexpr size_t raw() {
    return sizeof(SD) * (kTile + 3 * KMAX + 2 * MMAX + kRR * KP + 2 * kRR * kRR) +
           sizeof(S) * (kTile + 2 * KP * KMAX + KMAX) +
           sizeof(double) * (MMAX + 2 * KMAX) + idx_bytes<KMAX, MMAX>();
  }
  static constexpr size_t bytes() { return (raw() + 15) / 16 * 16; }
};

template <class S, int KMAX, int MMAX, int ALG>
__device__ void solve_column_mixed(const ColArgs& a, int j, unsigned char* smem, int lane) {
  using SD = typename DoubleOf<S>::T;
  using R = RealOf<S>;
  using L = MixedLayout<S, KMAX, MMAX, ALG>;
  constexpr int LDT = L::LDT, KP = L::KP, kRR = L::kRR;
  SD* Ts = reinterpret_cast<SD*>(smem);  // FP64 tile (LDT x KMAX)
  SD* rinvD = Ts + L::kTile;             // FP64 reciprocal diagonal of the FP32 factor
  SD* wv = rinvD + KMAX;                 // w
  SD* gg = wv + KMAX;                    // k-vector scratch
  SD* vv = gg + KMAX;                    // v (MMAX)
  SD* zz = vv + MMAX;                    // m-vector scratch
  SD* Xs = zz + MMAX;                    // DIAF-Q: X = (T^* T)^-1 T_I^* (KP x kRR)
  SD* Cs = Xs + kRR * KP;                // DIAF-Q: C = T_I X (kRRMax x kRRMax)
  SD* Ms = Cs + kRR * kRR;               // DIAF-Q: C - mu I, eliminated in place
  S* Tw = reinterpret_cast<S*>(Ms + kRR * kRR);  // FP32 working tile
  S* Rs = Tw + L::kTile;                 // FP32 R of T, then R-hat (Jacobi works on it)
  S* Vj = Rs + KP * KMAX;                // FP32 Jacobi V
  S* rinv = Vj + KP * KMAX;              // FP32 reciprocal diagonal
  float* hk = reinterpret_cast<float*>(rinv + KMAX);  // FP32 keys (MMAX; 2 MMAX floats reserved)
  double* sig = reinterpret_cast<double*>(hk + 2 * MMAX);
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
    if (l > 1 && margin <= 2.0 * delta) { hand_back(2); return; }
  }
  const int jpos = build_I(a, j, m, l, ix, lane);
  double rank_thr = -1.0;
  for (int t = lane; t < l; t += DIAF_WARP) vv[t] = sc_zero<SD>();
  __syncwarp();
  DIAF_PHASE(4);

  if (ALG == DIAF_ALG_S) {
    // ---- FP32 QR of A-hat (I_j rows zeroed); Jacobi SVD of R-hat in registers
    for (int i = lane; i < me * k; i += DIAF_WARP) {
      int r = i % me, c = i / me;
      Tw[r + c * LDT] = (r < m && ix.inI[r] >= 0) ? sc_zero<S>() : sc_cast<S>(Ts[r + c * LDT]);
    }
    __syncwarp();
    for (int c = lane; c < k; c += DIAF_WARP) {
      R s2 = R(0);
      for (int r = 0; r < m; ++r) s2 += sc_abs2(Tw[r + c * LDT]);
      cn[c] = (double)sqrt(s2);
    }
    __syncwarp();
    DIAF_PHASE(5);
    warp_householder_qr_rs<S, LDT, KMAX, MMAX / DIAF_WARP>(Tw, me, k, lane);
    DIAF_PHASE(6);
    // an exactly zero column of A-hat (all its tile entries in I_j) is no
    // conditioning problem: it is an exact zero singular value, which the FP32
    // Jacobi keeps exact (w = e_c, residual 0, flagged from the residual)
    float kh = 0.0f;
    for (int c = lane; c < k; c += DIAF_WARP) {
      const float d = (float)sc_abs(Tw[c + c * LDT]);
      kh = fmaxf(kh, d > 0.0f ? (float)cn[c] / d : (cn[c] > 0.0 ? INFINITY : 0.0f));
    }
    kh = warp_max(kh);
    if (!(kh <= kMixedKappaMax)) { hand_back(3); return; }
    for (int i = lane; i < k * k; i += DIAF_WARP) {
      int r = i % k, c = i / k;
      Rs[r + c * KP] = (r <= c) ? Tw[r + c * LDT] : sc_zero<S>();
    }
    __syncwarp();
    int sw = warp_jacobi<S, KP, KP, KMAX, true>(Rs, k, k, Vj, lane);
    if (sw < 0) flags |= DIAF_FLAG_JACOBI_NOCONV;
#ifdef DIAF_PHASE_TIMING
    if (lane == 0 && a.phase) atomicAdd(&a.phase[20], (unsigned long long)(sw < 0 ? kMaxSweeps : sw));
#endif
    DIAF_PHASE(7);
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
      SD g = sc_zero<SD>();  // (H x)_q = (A-hat^* (A-hat x))_q
      if (lane < k)
        for (int r = 0; r < m; ++r) g += sc_cmul(Ts[r + lane * LDT], zz[r]);
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
    // ---- FP32 Jacobi on Q_I (FP32 rows of Q = T R^-1 in Tw)
    if (l > kRRMax) { hand_back(5); return; }
    compact_rows<S, LDT>(Tw, ix.Iloc, l, k, lane);
    int sw = warp_jacobi<S, LDT, KP, KMAX, true>(Tw, l, k, Vj, lane);
    if (sw < 0) flags |= DIAF_FLAG_JACOBI_NOCONV;
    warp_col_norms<S, LDT>(Tw, l, k, sig, lane);
    int imax = 0;
    double smax = sig[0];
    for (int c = 1; c < k; ++c) if (sig[c] > smax) { smax = sig[c]; imax = c; }
    double snext = 0.0;
    for (int c = 0; c < k; ++c) if (c != imax) snext = dmax(snext, sig[c]);
    if (!(smax > 0.0)) { hand_back(6); return; }
    if (k > 1 && (smax - snext) <= 1e-6 * smax) flags |= DIAF_FLAG_DEGENERATE;
    // one Rayleigh-quotient step refines v0 to FP64 accuracy only when v0's
    // FP32 error (about eps_32 / relative gap) is small against the gap to the
    // second eigenvalue of Q_I Q_I^*: closer gaps go to the FP64 kernel
    if (k > 1 && (smax * smax - snext * snext) < 1e-3 * smax * smax) { hand_back(4); return; }
    for (int t = lane; t < l; t += DIAF_WARP) vv[t] = sc_cast<SD>(Tw[t + imax * LDT]);
    for (int c = lane; c < k; c += DIAF_WARP) rinvD[c] = sc_recip_or_zero(sc_cast<SD>(Rs[c + c * KP]), 0.0);
    __syncwarp();
    // X(:,t) = (T^* T)^-1 T(I_t,:)^*: one solve with the FP32 R, one correction
    for (int t = 0; t < l; ++t) {
      const int rI = ix.Iloc[t];
      const SD b = (lane < k && rI >= 0) ? sc_conj(Ts[rI + lane * LDT]) : sc_zero<SD>();
      SD x = warp_solve_RhR<SD, S, KP>(Rs, rinvD, b, k, lane);
      if (lane < k) gg[lane] = x;
      __syncwarp();
      for (int r = lane; r < m; r += DIAF_WARP) {
        SD z = sc_zero<SD>();
        for (int q = 0; q < k; ++q) z -= Ts[r + q * LDT] * gg[q];
        zz[r] = z;
      }
      __syncwarp();
      SD rn = b;
      if (lane < k)
        for (int r = 0; r < m; ++r) rn += sc_cmul(Ts[r + lane * LDT], zz[r]);
      x += warp_solve_RhR<SD, S, KP>(Rs, rinvD, rn, k, lane);
      if (lane < k) Xs[lane + t * KP] = x;
      __syncwarp();
    }
    // C = T_I X (Hermitian positive semidefinite, l x l)
    for (int e = lane; e < l * l; e += DIAF_WARP) {
      const int s2 = e % l, t = e / l, rI = ix.Iloc[s2];
      SD c = sc_zero<SD>();
      if (rI >= 0)
        for (int q = 0; q < k; ++q) c += Ts[rI + q * LDT] * Xs[q + t * KP];
      Cs[s2 + t * kRRMax] = c;
    }
    __syncwarp();
    // one Rayleigh-quotient-iteration step from v0 (lane 0; l <= 8)
    if (lane == 0) {
      using RD = RealOf<SD>;
      RD n2 = RD(0);
      for (int t = 0; t < l; ++t) n2 += sc_abs2(vv[t]);
      const RD ninv = RD(1) / sqrt(n2);
      SD y[kRRMax];
      for (int t = 0; t < l; ++t) y[t] = ninv * vv[t];
      RD mu = RD(0), cmax = RD(0);
      for (int s2 = 0; s2 < l; ++s2)
        for (int t = 0; t < l; ++t) {
          const SD c = Cs[s2 + t * kRRMax];
          mu += sc_real(sc_cmul(y[s2], c * y[t]));
          cmax = dmax(cmax, sc_abs(c));
        }
      for (int s2 = 0; s2 < l; ++s2)
        for (int t = 0; t < l; ++t)
          Ms[s2 + t * kRRMax] = Cs[s2 + t * kRRMax] - (s2 == t ? sc_real_s<SD>(mu) : sc_zero<SD>());
      // Gaussian elimination with partial pivoting; an exactly singular pivot
      // (v0 already an eigenvector) is replaced by eps ||C||
      const RD tinyp = eps_of<RD>() * (cmax > RD(0) ? cmax : RD(1));
      for (int c = 0; c < l; ++c) {
        int pr = c;
        RD pa = sc_abs(Ms[c + c * kRRMax]);
        for (int r = c + 1; r < l; ++r) {
          RD ar = sc_abs(Ms[r + c * kRRMax]);
          if (ar > pa) { pa = ar; pr = r; }
        }
        if (pr != c) {
          for (int t = 0; t < l; ++t) {
            SD tmp = Ms[c + t * kRRMax]; Ms[c + t * kRRMax] = Ms[pr + t * kRRMax]; Ms[pr + t * kRRMax] = tmp;
          }
          SD tmp = y[c]; y[c] = y[pr]; y[pr] = tmp;
        }
        if (!(sc_abs(Ms[c + c * kRRMax]) > tinyp)) Ms[c + c * kRRMax] = sc_real_s<SD>(tinyp);
        const SD dinv = sc_recip_or_zero(Ms[c + c * kRRMax], RD(0));
        for (int r = c + 1; r < l; ++r) {
          const SD f = Ms[r + c * kRRMax] * dinv;
          for (int t = c + 1; t < l; ++t) Ms[r + t * kRRMax] -= f * Ms[c + t * kRRMax];
          y[r] -= f * y[c];
        }
      }
      for (int c = l - 1; c >= 0; --c) {
        SD acc = y[c];
        for (int t = c + 1; t < l; ++t) acc -= Ms[c + t * kRRMax] * y[t];
        y[c] = acc * sc_recip_or_zero(Ms[c + c * kRRMax], RD(0));
      }
      RD yn2 = RD(0);
      for (int t = 0; t < l; ++t) yn2 += sc_abs2(y[t]);
      const RD yinv = RD(1) / sqrt(yn2);
      for (int t = 0; t < l; ++t) vv[t] = yinv * y[t];
    }
    __syncwarp();
    // stabilised DIAF-Q (Sec. 3.2): the FP64 kernel takes every column at or
    // near the trigger, so the decision is the FP64 one
    if (a.stab_tol > 0.0 && jpos >= 0 && l > 1 && (double)sc_abs(vv[jpos]) < a.stab_tol * (1.0 + 1e-6)) {
      hand_back(7);
      return;
    }
    // w = X v (eq. condwj for the refined v)
    if (lane < k) {
      SD x = sc_zero<SD>();
      for (int t = 0; t < l; ++t) x += Xs[lane + t * KP] * vv[t];
      wv[lane] = x;
    }
    __syncwarp();
  }
  DIAF_PHASE(9);
  finish_column<SD, LDT>(a, j, k, m, l, jpos, Ts, wv, vv, ix, flags, true, lane, rank_thr);
  DIAF_PHASE(10);
}

template <class S, int KMAX, int MMAX, int ALG>
__global__ void column_mixed_kernel(ColArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* smem = smem_raw + warp * MixedLayout<S, KMAX, MMAX, ALG>::bytes();
  const int count = *a.list_count;
  while (true) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(a.work_counter, 1);
    idx = __shfl_sync(DIAF_FULL, idx, 0);
    if (idx >= count) break;
    solve_column_mixed<S, KMAX, MMAX, ALG>(a, a.list[idx], smem, lane);
  }
}
