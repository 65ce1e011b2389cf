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

// Returns true when the column was finished here, false when it is handed back.
__device__ bool solve_column_cta_mixed(const ColArgs& a, const CtaScratch& sc, int j, unsigned char* smem) {
  using L = CtaMixedSmem;
  constexpr int KP = L::KP;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int mcap = sc.ldm;
  float* Rs = reinterpret_cast<float*>(smem);  // R of T, then R-hat (KP x KMAX)
  float* Vj = Rs + KP * kCtaKmax;               // Jacobi V
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

  // the slab holds two tiles of the FP64 kernel's size: the FP64 tile, then the FP32 one
  double* Ts = reinterpret_cast<double*>(sc.slab) + (size_t)blockIdx.x * 2 * sc.ldm * sc.kcap;
  float* Tw = reinterpret_cast<float*>(Ts + (size_t)sc.ldm * sc.kcap);
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

  // ---- gather (FP64) and the FP32 copy
  for (int r = tid; r < mcap; r += kCtaThreads) {
    rs[r] = r < m ? Rj[r] : INT_MAX;
    inI[r] = -1;
    pick[r] = 0;
  }
  for (size_t i = tid; i < (size_t)me * k; i += kCtaThreads) Ts[(i % me) + (i / me) * ld] = 0.0;
  if (tid == 0) {
    int e = 0;
    for (int q = 0; q < k; ++q) {
      const int c = J[q];
      cst[q] = a.Acp[c];
      coff[q] = e;
      e += a.Acp[c + 1] - a.Acp[c];
    }
    misc[1] = e;
  }
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
  const float kap = block_max(kp, redF);
  if (!(kap <= kMixedKappaMax)) return false;
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
    const double margin = cta_select_rows(rs, hk, pick, m, a.rule, j, l - 1, a.tie_tol, red, a.blk);
    const double delta = kMixedDeltaScale * (m + k) * (double)FLT_EPSILON * (double)kap;
    if (l > 1 && margin <= 2.0 * delta) {
      // the FP32 keys cannot decide this column: the FP64 CTA kernel's QR and
      // key computation on an FP64 copy of the tile (in the FP32 tile's slab
      // space, rewritten for A-hat below), then the selection with those keys,
      // so I_j is the FP64 kernel's choice
      double* Tq = reinterpret_cast<double*>(Tw);
      double* Rq = reinterpret_cast<double*>(Rs);  // KP x KMAX doubles over Rs and Vj (both free here)
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
      cta_select_rows(rs, hk, pick, m, a.rule, j, l - 1, a.tie_tol, red, a.blk);
    }
  }
  // I_j
  if (tid == 0) {
    misc[0] = -1;
    int cnt = 0;
    if (a.rule == DIAF_RULE_FIXED) {
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
    } else {
      bool placed = false;
      for (int r = 0; r < m; ++r) {
        if (!placed && !a.jin[j] && rs[r] > j) { Is[cnt] = j; Iloc[cnt] = -1; misc[0] = cnt; ++cnt; placed = true; }
        if (pick[r] || rs[r] == j) {
          Is[cnt] = rs[r];
          Iloc[cnt] = r;
          inI[r] = cnt;
          if (rs[r] == j) misc[0] = cnt;
          ++cnt;
        }
      }
      if (!placed && !a.jin[j]) { Is[cnt] = j; Iloc[cnt] = -1; misc[0] = cnt; ++cnt; }
    }
  }
  __syncthreads();
  const int jpos = misc[0];
  int inrows = 0;
  for (int t = 0; t < l; ++t) inrows += (Iloc[t] >= 0);
  if (m - inrows < k) return false;  // A-hat has fewer rows than columns

  // ---- FP32 QR of A-hat, Jacobi SVD of R-hat
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
  if (!(block_max(kh, redF) <= kMixedKappaMax)) return false;
  for (int i = tid; i < k * k; i += kCtaThreads) {
    const int r = i % k, c = i / k;
    Rs[r + c * KP] = (r <= c) ? Tw[r + (size_t)c * ld] : 0.0f;
  }
  __syncthreads();
  if (cta_jacobi<float, KP, KP>(Rs, k, k, Vj, redF) < 0) flags |= DIAF_FLAG_JACOBI_NOCONV;
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
  if (k > 1 && gap <= 1e-5 * smax * smax) return false;
  const int iters = (k > 1 && gap < 1e-2 * smax * smax) ? 2 : 1;

  // ---- FP64 correction in the FP32 singular basis
  for (int c = tid; c < k; c += kCtaThreads) wv[c] = (double)Vj[c + imin * KP];
  __syncthreads();
  for (int it = 0; it < iters; ++it) {
    for (int r = tid; r < m; r += kCtaThreads) {  // z = A-hat x
      double z = 0.0;
      if (inI[r] < 0)
        for (int q = 0; q < k; ++q) z += Ts[r + (size_t)q * ld] * wv[q];
      zz[r] = z;
    }
    __syncthreads();
    for (int c = warp; c < k; c += kCtaWarps) {  // H x = A-hat^T z
      double g = 0.0;
      for (int r = lane; r < m; r += 32) g += Ts[r + (size_t)c * ld] * zz[r];
      g = warp_sum(g);
      if (lane == 0) gg[c] = g;
    }
    __syncthreads();
    double xg = 0.0, xx = 0.0;
    for (int c = tid; c < k; c += kCtaThreads) {
      xg += wv[c] * gg[c];
      xx += wv[c] * wv[c];
    }
    xg = block_sum(xg, red);
    xx = block_sum(xx, red);
    const double d = xg / xx;
    for (int c = tid; c < k; c += kCtaThreads) rf[c] = (float)(gg[c] - d * wv[c]);
    __syncthreads();
    for (int i = tid; i < k; i += kCtaThreads) {
      float vr = 0.0f;
      for (int q = 0; q < k; ++q) vr += Vj[q + i * KP] * rf[q];
      const float si = (float)sig[i];
      const float den = si * si - (float)d;
      cc[i] = i == imin ? 0.0f : -vr / den;
    }
    __syncthreads();
    for (int c = tid; c < k; c += kCtaThreads) {
      float dx = 0.0f;
      for (int i = 0; i < k; ++i) dx += Vj[c + i * KP] * cc[i];
      wv[c] += (double)dx;
    }
    __syncthreads();
  }
  double xn = 0.0;
  for (int c = tid; c < k; c += kCtaThreads) xn += wv[c] * wv[c];
  xn = block_sum(xn, red);
  const double inv = 1.0 / sqrt(xn);
  for (int c = tid; c < k; c += kCtaThreads) wv[c] *= inv;
  __syncthreads();
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
  return true;
}

__global__ void __launch_bounds__(kCtaThreads) column_cta_mixed_kernel(ColArgs a, CtaScratch sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int idx_s;
  const int count = *a.list_count;
  while (true) {
    if (threadIdx.x == 0) idx_s = atomicAdd(a.work_counter, 1);
    __syncthreads();
    const int idx = idx_s;
    __syncthreads();
    if (idx >= count) break;
    const int j = a.list[idx];
    if (!solve_column_cta_mixed(a, sc, j, smem_raw)) {
      if (threadIdx.x == 0) a.fb_list[atomicAdd(a.fb_count, 1)] = j;
    }
    __syncthreads();
  }
}
