// Per-column kernel for large tiles (size bucket 2: k_j <= 64, m_j <= 1024),
// FP64 (complex128), one CTA of kCtaThreads threads per column.  Same steps
// as the warp kernel (gather, Householder QR, leverage keys, V rule, DIAF-S
// or DIAF-Q, phase, residual, scatter); the two tiles live in a per-CTA slab
// of global scratch (L2-resident), the k x k factors in shared memory.
#pragma once

#include "column.cuh"

constexpr int kCtaThreads = 256;
constexpr int kCtaWarps = kCtaThreads / 32;
constexpr int kCtaKmax = 64;

struct CtaScratch {
  void* slab;     // per CTA: Ts then Tw, each ldm x kcap scalars
  int ldm;        // leading dimension (>= every m_j, k_j of the bucket)
  int kcap;       // columns per tile (>= every k_j of the bucket)
  int gram;       // mixed real DIAF-S: 1 = tensor-core Gram + Cholesky where the tile is well conditioned
};

// ----------------------------------------------------------------- block reductions
template <class T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = red[0];
  for (int w = 1; w < kCtaWarps; ++w) s += red[w];
  return s;
}
template <class T>
__device__ __forceinline__ T block_max(T v, T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = red[0];
  for (int w = 1; w < kCtaWarps; ++w) s = red[w] > s ? red[w] : s;
  return s;
}
template <class T>
__device__ __forceinline__ T block_min(T v, T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_min(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = red[0];
  for (int w = 1; w < kCtaWarps; ++w) s = red[w] < s ? red[w] : s;
  return s;
}

// Greedy V rule of Sec. 3.1 (as select_rows_greedy: s picks among the
// admissible rows, at each pick the lowest row whose key is within tau of
// the largest remaining key) run by warp 0 alone -- rows r = lane + 32 i as
// bits of a register, warp reductions instead of CTA barriers -- while the
// other warps wait.  Writes pick[r] for r < m (m <= 1024) and returns, to
// every thread, the smallest distance of a non-leading candidate key from a
// threshold it was compared with.  red: one double of shared scratch.
template <class K>
__device__ double cta_select_rows_w0(const int32_t* rs, const K* hk, int32_t* pick, int m, int rule, int j, int s,
                                     double tau, const int32_t* blk, double* red) {
  if ((threadIdx.x >> 5) == 0) {
    const int lane = threadIdx.x & 31;
    uint32_t adm = 0, picked = 0;
    for (int i = 0; i < 32 && lane + 32 * i < m; ++i)
      if (admissible_row(rule, rs[lane + 32 * i], j, blk)) adm |= 1u << i;
    K margin = std::numeric_limits<K>::max();
    for (int t = 0; t < s; ++t) {
      const uint32_t cand = adm & ~picked;
      K hm = -std::numeric_limits<K>::max();
      for (uint32_t b = cand; b; b &= b - 1) hm = dmax(hm, hk[lane + 32 * (__ffs(b) - 1)]);
      hm = warp_max(hm);
      int rmax = INT_MAX;
      for (uint32_t b = cand; b && rmax == INT_MAX; b &= b - 1) {
        const int r = lane + 32 * (__ffs(b) - 1);
        if (hk[r] == hm) rmax = r;
      }
      rmax = warp_min(rmax);
      const K thr = hm - K(tau);
      int best = INT_MAX;
      for (uint32_t b = cand; b; b &= b - 1) {
        const int r = lane + 32 * (__ffs(b) - 1);
        const K h = hk[r];
        if (r != rmax) margin = dmin(margin, (K)fabs(h - thr));
        if (h >= thr && best == INT_MAX) best = r;
      }
      best = warp_min(best);
      if (best == INT_MAX) {  // no key reaches the threshold (non-finite keys): the lowest remaining admissible row
        const int lo = cand ? lane + 32 * (__ffs(cand) - 1) : INT_MAX;
        best = warp_min(lo);
      }
      if (best < m && (best & 31) == lane) picked |= 1u << (best >> 5);
    }
    margin = warp_min(margin);
    for (int i = 0; i < 32 && lane + 32 * i < m; ++i) pick[lane + 32 * i] = (picked >> i) & 1u;
    if (lane == 0) red[0] = (double)margin;
  }
  __syncthreads();
  const double mg = red[0];
  __syncthreads();  // red is free again
  return mg;
}

// The same greedy V rule (the same picks and the same decision margin as
// cta_select_rows_w0) from one sort instead of a scan of every remaining key
// per pick: warp 0 lists the admissible rows, the CTA sorts the list by key
// (descending; the lower row first among equal keys), and thread 0 walks
// it.  At a pick the largest remaining key heads the remaining list, the
// rows within tau of it are the run that follows (the lowest of them is
// picked), and the smallest distance of a non-leading key from the
// threshold is in that run or at the first remaining key below it (|h -
// thr| grows with the distance in the sorted order), so a pick reads only
// that run.  Needs finite keys and tau >= 0.  ord: shared scratch of at
// least the power of two >= m ints; red: one double of shared scratch.
template <class K>
__device__ double cta_select_rows_sorted(const int32_t* rs, const K* hk, int32_t* pick, int m, int rule, int j, int s,
                                         double tau, const int32_t* blk, double* red, int32_t* ord) {
  const int tid = threadIdx.x;
  __shared__ int na_s;
  if ((tid >> 5) == 0) {  // compaction of the admissible rows, in row order
    const int lane = tid & 31;
    int cnt = 0;
    for (int base = 0; base < m; base += 32) {
      const int r = base + lane;
      const bool ad = r < m && admissible_row(rule, rs[r], j, blk);
      const uint32_t bal = __ballot_sync(DIAF_FULL, ad);
      if (ad) ord[cnt + __popc(bal & ((1u << lane) - 1u))] = r;
      cnt += __popc(bal);
    }
    if (lane == 0) na_s = cnt;
  }
  __syncthreads();
  const int na = na_s;
  int N = 1;
  while (N < na) N <<= 1;
  for (int i = na + tid; i < N; i += kCtaThreads) ord[i] = -1;  // padding, sorted last
  __syncthreads();
  // bitonic sort of ord[0, N) into the order "a before b"
  for (int size = 2; size <= N; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < (N >> 1); i += kCtaThreads) {
        const int lo = (i / stride) * 2 * stride + (i % stride), hi = lo + stride;
        const int a = ord[lo], b = ord[hi];
        bool b_first;  // b belongs before a
        if (a < 0 || b < 0) {
          b_first = a < 0 && b >= 0;
        } else {
          const K ka = hk[a], kb = hk[b];
          b_first = kb > ka || (kb == ka && b < a);
        }
        if (b_first == ((lo & size) == 0)) {
          ord[lo] = b;
          ord[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    K margin = std::numeric_limits<K>::max();
    int head = 0;
    for (int t = 0; t < s; ++t) {
      while (head < na && pick[ord[head]]) ++head;
      if (head == na) break;  // no admissible row left
      const int rmax = ord[head];
      const K thr = hk[rmax] - K(tau);
      int best = rmax;
      int q = head + 1;
      for (; q < na; ++q) {
        const int r = ord[q];
        if (pick[r]) continue;
        const K h = hk[r];
        margin = dmin(margin, (K)fabs(h - thr));
        if (!(h >= thr)) break;  // the first remaining key below the threshold
        best = r < best ? r : best;
      }
      pick[best] = 1;
    }
    red[0] = (double)margin;
  }
  __syncthreads();
  const double mg = red[0];
  __syncthreads();  // red is free again
  return mg;
}

// The greedy V rule for the CTA kernels: the sorted form where it applies
// (finite keys, tau >= 0), the scan otherwise.  ord as above.
template <class K>
__device__ double cta_select_rows_greedy(const int32_t* rs, const K* hk, int32_t* pick, int m, int rule, int j, int s,
                                         double tau, const int32_t* blk, double* red, int32_t* ord) {
  int bad = !(tau >= 0.0);
  for (int r = threadIdx.x; r < m && !bad; r += kCtaThreads) bad = !isfinite((double)hk[r]);
  if (__syncthreads_or(bad)) return cta_select_rows_w0(rs, hk, pick, m, rule, j, s, tau, blk, red);
  return cta_select_rows_sorted(rs, hk, pick, m, rule, j, s, tau, blk, red, ord);
}

// Gather offsets of the tile's k columns J (warp 0; k <= 64): cst[q] =
// the start of column J[q] of A, coff[q] = the entries of the columns before
// it, *total = all the entries (an exclusive scan by shuffles).
__device__ inline void cta_gather_offsets(const int32_t* Acp, const int32_t* J, int k, int32_t* cst, int32_t* coff,
                                          int32_t* total) {
  if ((threadIdx.x >> 5) != 0) return;
  const int lane = threadIdx.x & 31;
  int e = 0;
  for (int base = 0; base < k; base += 32) {
    const int q = base + lane;
    int st = 0, len = 0;
    if (q < k) {
      const int c = J[q];
      st = Acp[c];
      len = Acp[c + 1] - st;
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(DIAF_FULL, incl, o);
      if (lane >= o) incl += v;
    }
    if (q < k) {
      cst[q] = st;
      coff[q] = e + incl - len;
    }
    e += __shfl_sync(DIAF_FULL, incl, 31);
  }
  if (lane == 0) *total = e;
}

// I_j of a greedy rule (warp 0): the picked rows and j's own row of the
// tile, in row order, with j inserted before the first larger row when it
// is not a row of the tile (jin false).  Writes Is, Iloc (tile row, -1 for
// an inserted j), inI of the listed rows and *jpos (the place of j), as the
// one-thread construction in row order would.
__device__ inline void cta_form_I_greedy(const int32_t* rs, const int32_t* pick, int m, int j, bool jin, int32_t* Is,
                                         int32_t* Iloc, int32_t* inI, int32_t* jpos) {
  if ((threadIdx.x >> 5) != 0) return;
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  if (lane == 0) *jpos = -1;
  __syncwarp();
  int cnt = 0, below = 0;  // rows listed so far; of them, rows < j
  for (int base = 0; base < m; base += 32) {
    const int r = base + lane;
    const int row = r < m ? rs[r] : INT_MAX;
    const bool f = r < m && (pick[r] || row == j);
    const uint32_t bal = __ballot_sync(DIAF_FULL, f);
    const uint32_t bl = __ballot_sync(DIAF_FULL, f && row < j);
    if (f) {
      const int idx = cnt + __popc(bal & lt) + ((!jin && row > j) ? 1 : 0);
      Is[idx] = row;
      Iloc[idx] = r;
      inI[r] = idx;
      if (row == j) *jpos = idx;
    }
    cnt += __popc(bal);
    below += __popc(bl);
  }
  if (!jin && lane == 0) {
    Is[below] = j;
    Iloc[below] = -1;
    *jpos = below;
  }
}

// Householder QR of the m x k tile T (leading dimension ld, global memory):
// the norm of column c by a block reduction, then warp w updates the
// trailing columns q = c+1+w, c+1+w+kCtaWarps, ... (dot product by a warp
// reduction over the rows).
template <class S>
__device__ void cta_householder_qr(S* T, int ld, int m, int k, RealOf<S>* redR, S* bcast) {
  using R = RealOf<S>;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int p = m < k ? m : k;
  for (int c = 0; c < p; ++c) {
    S* tc = T + (size_t)c * ld;
    R part = R(0);
    for (int r = c + tid; r < m; r += kCtaThreads) part += sc_abs2(tc[r]);
    const R nrm2 = block_sum(part, redR);
    if (nrm2 == R(0)) continue;  // uniform
    const S alpha = tc[c];
    const R ax = sc_abs(alpha), nrm = sqrt(nrm2);
    const S ph = sc_unit(alpha);
    const S beta = -(nrm * ph);
    const S u0 = (ax + nrm) * ph;
    const R two_uu = R(1) / (nrm * (nrm + ax));
    for (int q = c + 1 + warp; q < k; q += kCtaWarps) {
      S* tq = T + (size_t)q * ld;
      S d = sc_zero<S>();
      for (int r = c + lane; r < m; r += 32) d += sc_cmul(r == c ? u0 : tc[r], tq[r]);
      const S f = two_uu * warp_sum(d);
      for (int r = c + lane; r < m; r += 32) tq[r] -= f * (r == c ? u0 : tc[r]);
    }
    __syncthreads();
    for (int r = c + tid; r < m; r += kCtaThreads) tc[r] = (r == c) ? beta : sc_zero<S>();
    __syncthreads();
  }
  (void)bcast;
}

// One-sided Jacobi on the p x q matrix G (shared memory, leading dimension
// LDG) with V (q x q, leading dimension LDV): the same rotation as
// warp_jacobi, the q/2 pairs of a round spread over the CTA (LPP threads per
// pair), a barrier between rounds.  PREDICT as for warp_jacobi (callers
// whose result is refined afterwards): no sweep that would only confirm
// convergence after a sweep whose rotations all had |gamma| < sqrt(tol)
// sqrt(alpha beta).
template <class S, int LDG, int LDV, bool PREDICT = false>
__device__ int cta_jacobi(S* G, int p, int q, S* V, RealOf<S>* redR) {
  using R = RealOf<S>;
  constexpr int LPP = kCtaThreads / (kCtaKmax / 2);  // 8 threads per pair
  const int tid = threadIdx.x;
  for (int i = tid; i < q * q; i += kCtaThreads) {
    int r = i % q, c = i / q;
    V[r + c * LDV] = (r == c) ? sc_real_s<S>(R(1)) : sc_zero<S>();
  }
  R part = R(0);
  for (int i = tid; i < p * q; i += kCtaThreads) part += sc_abs2(G[(i % p) + (i / p) * LDG]);
  const R nf2 = block_sum(part, redR);
  const R tol = R(p > 1 ? p : 1) * eps_of<R>();
  const R tol2 = tol * tol;
  const R tiny = tol2 * nf2;
  __syncthreads();
  if (q < 2) return 1;
  const int qq = (q + 1) & ~1;
  const int npairs = qq / 2;
  const int grp = tid / LPP, sub = tid % LPP;
  for (int sweep = 1; sweep <= kMaxSweeps; ++sweep) {
    int rotated = 0;
    int large = 0;  // PREDICT: a rotation with |gamma|^2 >= tol alpha beta
    for (int rnd = 0; rnd < qq - 1; ++rnd) {
      int a = -1, b = -1;
      if (grp < npairs) {
        int pa = grp, pb = qq - 1 - grp;
        a = pa == 0 ? 0 : 1 + (pa - 1 + rnd) % (qq - 1);
        b = 1 + (pb - 1 + rnd) % (qq - 1);
        if (a > b) { int t = a; a = b; b = t; }
        if (b >= q) a = -1;
      }
      const bool act = a >= 0;
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
      const bool rot = act && al > tiny && be > tiny && ag2 > R(0) && ag2 > tol2 * (al * be);
      if (rot) {
        rotated = 1;
        if (PREDICT && ag2 >= tol * (al * be)) large = 1;
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
        const R t = copysign(R(2) * ag, d) / (fabs(d) + sqrt(d * d + R(4) * ag2));
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
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) return sweep;
    if (PREDICT && !__syncthreads_or(large)) return sweep;
  }
  return -1;
}

template <class S>
struct CtaSmem {
  static constexpr int KP = kCtaKmax + 1;  // padded leading dimension of the k x k matrices
  static constexpr size_t bytes(int mcap) {
    return sizeof(S) * (2 * KP * kCtaKmax + 2 * kCtaKmax + mcap + kCtaKmax * KP) +
           sizeof(double) * (mcap + kCtaKmax + 2 * kCtaWarps) + sizeof(int32_t) * (5 * mcap + 2 * kCtaKmax + 8 + 2);
  }
};

// Phase (v_jj real >= 0), residual ||A w_j - v_j|| from its definition (in
// the tile's precision), NaN/Inf check and scatter of column j -- the end of
// every CTA column kernel.  rank_thr: a residual at or below it marks the
// column RANK_DEFICIENT (DIAF-S, where res = ||A-hat w|| = sigma_min).
template <class S>
__device__ void cta_finish(const ColArgs& a, int j, int k, int m, int l, int jpos, const S* Ts, int ld, S* wv, S* vv,
                           const int32_t* Is, const int32_t* Iloc, const int32_t* inI, uint32_t flags, bool do_phase,
                           RealOf<S>* redR, double rank_thr = -1.0) {
  using R = RealOf<S>;
  const int tid = threadIdx.x;
  if (do_phase) {
    S ph = sc_real_s<S>(R(1));
    const R vjj2 = jpos >= 0 ? sc_abs2(vv[jpos]) : R(0);
    R vn2 = R(0);
    for (int t = 0; t < l; ++t) vn2 += sc_abs2(vv[t]);
    const R zl = R(64) * eps_of<R>();
    if (jpos >= 0 && vjj2 > zl * zl * vn2) {
      if constexpr (ScalarInfo<S>::cplx) ph = (R(1) / sqrt(vjj2)) * sc_conj(vv[jpos]);
      else ph = vv[jpos] < R(0) ? sc_real_s<S>(R(-1)) : sc_real_s<S>(R(1));  // v_jj / |v_jj|, exactly
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
    __syncthreads();
    for (int q = tid; q < k; q += kCtaThreads) wv[q] = ph * wv[q];
    for (int t = tid; t < l; t += kCtaThreads) vv[t] = ph * vv[t];
    __syncthreads();
  }
  R r2 = R(0);
  for (int r = tid; r < m; r += kCtaThreads) {
    S s2 = sc_zero<S>();
    for (int q = 0; q < k; ++q) s2 += Ts[r + (size_t)q * ld] * wv[q];
    if (inI[r] >= 0) s2 -= vv[inI[r]];
    r2 += sc_abs2(s2);
  }
  for (int t = tid; t < l; t += kCtaThreads)
    if (Iloc[t] < 0) r2 += sc_abs2(vv[t]);
  r2 = block_sum(r2, redR);
  const double resj = sqrt((double)r2);
  if (resj <= rank_thr) flags |= DIAF_FLAG_RANK_DEFICIENT;
  int bad = !isfinite(resj);
  for (int q = tid; q < k; q += kCtaThreads) bad |= !(isfinite(sc_real(wv[q])) && isfinite(sc_imag(wv[q])));
  for (int t = tid; t < l; t += kCtaThreads) bad |= !(isfinite(sc_real(vv[t])) && isfinite(sc_imag(vv[t])));
  if (__syncthreads_or(bad)) flags |= DIAF_FLAG_NONFINITE;
  S* Wout = reinterpret_cast<S*>(a.Wv) + a.Wcp[j];
  for (int q = tid; q < k; q += kCtaThreads) Wout[q] = wv[q];
  const int v0 = a.Vcp[j];
  S* Vout = reinterpret_cast<S*>(a.Vv) + v0;
  for (int t = tid; t < l; t += kCtaThreads) {
    a.Vri[v0 + t] = Is[t];
    Vout[t] = vv[t];
  }
  if (tid == 0) {
    a.res[j] = resj;
    a.flags[j] = flags | a.extra_flags;
  }
  if (a.Hri) {  // the final I_j to the host: rows, then the column's word
    for (int t = tid; t < l; t += kCtaThreads) a.Hri[v0 + t] = Is[t];
    __threadfence_system();
    __syncthreads();
    if (tid == 0) store_release_sys(a.Hgen + j, a.gen);
  }
  __syncthreads();
}

template <class S, int ALG>
__device__ void solve_column_cta(const ColArgs& a, const CtaScratch& sc, int j, unsigned char* smem) {
  using R = RealOf<S>;
  using L = CtaSmem<S>;
  constexpr int KP = L::KP;
  const int tid = threadIdx.x;
  const int mcap = sc.ldm;
  S* Rs = reinterpret_cast<S*>(smem);   // R of T, then R-hat (KP x KMAX)
  S* Vj = Rs + KP * kCtaKmax;           // Jacobi V
  S* wv = Vj + KP * kCtaKmax;           // w
  S* rinv = wv + kCtaKmax;              // reciprocal diagonal
  S* vv = rinv + kCtaKmax;              // v (mcap)
  S* G = vv + mcap;                     // DIAF-Q: Q_I (l <= 64 rows, KP leading dimension)
  double* hk = reinterpret_cast<double*>(G + kCtaKmax * KP);
  double* sig = hk + mcap;
  double* red = sig + kCtaKmax;         // 2 x kCtaWarps
  int32_t* ibase = reinterpret_cast<int32_t*>(red + 2 * kCtaWarps);
  int32_t* rs = ibase;
  int32_t* inI = rs + mcap;
  int32_t* pick = inI + mcap;
  int32_t* Is = pick + mcap;
  int32_t* Iloc = Is + mcap;
  int32_t* cst = Iloc + mcap;
  int32_t* coff = cst + kCtaKmax;
  int32_t* misc = coff + kCtaKmax;      // [0] jpos, [1] count, [2..] warp counts
  R* redR = reinterpret_cast<R*>(red);

  S* Ts = reinterpret_cast<S*>(sc.slab) + (size_t)blockIdx.x * 2 * sc.ldm * sc.kcap;
  S* Tw = Ts + (size_t)sc.ldm * sc.kcap;
  const int ld = sc.ldm;

  const int k = a.Wcp[j + 1] - a.Wcp[j];
  const int m = a.m[j];
  const int l = a.l[j];
  const int me = m > k ? m : k;
  const int32_t* J = a.Wri + a.Wcp[j];
  const int32_t* Rj = a.rows + a.Eoff[j];
  const S* Av = reinterpret_cast<const S*>(a.Av);
  uint32_t flags = 0;

  // ---- gather
  for (int r = tid; r < mcap; r += kCtaThreads) {
    rs[r] = r < m ? Rj[r] : INT_MAX;
    inI[r] = -1;
    pick[r] = 0;
  }
  for (size_t i = tid; i < (size_t)me * k; i += kCtaThreads) Ts[(i % me) + (i / me) * ld] = sc_zero<S>();
  cta_gather_offsets(a.Acp, J, k, cst, coff, misc + 1);
  __syncthreads();
  const int E = misc[1];
  for (int e = tid; e < E; e += kCtaThreads) {
    int q = upper_bound_i32(coff, k, e) - 1;
    int p = cst[q] + (e - coff[q]);
    int r = lower_bound_i32(rs, m, a.Ari[p]);
    Ts[r + (size_t)q * ld] = Av[p];
  }
  __syncthreads();

  // ---- QR of T, keys, I_j
  if (k > 0) {
    for (size_t i = tid; i < (size_t)me * k; i += kCtaThreads) Tw[(i % me) + (i / me) * ld] = Ts[(i % me) + (i / me) * ld];
    __syncthreads();
    cta_householder_qr<S>(Tw, ld, me, k, redR, nullptr);
    for (int i = tid; i < k * k; i += kCtaThreads) {
      int r = i % k, c = i / k;
      Rs[r + c * KP] = (r <= c) ? Tw[r + (size_t)c * ld] : sc_zero<S>();
    }
    __syncthreads();
  }
  R part = R(0);
  for (int c = tid; c < k; c += kCtaThreads) part = dmax(part, sc_abs(Rs[c + c * KP]));
  const R rdmax = block_max(part, redR);
  const R piv = R(1e-14) * rdmax;
  for (int c = tid; c < k; c += kCtaThreads) rinv[c] = sc_recip_or_zero(Rs[c + c * KP], piv);
  __syncthreads();
  if (k > 0 && (a.rule != DIAF_RULE_FIXED || ALG == DIAF_ALG_Q)) {
    for (int r = tid; r < m; r += kCtaThreads) {  // Q = T R^-1 by rows, into Tw
      R h = R(0);
      for (int c = 0; c < k; ++c) {
        S acc = Ts[r + (size_t)c * ld];
        for (int p2 = 0; p2 < c; ++p2) acc -= Tw[r + (size_t)p2 * ld] * Rs[p2 + c * KP];
        S z = acc * rinv[c];
        Tw[r + (size_t)c * ld] = z;
        h += sc_abs2(z);
      }
      hk[r] = (double)h;
    }
    __syncthreads();
  }
  if (a.rule != DIAF_RULE_FIXED) {
    double* redD = reinterpret_cast<double*>(red);
    cta_select_rows_greedy(rs, hk, pick, m, a.rule, j, l - 1, a.tie_tol, a.blk, redD, Is);  // Is, Iloc: scratch until I_j
  }
  // I_j
  if (a.rule == DIAF_RULE_FIXED) {
    if (tid == 0) {
      misc[0] = -1;
      const int32_t* Vf = a.Vfri + a.Vfcp[j];
      for (int t = 0; t < l; ++t) {
        int row = Vf[t];
        int r = lower_bound_i32(rs, m, row);
        int loc = (r < m && rs[r] == row) ? r : -1;
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
  for (int t = tid; t < l; t += kCtaThreads) vv[t] = sc_zero<S>();
  for (int q = tid; q < k; q += kCtaThreads) wv[q] = sc_zero<S>();
  __syncthreads();

  if (k == 0) {
    flags |= DIAF_FLAG_EMPTY;
    if (ALG == DIAF_ALG_Q) {
      if (tid == 0) vv[jpos >= 0 ? jpos : 0] = sc_real_s<S>(R(1));
      flags |= DIAF_FLAG_DEGENERATE;
    } else {
      flags |= DIAF_FLAG_RANK_DEFICIENT;
    }
    __syncthreads();
  } else if (ALG == DIAF_ALG_S) {
    for (size_t i = tid; i < (size_t)me * k; i += kCtaThreads) {
      int r = i % me, c = i / me;
      Tw[r + (size_t)c * ld] = (r < m && inI[r] >= 0) ? sc_zero<S>() : Ts[r + (size_t)c * ld];
    }
    __syncthreads();
    cta_householder_qr<S>(Tw, ld, me, k, redR, nullptr);
    for (int i = tid; i < k * k; i += kCtaThreads) {
      int r = i % k, c = i / k;
      Rs[r + c * KP] = (r <= c) ? Tw[r + (size_t)c * ld] : sc_zero<S>();
    }
    __syncthreads();
    int sw = cta_jacobi<S, KP, KP>(Rs, k, k, Vj, redR);
    if (sw < 0) flags |= DIAF_FLAG_JACOBI_NOCONV;
    for (int c = tid; c < k; c += kCtaThreads) {
      R s2 = R(0);
      for (int i = 0; i < k; ++i) s2 += sc_abs2(Rs[i + c * KP]);
      sig[c] = sqrt((double)s2);
    }
    __syncthreads();
    int imin = 0;
    double smin = sig[0], smax = sig[0];
    for (int c = 1; c < k; ++c) {
      if (sig[c] < smin) { smin = sig[c]; imin = c; }
      smax = dmax(smax, sig[c]);
    }
    double snext = INFINITY;
    for (int c = 0; c < k; ++c) if (c != imin) snext = dmin(snext, sig[c]);
    int inrows = 0;
    for (int t = 0; t < l; ++t) inrows += (Iloc[t] >= 0);
    if (smin <= 1e-14 * smax || m - inrows < k) flags |= DIAF_FLAG_RANK_DEFICIENT;
    if (k > 1 && (snext - smin) <= 1e-6 * smax) flags |= DIAF_FLAG_DEGENERATE;
    for (int q = tid; q < k; q += kCtaThreads) wv[q] = Vj[q + imin * KP];
    __syncthreads();
    for (int t = tid; t < l; t += kCtaThreads) {
      S s2 = sc_zero<S>();
      int r = Iloc[t];
      if (r >= 0)
        for (int q = 0; q < k; ++q) s2 += Ts[r + (size_t)q * ld] * wv[q];
      vv[t] = s2;
    }
    __syncthreads();
  } else {
    // DIAF-Q: Q_I (rows I_j of Q, in Tw) into G, Jacobi, v, w = sigma R^-1 u
    for (int i = tid; i < l * k; i += kCtaThreads) {
      int t = i % l, c = i / l;
      int r = Iloc[t];
      G[t + c * KP] = r >= 0 ? Tw[r + (size_t)c * ld] : sc_zero<S>();
    }
    __syncthreads();
    int sw = cta_jacobi<S, KP, KP>(G, l, k, Vj, redR);
    if (sw < 0) flags |= DIAF_FLAG_JACOBI_NOCONV;
    for (int c = tid; c < k; c += kCtaThreads) {
      R s2 = R(0);
      for (int i = 0; i < l; ++i) s2 += sc_abs2(G[i + c * KP]);
      sig[c] = sqrt((double)s2);
    }
    __syncthreads();
    int imax = 0;
    double smax = sig[0];
    for (int c = 1; c < k; ++c) if (sig[c] > smax) { smax = sig[c]; imax = c; }
    double snext = 0.0;
    for (int c = 0; c < k; ++c) if (c != imax) snext = dmax(snext, sig[c]);
    if (smax == 0.0 || (k > 1 && (smax - snext) <= 1e-6 * smax)) flags |= DIAF_FLAG_DEGENERATE;
    if (smax > 0.0) {
      const R inv = R(1) / R(smax);
      for (int t = tid; t < l; t += kCtaThreads) vv[t] = inv * G[t + imax * KP];
    } else if (tid == 0) {
      vv[jpos >= 0 ? jpos : 0] = sc_real_s<S>(R(1));
    }
    bool rd = false;
    for (int c = 0; c < k; ++c) rd |= !(sc_abs(Rs[c + c * KP]) > piv);
    if (rd) flags |= DIAF_FLAG_RANK_DEFICIENT;
    __syncthreads();
    const bool stab = a.stab_tol > 0.0 && jpos >= 0 && l > 1 && (double)sc_abs(vv[jpos]) < a.stab_tol;
    if (stab) {
      // Stabilised DIAF-Q (Sec. 3.2), as in the warp kernel: G = Q_I V1; drop
      // row j, Jacobi of the rest gives z = B Y(:,1)/s_1 and the phase from
      // conj(sum_c Y(c,1) q_c), q = row j of Q_I V1; v = (r e_j + e^{i theta} z)
      // / sqrt(r^2 + 1); the right-hand side of eq. condwj is R^-* T_I^* v.
      for (int q = tid; q < k; q += kCtaThreads) wv[q] = G[jpos + q * KP];
      __syncthreads();
      for (int c = tid; c < k; c += kCtaThreads)
        for (int t = jpos; t < l - 1; ++t) G[t + c * KP] = G[t + 1 + c * KP];
      __syncthreads();
      const int lh = l - 1;
      if (cta_jacobi<S, KP, KP>(G, lh, k, Vj, redR) < 0) flags |= DIAF_FLAG_JACOBI_NOCONV;
      for (int c = tid; c < k; c += kCtaThreads) {
        R s2 = R(0);
        for (int i = 0; i < lh; ++i) s2 += sc_abs2(G[i + c * KP]);
        sig[c] = sqrt((double)s2);
      }
      __syncthreads();
      int i1 = 0;
      double s1 = sig[0];
      for (int c = 1; c < k; ++c) if (sig[c] > s1) { s1 = sig[c]; i1 = c; }
      double sn = 0.0;
      for (int c = 0; c < k; ++c) if (c != i1) sn = dmax(sn, sig[c]);
      flags &= ~DIAF_FLAG_DEGENERATE;
      if (s1 == 0.0 || (lh > 1 && k > 1 && (s1 - sn) <= 1e-6 * s1)) flags |= DIAF_FLAG_DEGENERATE;
      S pt = sc_zero<S>();
      R pn = R(0);
      for (int q = 0; q < k; ++q) {  // every thread: a uniform result without another reduction
        pt += Vj[q + i1 * KP] * wv[q];
        pn += sc_abs2(wv[q]);
      }
      pt = sc_conj(pt);
      const R apt = sc_abs(pt);
      if (!(apt > R(1e-10) * sqrt(pn))) flags |= DIAF_FLAG_DEGENERATE;
      const S eth = apt > R(0) ? (R(1) / apt) * pt : sc_real_s<S>(R(1));
      const R r = a.stab_r > 0.0 ? R(a.stab_r) : R(2);
      const R scl = R(1) / sqrt(r * r + R(1));
      const R zs = s1 > 0.0 ? scl / R(s1) : R(0);
      for (int u = tid; u < lh; u += kCtaThreads) vv[u < jpos ? u : u + 1] = (zs * eth) * G[u + i1 * KP];
      if (tid == 0) vv[jpos] = sc_real_s<S>(r * scl);
      __syncthreads();
      for (int c = tid; c < k; c += kCtaThreads) {  // T_I^* v
        S y = sc_zero<S>();
        for (int t = 0; t < l; ++t)
          if (Iloc[t] >= 0) y += sc_conj(Ts[Iloc[t] + (size_t)c * ld]) * vv[t];
        wv[c] = y;
      }
      __syncthreads();
      flags |= DIAF_FLAG_STABILISED;
    }
    if (tid == 0) {  // R w = Q_I^* v: sigma u, or R^-* T_I^* v when stabilised
      if (stab) {
        for (int c = 0; c < k; ++c) {
          S acc = wv[c];
          for (int p = 0; p < c; ++p) acc -= sc_conj(Rs[p + c * KP]) * wv[p];
          wv[c] = acc * sc_conj(rinv[c]);
        }
      } else {
        for (int c = 0; c < k; ++c) wv[c] = R(smax) * Vj[c + imax * KP];
      }
      for (int c = k - 1; c >= 0; --c) {
        S acc = wv[c];
        for (int t = c + 1; t < k; ++t) acc -= Rs[c + t * KP] * wv[t];
        wv[c] = acc * rinv[c];
      }
    }
    __syncthreads();
  }

  cta_finish<S>(a, j, k, m, l, jpos, Ts, ld, wv, vv, Is, Iloc, inI, flags, k > 0 || ALG == DIAF_ALG_Q, redR);
}

template <class S, int ALG>
__global__ void __launch_bounds__(kCtaThreads) column_cta_kernel(ColArgs a, CtaScratch sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int idx_s;
  const int count = *a.list_count;
  while (true) {
    if (threadIdx.x == 0) idx_s = atomicAdd(a.work_counter, 1);
    __syncthreads();
    const int idx = idx_s;
    __syncthreads();
    if (idx >= count) break;
    solve_column_cta<S, ALG>(a, sc, list_at(a, count, idx), smem_raw);
  }
}
