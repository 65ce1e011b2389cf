/*
 * diaf_oracle.c -- plain CPU oracle for the columnwise construction of W, V
 * with AW ~ V (Byckling & Huhtanen, "Preconditioning with direct approximate
 * factoring of the inverse").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call
 * this file: it exists so that tests, smoke checks and the CPU-baseline leg
 * of the benchmark can check the CUDA library against an obviously correct,
 * independent restatement of the method.  It shares no code with the CUDA
 * path.
 *
 * Everything is complex128 (`double complex`); real problems are the special
 * case with zero imaginary parts (every operation below keeps them exactly
 * zero).  Per column j (Sec. 2, "standard matrix subspaces", columns are
 * independent):
 *
 *   1. R_j = sorted union of the row indices of A(:,c), c in J_j, and the
 *      dense tile T = A(R_j, J_j)  (A_j of eq. spaqr restricted to its
 *      nonzero rows; Sec. 2.1).
 *   2. Householder QR T = Q R (thin), eq. spaqr.
 *   3. Leverage h_i = ||Q(i,:)||^2 = squared norm of the i-th column of Q_j^*
 *      (Sec. 3.1: choose the l_j admissible columns of Q_j^* of largest
 *      norm).
 *   4. I_j: a fixed pattern column, or {j} plus the l_j - 1 admissible rows
 *      of largest leverage (greedy, ties within tie_tol to the lower row).
 *   5a. DIAF-S (Sec. 2.2): A_hat = T with the rows I_j removed;
 *       A_hat = Q' R' (Householder), one-sided Jacobi SVD of R';
 *       w_j = right singular vector of the smallest singular value,
 *       v_j = (A w_j) restricted to I_j (V = P_V A W).
 *   5b. DIAF-Q (Sec. 2.1): M_j = Q(I_j,:)^* (k x l); v_j = top right singular
 *       vector of M_j (eq. nocond), via one-sided Jacobi; w_j solves the
 *       least-squares problem eq. condwj, R w = Q^* v = M_j v.
 *   5c. Stabilised DIAF-Q (Sec. 3.2, optional): when |v_jj| < stab_tol
 *       (v_j of unit norm), the j-th component is imposed as r > 0 and the
 *       rest is taken from the SVD of M_hat = the columns of M_j other than
 *       j: v_hat = e^{i theta} z, z its top right singular vector, theta the
 *       argument of the first component of U_hat^* p (p = column j of M_j);
 *       v_j = r e_j + v_hat, scaled to unit norm; w_j from eq. condwj as
 *       before.  Flag STABILISED (and DEGENERATE where z or theta is not
 *       unique).
 *   6. Phase: scale (w_j, v_j) by a unit scalar so that v_jj is real >= 0
 *      (allowed by the scaling-invariance theorem of Sec. 2.1).  When v_jj is
 *      zero to rounding (|v_jj| <= 64 eps ||v_j||) the flag VJJ_ZERO is set
 *      and the largest-modulus entry of w_j is made real instead.
 *   7. res_j = ||A w_j - v_j||_2, computed from its definition.
 *
 * Jacobi SVD: cyclic one-sided (Hestenes) Jacobi, rotation when
 * |g_a^* g_b| > p*eps*sqrt(|g_a|^2 |g_b|^2) and neither column is below
 * p*eps*||g||_F, at most 30 sweeps.
 */
#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex zd;

enum { RULE_FIXED = 0, RULE_UPPER = 1, RULE_LOWER = 2, RULE_ALL = 3, RULE_BLOCK = 4 };
enum { ALG_Q = 1, ALG_S = 2 };
enum {
    F_RANK_DEFICIENT = 1u, F_DEGENERATE = 2u, F_VJJ_ZERO = 4u,
    F_JACOBI_NOCONV = 8u, F_NONFINITE = 16u, F_EMPTY = 32u, F_STABILISED = 128u
};
#define MAX_SWEEPS 30

static double abs2(zd z) { double a = creal(z), b = cimag(z); return a * a + b * b; }

static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* index of key in sorted rows[0..m), or -1 */
static int find_row(const int *rows, int m, int key) {
    int lo = 0, hi = m - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (rows[mid] == key) return mid;
        if (rows[mid] < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* ---------------------------------------------------------------- QR ---- */
/* Householder QR of the column-major m x k matrix a (ld m), overwritten.
 * Reflector c: H_c = I - 2 u u^* / (u^* u) acting on rows c..m-1, with
 * u = x - beta e_1, beta = -(x_0/|x_0|) ||x||, so H_c x = beta e_1.
 * On return r (k x k, ld k) holds R (rows beyond m are zero when m < k) and,
 * if q != NULL, q (m x min(m,k), ld m) holds the thin Q = H_0 ... H_{p-1} [I;0]. */
static void householder_qr(int m, int k, zd *a, zd *r, zd *q) {
    int p = m < k ? m : k;
    zd *u = (zd *)calloc((size_t)m * (p > 0 ? p : 1), sizeof(zd));
    double *uu = (double *)calloc(p > 0 ? p : 1, sizeof(double));
    for (int c = 0; c < p; ++c) {
        double nrm2 = 0.0;
        for (int i = c; i < m; ++i) nrm2 += abs2(a[i + (size_t)c * m]);
        zd *uc = u + (size_t)c * m;
        if (nrm2 == 0.0) { uu[c] = 0.0; continue; }
        zd x0 = a[c + (size_t)c * m];
        double ax0 = cabs(x0);
        zd ph = ax0 > 0.0 ? x0 / ax0 : 1.0;
        zd beta = -ph * sqrt(nrm2);
        for (int i = c; i < m; ++i) uc[i] = a[i + (size_t)c * m];
        uc[c] = x0 - beta;
        double s2 = 0.0;
        for (int i = c; i < m; ++i) s2 += abs2(uc[i]);
        uu[c] = s2;
        for (int col = c; col < k; ++col) {
            zd *ac = a + (size_t)col * m;
            zd s = 0.0;
            for (int i = c; i < m; ++i) s += conj(uc[i]) * ac[i];
            zd f = 2.0 * s / s2;
            for (int i = c; i < m; ++i) ac[i] -= f * uc[i];
        }
    }
    for (int col = 0; col < k; ++col)
        for (int i = 0; i < k; ++i)
            r[i + (size_t)col * k] = (i <= col && i < m) ? a[i + (size_t)col * m] : 0.0;
    if (q) {
        for (int col = 0; col < p; ++col)
            for (int i = 0; i < m; ++i) q[i + (size_t)col * m] = (i == col) ? 1.0 : 0.0;
        for (int c = p - 1; c >= 0; --c) {
            if (uu[c] == 0.0) continue;
            zd *uc = u + (size_t)c * m;
            for (int col = 0; col < p; ++col) {
                zd *qc = q + (size_t)col * m;
                zd s = 0.0;
                for (int i = c; i < m; ++i) s += conj(uc[i]) * qc[i];
                zd f = 2.0 * s / uu[c];
                for (int i = c; i < m; ++i) qc[i] -= f * uc[i];
            }
        }
    }
    free(u); free(uu);
}

/* ------------------------------------------------------- Jacobi SVD ---- */
/* One-sided Jacobi on the column-major p x q matrix g (ld p): finds a unitary
 * V (q x q, ld q) with g V = U diag(sigma) and orthogonal columns.
 * sigma[i] = ||(g V)(:,i)||.  Returns the number of sweeps used, or -1 if
 * MAX_SWEEPS did not reach the tolerance. */
static int jacobi_svd(int p, int q, zd *g, zd *v, double *sigma) {
    for (int i = 0; i < q; ++i)
        for (int t = 0; t < q; ++t) v[t + (size_t)i * q] = (t == i) ? 1.0 : 0.0;
    double tol = (p > 1 ? p : 1) * DBL_EPSILON;
    /* A column whose norm is below p*eps*||g||_F is numerically zero: it is
     * not rotated against (otherwise its rounding residue keeps rotating). */
    double nf2 = 0.0;
    for (size_t i = 0; i < (size_t)p * q; ++i) nf2 += abs2(g[i]);
    double tiny = tol * tol * nf2;
    int sweep, conv = 0;
    for (sweep = 0; sweep < MAX_SWEEPS && !conv; ++sweep) {
        conv = 1;
        for (int a = 0; a < q - 1; ++a) {
            for (int b = a + 1; b < q; ++b) {
                zd *ga = g + (size_t)a * p, *gb = g + (size_t)b * p;
                double alpha = 0.0, beta = 0.0;
                zd gamma = 0.0;
                for (int i = 0; i < p; ++i) {
                    alpha += abs2(ga[i]);
                    beta += abs2(gb[i]);
                    gamma += conj(ga[i]) * gb[i];
                }
                double ag = cabs(gamma);
                if (alpha <= tiny || beta <= tiny) continue;
                if (ag == 0.0 || ag <= tol * sqrt(alpha * beta)) continue;
                conv = 0;
                /* b' = e^{-i phi} b makes a^* b' = |gamma| real, then a real
                 * rotation [a b'] [[c, s], [-s, c]] orthogonalises the pair:
                 * t = s/c is the smaller root of t^2 + 2 zeta t - 1 = 0. */
                zd eph = conj(gamma) / ag;
                double zeta = (beta - alpha) / (2.0 * ag);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < p; ++i) {
                    zd x = ga[i], y = eph * gb[i];
                    ga[i] = c * x - s * y;
                    gb[i] = s * x + c * y;
                }
                zd *va = v + (size_t)a * q, *vb = v + (size_t)b * q;
                for (int i = 0; i < q; ++i) {
                    zd x = va[i], y = eph * vb[i];
                    va[i] = c * x - s * y;
                    vb[i] = s * x + c * y;
                }
            }
        }
    }
    for (int i = 0; i < q; ++i) {
        double s2 = 0.0;
        for (int t = 0; t < p; ++t) s2 += abs2(g[t + (size_t)i * p]);
        sigma[i] = sqrt(s2);
    }
    return conv ? sweep : -1;
}

/* ------------------------------------------------------ column plan ---- */
typedef struct {
    int m;        /* |R_j| */
    int *rows;    /* R_j sorted, owned */
} rowset;

static rowset row_union(const int *Acp, const int *Ari, const int *Jr, int k) {
    int tot = 0;
    for (int q = 0; q < k; ++q) tot += Acp[Jr[q] + 1] - Acp[Jr[q]];
    int *buf = (int *)malloc(sizeof(int) * (tot > 0 ? tot : 1));
    int e = 0;
    for (int q = 0; q < k; ++q)
        for (int p = Acp[Jr[q]]; p < Acp[Jr[q] + 1]; ++p) buf[e++] = Ari[p];
    qsort(buf, tot, sizeof(int), cmp_int);
    int m = 0;
    for (int i = 0; i < tot; ++i)
        if (m == 0 || buf[i] != buf[m - 1]) buf[m++] = buf[i];
    rowset rs = {m, buf};
    return rs;
}

/* Admissible rows of column j: upper (i < j) or lower (i > j) triangular V
 * (the Gauss-Seidel structures of Sec. 4.2), any row, or the rows of j's
 * diagonal block (block-diagonal V, the structure of Sec. 5's experiments). */
static int admissible(int rule, int i, int j, const int *blk) {
    if (i == j) return 0; /* the diagonal is always in I_j, never a candidate */
    if (rule == RULE_UPPER) return i < j;
    if (rule == RULE_LOWER) return i > j;
    if (rule == RULE_BLOCK) return blk[i] == blk[j];
    return 1;
}

static int n_candidates(const rowset *rs, int rule, int j, const int *blk) {
    int c = 0;
    for (int i = 0; i < rs->m; ++i) c += admissible(rule, rs->rows[i], j, blk);
    return c;
}

static int extra_count(int ncand, const int *budget, int j) {
    int s = budget ? budget[j] - 1 : ncand;
    if (s < 0) s = 0;
    if (s > ncand) s = ncand;
    return s;
}

/* Greedy selection of s candidates by leverage: at each pick, among the
 * remaining candidates whose leverage is within tie_tol of the largest, take
 * the lowest row.  *margin receives the smallest distance of any remaining
 * candidate's key (other than the current maximum itself) to a pick
 * threshold: how close a decision came to flipping under rounding. */
static void select_rows(const rowset *rs, const double *h, int rule, int j, int s,
                        double tie_tol, int *picked, double *margin, const int *blk) {
    int m = rs->m;
    char *used = (char *)calloc(m > 0 ? m : 1, 1);
    double mg = INFINITY;
    for (int t = 0; t < s; ++t) {
        double hmax = -INFINITY;
        for (int i = 0; i < m; ++i)
            if (!used[i] && admissible(rule, rs->rows[i], j, blk) && h[i] > hmax) hmax = h[i];
        double thr = hmax - tie_tol;
        int best = -1;
        for (int i = 0; i < m; ++i) {
            if (used[i] || !admissible(rule, rs->rows[i], j, blk)) continue;
            double d = fabs(h[i] - thr);
            if (h[i] != hmax && d < mg) mg = d;
            if (best < 0 && h[i] >= thr) best = i;
        }
        used[best] = 1;
        picked[t] = rs->rows[best];
    }
    free(used);
    *margin = mg;
}

/* ---------------------------------------------------- one column ---- */
typedef struct {
    /* problem */
    int n;
    const int *Acp, *Ari;
    const zd *Av;
    const int *Wcp, *Wri;
    int rule;
    const int *Vcp, *Vri, *budget;
    const int *blk;           /* RULE_BLOCK: block of every row */
    int alg;
    double tie_tol;
    double stab_tol, stab_r;  /* stabilised DIAF-Q: trigger |v_jj| < stab_tol (0: off), imposed v_jj = r */
} problem;

typedef struct {
    zd *w;          /* k_j, at W's slots */
    int *Irows;     /* l_j */
    zd *v;          /* l_j */
    double res, margin, sig_sel, sig_next;
    unsigned flags;
} colout;

static int count_l(const problem *P, int j) {
    if (P->rule == RULE_FIXED) return P->Vcp[j + 1] - P->Vcp[j];
    const int *Jr = P->Wri + P->Wcp[j];
    int k = P->Wcp[j + 1] - P->Wcp[j];
    rowset rs = row_union(P->Acp, P->Ari, Jr, k);
    int s = extra_count(n_candidates(&rs, P->rule, j, P->blk), P->budget, j);
    free(rs.rows);
    return 1 + s;
}

/* Computes column j; `out` arrays sized k_j and l_j (l_j from count_l). */
static void solve_column(const problem *P, int j, colout *out, double *h_dbg, int *rows_dbg, int *m_dbg) {
    const int *Jr = P->Wri + P->Wcp[j];
    int k = P->Wcp[j + 1] - P->Wcp[j];
    rowset rs = row_union(P->Acp, P->Ari, Jr, k);
    int m = rs.m;
    unsigned flags = 0;
    out->margin = INFINITY;
    out->sig_sel = out->sig_next = 0.0;

    /* 1. tile T = A(R_j, J_j), column-major m x k */
    zd *T = (zd *)calloc((size_t)m * k + 1, sizeof(zd));
    for (int q = 0; q < k; ++q) {
        int c = Jr[q];
        for (int p = P->Acp[c]; p < P->Acp[c + 1]; ++p)
            T[find_row(rs.rows, m, P->Ari[p]) + (size_t)q * m] = P->Av[p];
    }

    /* 2-3. QR of T and leverage */
    int pq = m < k ? m : k;
    zd *Ra = (zd *)calloc((size_t)k * k + 1, sizeof(zd));
    zd *Q = (zd *)calloc((size_t)m * (pq > 0 ? pq : 1) + 1, sizeof(zd));
    zd *Tc = (zd *)malloc(sizeof(zd) * ((size_t)m * k + 1));
    memcpy(Tc, T, sizeof(zd) * (size_t)m * k);
    householder_qr(m, k, Tc, Ra, Q);
    double *h = (double *)calloc(m + 1, sizeof(double));
    for (int i = 0; i < m; ++i)
        for (int c = 0; c < pq; ++c) h[i] += abs2(Q[i + (size_t)c * m]);
    if (h_dbg) { memcpy(h_dbg, h, sizeof(double) * m); memcpy(rows_dbg, rs.rows, sizeof(int) * m); *m_dbg = m; }

    /* 4. I_j */
    int l;
    if (P->rule == RULE_FIXED) {
        l = P->Vcp[j + 1] - P->Vcp[j];
        memcpy(out->Irows, P->Vri + P->Vcp[j], sizeof(int) * l);
    } else {
        int s = extra_count(n_candidates(&rs, P->rule, j, P->blk), P->budget, j);
        l = 1 + s;
        out->Irows[0] = j;
        select_rows(&rs, h, P->rule, j, s, P->tie_tol, out->Irows + 1, &out->margin, P->blk);
        qsort(out->Irows, l, sizeof(int), cmp_int);
    }
    int *Iloc = (int *)malloc(sizeof(int) * (l + 1));
    char *inI = (char *)calloc(m + 1, 1);
    for (int t = 0; t < l; ++t) {
        Iloc[t] = find_row(rs.rows, m, out->Irows[t]);
        if (Iloc[t] >= 0) inI[Iloc[t]] = 1;
    }
    int jpos = -1;
    for (int t = 0; t < l; ++t) if (out->Irows[t] == j) jpos = t;

    zd *w = out->w, *v = out->v;
    for (int t = 0; t < l; ++t) v[t] = 0.0;

    if (k == 0) {
        flags |= F_EMPTY;
        if (P->alg == ALG_Q && l > 0) { v[jpos >= 0 ? jpos : 0] = 1.0; flags |= F_DEGENERATE; }
        else flags |= F_RANK_DEFICIENT;
    } else if (P->alg == ALG_S) {
        /* 5a. DIAF-S: QR of A_hat then SVD of its R factor */
        int mh = 0;
        for (int i = 0; i < m; ++i) mh += !inI[i];
        int mr = mh > k ? mh : k;
        zd *Ah = (zd *)calloc((size_t)mr * k + 1, sizeof(zd));
        for (int q = 0; q < k; ++q) {
            int r = 0;
            for (int i = 0; i < m; ++i)
                if (!inI[i]) Ah[r++ + (size_t)q * mr] = T[i + (size_t)q * m];
        }
        zd *Rh = (zd *)calloc((size_t)k * k + 1, sizeof(zd));
        householder_qr(mr, k, Ah, Rh, NULL);
        zd *Vj = (zd *)malloc(sizeof(zd) * ((size_t)k * k + 1));
        double *sg = (double *)malloc(sizeof(double) * (k + 1));
        if (jacobi_svd(k, k, Rh, Vj, sg) < 0) flags |= F_JACOBI_NOCONV;
        int imin = 0;
        double smax = sg[0];
        for (int i = 1; i < k; ++i) { if (sg[i] < sg[imin]) imin = i; if (sg[i] > smax) smax = sg[i]; }
        double snext = INFINITY;
        for (int i = 0; i < k; ++i) if (i != imin && sg[i] < snext) snext = sg[i];
        out->sig_sel = sg[imin];
        out->sig_next = k > 1 ? snext : sg[imin];
        if (sg[imin] <= 1e-14 * smax || mh < k) flags |= F_RANK_DEFICIENT;
        if (k > 1 && (snext - sg[imin]) <= 1e-6 * smax) flags |= F_DEGENERATE;
        for (int q = 0; q < k; ++q) w[q] = Vj[q + (size_t)imin * k];
        /* v_j = P_V (A w_j): the tile rows in I_j */
        for (int t = 0; t < l; ++t) {
            zd s = 0.0;
            if (Iloc[t] >= 0)
                for (int q = 0; q < k; ++q) s += T[Iloc[t] + (size_t)q * m] * w[q];
            v[t] = s;
        }
        free(Ah); free(Rh); free(Vj); free(sg);
    } else {
        /* 5b. DIAF-Q: M_j = Q(I_j,:)^*, k x l; top right singular vector */
        zd *M = (zd *)calloc((size_t)k * l + 1, sizeof(zd));
        for (int t = 0; t < l; ++t)
            if (Iloc[t] >= 0)
                for (int c = 0; c < pq; ++c) M[c + (size_t)t * k] = conj(Q[Iloc[t] + (size_t)c * m]);
        zd *Mc = (zd *)malloc(sizeof(zd) * ((size_t)k * l + 1));
        memcpy(Mc, M, sizeof(zd) * (size_t)k * l);
        zd *Vm = (zd *)malloc(sizeof(zd) * ((size_t)l * l + 1));
        double *sg = (double *)malloc(sizeof(double) * (l + 1));
        if (jacobi_svd(k, l, Mc, Vm, sg) < 0) flags |= F_JACOBI_NOCONV;
        int imax = 0;
        for (int i = 1; i < l; ++i) if (sg[i] > sg[imax]) imax = i;
        double snext = -INFINITY;
        for (int i = 0; i < l; ++i) if (i != imax && sg[i] > snext) snext = sg[i];
        out->sig_sel = sg[imax];
        out->sig_next = l > 1 ? snext : 0.0;
        if (sg[imax] == 0.0 || (l > 1 && (sg[imax] - snext) <= 1e-6 * sg[imax])) flags |= F_DEGENERATE;
        for (int t = 0; t < l; ++t) v[t] = Vm[t + (size_t)imax * l];
        /* 5c. stabilisation (Sec. 3.2): v_jj too small -> impose it */
        if (P->stab_tol > 0.0 && jpos >= 0 && l > 1 && cabs(v[jpos]) < P->stab_tol) {
            int lh = l - 1;
            zd *Mh = (zd *)malloc(sizeof(zd) * ((size_t)k * lh + 1));
            for (int t = 0, u = 0; t < l; ++t) {
                if (t == jpos) continue;
                for (int c = 0; c < k; ++c) Mh[c + (size_t)u * k] = M[c + (size_t)t * k];
                ++u;
            }
            zd *Vh = (zd *)malloc(sizeof(zd) * ((size_t)lh * lh + 1));
            double *sh = (double *)malloc(sizeof(double) * (lh + 1));
            /* one-sided Jacobi on M_hat: its columns become U_hat Sigma_hat, Vh = V_hat */
            if (jacobi_svd(k, lh, Mh, Vh, sh) < 0) flags |= F_JACOBI_NOCONV;
            int i1 = 0;
            for (int i = 1; i < lh; ++i) if (sh[i] > sh[i1]) i1 = i;
            double s2 = -INFINITY;
            for (int i = 0; i < lh; ++i) if (i != i1 && sh[i] > s2) s2 = sh[i];
            /* the DEGENERATE flag now describes the stabilised problem */
            flags &= ~F_DEGENERATE;
            if (sh[i1] == 0.0 || (lh > 1 && (sh[i1] - s2) <= 1e-6 * sh[i1])) flags |= F_DEGENERATE;
            /* first component of U_hat^* p, U_hat(:,1) = M_hat(:,i1) / sigma_1 */
            zd pt = 0.0;
            for (int c = 0; c < k; ++c) pt += conj(Mh[c + (size_t)i1 * k]) * M[c + (size_t)jpos * k];
            /* p_tilde_1 = 0: every theta gives the same objective (the paper: any
             * theta will do); theta = 0 is taken and the column is DEGENERATE */
            double pn = 0.0;
            for (int c = 0; c < k; ++c) pn += abs2(M[c + (size_t)jpos * k]);
            if (cabs(pt) <= 1e-10 * sh[i1] * sqrt(pn)) flags |= F_DEGENERATE;
            zd eth = cabs(pt) > 0.0 ? pt / cabs(pt) : 1.0;
            double r = P->stab_r > 0.0 ? P->stab_r : 2.0;
            double sc = 1.0 / sqrt(r * r + 1.0);
            for (int t = 0, u = 0; t < l; ++t) {
                if (t == jpos) { v[t] = r * sc; continue; }
                v[t] = sc * eth * Vh[u + (size_t)i1 * lh];
                ++u;
            }
            out->sig_sel = sh[i1];
            out->sig_next = lh > 1 ? s2 : 0.0;
            flags |= F_STABILISED;
            free(Mh); free(Vh); free(sh);
        }
        /* eq. condwj: R w = Q^* v_full = M v */
        zd *z = (zd *)calloc(k + 1, sizeof(zd));
        for (int c = 0; c < k; ++c)
            for (int t = 0; t < l; ++t) z[c] += M[c + (size_t)t * k] * v[t];
        double rmax = 0.0;
        for (int c = 0; c < k; ++c) if (cabs(Ra[c + (size_t)c * k]) > rmax) rmax = cabs(Ra[c + (size_t)c * k]);
        for (int c = k - 1; c >= 0; --c) {
            zd s = z[c];
            for (int t = c + 1; t < k; ++t) s -= Ra[c + (size_t)t * k] * w[t];
            zd d = Ra[c + (size_t)c * k];
            if (cabs(d) <= 1e-14 * rmax) { flags |= F_RANK_DEFICIENT; w[c] = 0.0; }
            else w[c] = s / d;
        }
        free(M); free(Mc); free(Vm); free(sg); free(z);
    }

    /* 6. phase: v_jj real and >= 0 */
    if (k > 0 || P->alg == ALG_Q) {
        zd ph = 1.0;
        double vjj = jpos >= 0 ? cabs(v[jpos]) : 0.0;
        double vn2 = 0.0;
        for (int t = 0; t < l; ++t) vn2 += abs2(v[t]);
        /* v_jj counts as zero below the rounding level of the column */
        if (jpos >= 0 && vjj > 64.0 * DBL_EPSILON * sqrt(vn2)) {
            ph = conj(v[jpos]) / vjj;
        } else {
            flags |= F_VJJ_ZERO;
            int imx = -1;
            double amx = 0.0;
            for (int q = 0; q < k; ++q) if (cabs(w[q]) > amx) { amx = cabs(w[q]); imx = q; }
            if (imx >= 0) ph = conj(w[imx]) / amx;
        }
        for (int q = 0; q < k; ++q) w[q] *= ph;
        for (int t = 0; t < l; ++t) v[t] *= ph;
    }

    /* 7. res_j = ||A_j w_j - v_j|| over all rows */
    double r2 = 0.0;
    for (int i = 0; i < m; ++i) {
        zd s = 0.0;
        for (int q = 0; q < k; ++q) s += T[i + (size_t)q * m] * w[q];
        for (int t = 0; t < l; ++t) if (Iloc[t] == i) s -= v[t];
        r2 += abs2(s);
    }
    for (int t = 0; t < l; ++t) if (Iloc[t] < 0) r2 += abs2(v[t]);
    out->res = sqrt(r2);

    int finite = isfinite(out->res);
    for (int q = 0; q < k; ++q) finite &= isfinite(creal(w[q])) && isfinite(cimag(w[q]));
    for (int t = 0; t < l; ++t) finite &= isfinite(creal(v[t])) && isfinite(cimag(v[t]));
    if (!finite) flags |= F_NONFINITE;
    out->flags = flags;

    free(T); free(Ra); free(Q); free(Tc); free(h); free(Iloc); free(inI); free(rs.rows);
}

/* ------------------------------------------------------------ ABI ---- */
static problem make_problem(int n, const int *Acp, const int *Ari, const double *Av,
                            const int *Wcp, const int *Wri, int rule, const int *Vcp,
                            const int *Vri, const int *budget, const int *blk, int alg, double tie_tol,
                            double stab_tol, double stab_r) {
    problem P = {n, Acp, Ari, (const zd *)Av, Wcp, Wri, rule, Vcp, Vri, budget, blk, alg, tie_tol, stab_tol, stab_r};
    return P;
}

/* l_j for each listed column (cols == NULL: all n columns). */
int diaf_oracle_vcount(int n, const int *Acp, const int *Ari, const int *Wcp, const int *Wri,
                       int rule, const int *Vcp, const int *Vri, const int *budget, const int *blk,
                       int ncols, const int *cols, int *lcount, int nthreads) {
    problem P = make_problem(n, Acp, Ari, NULL, Wcp, Wri, rule, Vcp, Vri, budget, blk, ALG_S, 0.0, 0.0, 0.0);
    if (nthreads <= 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
    for (int t = 0; t < ncols; ++t) lcount[t] = count_l(&P, cols ? cols[t] : t);
    return 0;
}

/* Columns cols[0..ncols) (NULL: all).  A values interleaved (re, im).
 * Outputs: Wv interleaved at W's slots Wcp[j]..; Vri/Vv at voff[t]..voff[t]+l;
 * res, flags, margin, sig (2 per column) indexed by t. */
int diaf_oracle_factor(int n, const int *Acp, const int *Ari, const double *Av,
                       const int *Wcp, const int *Wri, int rule, const int *Vcp,
                       const int *Vri, const int *budget, const int *blk, int alg, double tie_tol,
                       double stab_tol, double stab_r,
                       int ncols, const int *cols, const long long *voff,
                       double *Wv, int *Vri_out, double *Vv, double *res,
                       unsigned *flags, double *margin, double *sig, int nthreads) {
    problem P = make_problem(n, Acp, Ari, Av, Wcp, Wri, rule, Vcp, Vri, budget, blk, alg, tie_tol, stab_tol, stab_r);
    if (nthreads <= 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
    for (int t = 0; t < ncols; ++t) {
        int j = cols ? cols[t] : t;
        colout o;
        o.w = (zd *)Wv + Wcp[j];
        o.Irows = Vri_out + voff[t];
        o.v = (zd *)Vv + voff[t];
        solve_column(&P, j, &o, NULL, NULL, NULL);
        res[t] = o.res;
        flags[t] = o.flags;
        margin[t] = o.margin;
        sig[2 * t] = o.sig_sel;
        sig[2 * t + 1] = o.sig_next;
    }
    return 0;
}

/* Single column with its tile rows and leverage (for tests). */
int diaf_oracle_column(int n, const int *Acp, const int *Ari, const double *Av,
                       const int *Wcp, const int *Wri, int rule, const int *Vcp,
                       const int *Vri, const int *budget, const int *blk, int alg, double tie_tol,
                       double stab_tol, double stab_r, int j,
                       double *w, int *Irows, double *v, double *res, unsigned *flags,
                       double *margin, double *sig, int *m, int *rows, double *h) {
    problem P = make_problem(n, Acp, Ari, Av, Wcp, Wri, rule, Vcp, Vri, budget, blk, alg, tie_tol, stab_tol, stab_r);
    colout o = {(zd *)w, Irows, (zd *)v, 0, 0, 0, 0, 0};
    solve_column(&P, j, &o, h, rows, m);
    *res = o.res; *flags = o.flags; *margin = o.margin;
    sig[0] = o.sig_sel; sig[1] = o.sig_next;
    return 0;
}

/* Exposed building blocks, so tests can check them against LAPACK. */
int diaf_oracle_qr(int m, int k, double *a, double *r, double *q) {
    householder_qr(m, k, (zd *)a, (zd *)r, (zd *)q);
    return 0;
}

int diaf_oracle_jacobi_svd(int p, int q, double *g, double *v, double *sigma) {
    return jacobi_svd(p, q, (zd *)g, (zd *)v, sigma);
}
