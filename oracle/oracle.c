/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the polynomial-filtered interior eigensolver
 * of Accaputo, Derlet & Arbenz (arXiv 1902.07041).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark load this file.  It shares no code, header, table or helper with the GPU
 * library; the two meet only through the seeded input generator's arrays.
 *
 * Storage: scalar CSR (like the paper's Epetra_CrsMatrix, Sec. 3), multivectors column-major
 * with a leading dimension (like Epetra_MultiVector: each column contiguous).
 * Every routine is written as the plain definition or as the paper's algorithm in the paper's
 * order, with no blocking or fusion.  Each function names the passage it follows.
 *
 * Parity status: every function here is pinned by a CPU test against values the paper prints
 * (Tables 1-3 degrees, Fig. 2, Fig. 3, the spectral-transform example of Sec. 4.2), closed
 * forms (Chebyshev polynomials of diagonal matrices, Hellmann-Feynman derivatives, central
 * finite differences) or library routines (LAPACK eigh / qr through numpy).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846264338327950288

/* ======================================================================================
 * Scalar CSR matrix
 * ==================================================================================== */
typedef struct {
  int64_t n;
  int64_t nnz;
  int64_t *rp;
  int32_t *ci;
  double *v;
} or_csr;

static or_csr *or_csr_alloc(int64_t n, int64_t nnz) {
  or_csr *A = (or_csr *)calloc(1, sizeof(or_csr));
  if (!A) return NULL;
  A->n = n;
  A->nnz = nnz;
  A->rp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  A->ci = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  A->v = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  if (!A->rp || !A->ci || !A->v) {
    free(A->rp); free(A->ci); free(A->v); free(A);
    return NULL;
  }
  return A;
}

void or_csr_free(or_csr *A) {
  if (!A) return;
  free(A->rp);
  free(A->ci);
  free(A->v);
  free(A);
}

int64_t or_csr_n(const or_csr *A) { return A->n; }
int64_t or_csr_nnz(const or_csr *A) { return A->nnz; }

void or_csr_export(const or_csr *A, int64_t *rp, int32_t *ci, double *v) {
  memcpy(rp, A->rp, sizeof(int64_t) * (size_t)(A->n + 1));
  memcpy(ci, A->ci, sizeof(int32_t) * (size_t)A->nnz);
  memcpy(v, A->v, sizeof(double) * (size_t)A->nnz);
}

or_csr *or_csr_from_arrays(int64_t n, const int64_t *rp, const int32_t *ci, const double *v) {
  or_csr *A = or_csr_alloc(n, rp[n]);
  if (!A) return NULL;
  memcpy(A->rp, rp, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(A->ci, ci, sizeof(int32_t) * (size_t)rp[n]);
  memcpy(A->v, v, sizeof(double) * (size_t)rp[n]);
  return A;
}

/*
 * Mass-weighted Hessian of a spring network, Sec. 1 eqs. (1)-(2):
 *   Delta_ij = -k_ij r_ij r_ij^T for a bond (i, j), Delta_ii = -sum_{j != i} Delta_ij,
 *   H_ij = Delta_ij / sqrt(m_i m_j).
 * Scalar row 3i+a holds the 3x3 blocks of atom i's neighbours and itself, columns ascending.
 */
typedef struct {
  int32_t j;
  int64_t bond;
} or_adj;

static int or_cmp_adj(const void *a, const void *b) {
  const or_adj *x = (const or_adj *)a, *y = (const or_adj *)b;
  return x->j < y->j ? -1 : (x->j > y->j);
}

or_csr *or_csr_from_springs(int32_t N, int64_t nb, const int32_t *bi, const int32_t *bj,
                            const double *k, const double *rhat, const double *mass) {
  int64_t *deg = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
  if (!deg) return NULL;
  for (int64_t e = 0; e < nb; ++e) {
    deg[bi[e] + 1]++;
    deg[bj[e] + 1]++;
  }
  for (int32_t i = 0; i < N; ++i) deg[i + 1] += deg[i];
  or_adj *adj = (or_adj *)malloc(sizeof(or_adj) * (size_t)(2 * nb + 1));
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
  if (!adj || !fill) {
    free(deg); free(adj); free(fill);
    return NULL;
  }
  for (int32_t i = 0; i < N; ++i) fill[i] = deg[i];
  for (int64_t e = 0; e < nb; ++e) {
    adj[fill[bi[e]]].j = bj[e];
    adj[fill[bi[e]]++].bond = e;
    adj[fill[bj[e]]].j = bi[e];
    adj[fill[bj[e]]++].bond = e;
  }
  free(fill);
  for (int32_t i = 0; i < N; ++i) qsort(adj + deg[i], (size_t)(deg[i + 1] - deg[i]), sizeof(or_adj), or_cmp_adj);

  /* every atom row has (degree + 1) blocks of 3 entries per scalar row */
  int64_t nnz = 0;
  for (int32_t i = 0; i < N; ++i) nnz += 3 * 3 * (deg[i + 1] - deg[i] + 1);
  or_csr *H = or_csr_alloc(3 * (int64_t)N, nnz);
  if (!H) {
    free(deg); free(adj);
    return NULL;
  }
  int64_t pos = 0;
  for (int32_t i = 0; i < N; ++i) {
    /* the diagonal block Delta_ii = sum_j k_ij r r^T */
    double D[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t t = deg[i]; t < deg[i + 1]; ++t) {
      int64_t e = adj[t].bond;
      const double *r = rhat + 3 * e;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) D[3 * a + b] += k[e] * (r[a] * r[b]); /* r_a r_b == r_b r_a bitwise */
    }
    for (int a = 0; a < 3; ++a) {
      int64_t row = 3 * (int64_t)i + a;
      H->rp[row] = pos;
      int diag_done = 0;
      for (int64_t t = deg[i]; t <= deg[i + 1]; ++t) {
        int at_end = (t == deg[i + 1]);
        if (!diag_done && (at_end || adj[t].j > i)) {
          for (int b = 0; b < 3; ++b) {
            H->ci[pos] = 3 * i + b;
            H->v[pos++] = D[3 * a + b] / mass[i];
          }
          diag_done = 1;
        }
        if (at_end) break;
        int32_t j = adj[t].j;
        int64_t e = adj[t].bond;
        const double *r = rhat + 3 * e;
        double w = -k[e] / sqrt(mass[i] * mass[j]);
        for (int b = 0; b < 3; ++b) {
          H->ci[pos] = 3 * j + b;
          H->v[pos++] = w * (r[a] * r[b]);
        }
      }
    }
  }
  H->rp[3 * (int64_t)N] = pos;
  free(deg);
  free(adj);
  return H;
}

/* Y = A X for column-major multivectors (the plain definition of a sparse product). */
void or_spmm(const or_csr *A, int32_t k, const double *X, int64_t ldx, double *Y, int64_t ldy) {
  for (int32_t c = 0; c < k; ++c) {
    const double *x = X + (int64_t)c * ldx;
    double *y = Y + (int64_t)c * ldy;
    for (int64_t i = 0; i < A->n; ++i) {
      double s = 0.0;
      for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) s += A->v[p] * x[A->ci[p]];
      y[i] = s;
    }
  }
}

/* r_i = || A v_i - lam_i v_i ||_2 for k pairs (the residual reported by Alg. 3). */
void or_residuals(const or_csr *A, int32_t k, const double *lam, const double *V, int64_t ldv, double *res) {
  double *w = (double *)malloc(sizeof(double) * (size_t)A->n);
  for (int32_t c = 0; c < k; ++c) {
    or_spmm(A, 1, V + (int64_t)c * ldv, ldv, w, A->n);
    double s = 0.0;
    for (int64_t i = 0; i < A->n; ++i) {
      double d = w[i] - lam[c] * V[(int64_t)c * ldv + i];
      s += d * d;
    }
    res[c] = sqrt(s);
  }
  free(w);
}

/* ======================================================================================
 * Chebyshev machinery, Sec. 2.2-2.3 and App. A
 * ==================================================================================== */

/* int_a^b T_l(x) dx / sqrt(1 - x^2), App. A eq. (app.3). a <= b, both in [-1, 1]. */
static double or_int_T(int64_t l, double a, double b) {
  double ta = acos(a), tb = acos(b);
  if (l == 0) return ta - tb;
  return (sin((double)l * ta) - sin((double)l * tb)) / (double)l;
}

/*
 * int_a^b (al + be x + ga x^2) T_j(x) dx / sqrt(1 - x^2) by the product formula
 * 2 T_m T_n = T_{m+n} + T_{m-n} of App. A eq. (app.1): x = T_1, x^2 = (T_0 + T_2)/2.
 */
static double or_int_quad_T(int64_t j, double al, double be, double ga, double a, double b) {
  double c0 = al + 0.5 * ga;
  if (j == 0) return c0 * or_int_T(0, a, b) + be * or_int_T(1, a, b) + 0.5 * ga * or_int_T(2, a, b);
  if (j == 1)
    return c0 * or_int_T(1, a, b) + 0.5 * be * (or_int_T(2, a, b) + or_int_T(0, a, b)) +
           0.25 * ga * (or_int_T(3, a, b) + or_int_T(1, a, b));
  return c0 * or_int_T(j, a, b) + 0.5 * be * (or_int_T(j + 1, a, b) + or_int_T(j - 1, a, b)) +
         0.25 * ga * (or_int_T(j + 2, a, b) + or_int_T(j - 2, a, b));
}

/* <T_j, T_j>, eq. (cheby-ip.1) */
static double or_norm_T(int64_t j) { return j == 0 ? OR_PI : 0.5 * OR_PI; }

/*
 * Chebyshev coefficients gamma_0..gamma_m (eq. (cheby-ip.2a)) of the piecewise quadratic
 * filter target p of eq. (fct_f).  Each piece is clipped to [-1, 1] (only the part of p in
 * (-1, 1) enters, Sec. 2.6).  The last piece of eq. (fct_f) is read as eta+eps <= x < 1.
 */
void or_pq_coeffs(double xi, double eta, double eps, int32_t m, double *gam) {
  double lo[3], hi[3], al[3], be[3], ga[3];
  double e2 = eps * eps;
  /* (x - xi + eps)^2 / eps^2 on [xi - eps, xi] */
  lo[0] = xi - eps; hi[0] = xi;
  al[0] = (xi - eps) * (xi - eps) / e2; be[0] = -2.0 * (xi - eps) / e2; ga[0] = 1.0 / e2;
  /* 1 + ((eta - xi)^2 - (2x - xi - eta)^2) / (2 eps (eta - xi)) on [xi, eta] */
  double w = eta - xi, s = xi + eta, den = 2.0 * eps * w;
  lo[1] = xi; hi[1] = eta;
  al[1] = 1.0 + (w * w - s * s) / den; be[1] = 4.0 * s / den; ga[1] = -4.0 / den;
  /* (x - eta - eps)^2 / eps^2 on [eta, eta + eps] */
  lo[2] = eta; hi[2] = eta + eps;
  al[2] = (eta + eps) * (eta + eps) / e2; be[2] = -2.0 * (eta + eps) / e2; ga[2] = 1.0 / e2;
  for (int32_t j = 0; j <= m; ++j) {
    double acc = 0.0;
    for (int p = 0; p < 3; ++p) {
      double a = lo[p] < -1.0 ? -1.0 : lo[p], b = hi[p] > 1.0 ? 1.0 : hi[p];
      if (a >= b) continue;
      acc += or_int_quad_T(j, al[p], be[p], ga[p], a, b);
    }
    gam[j] = acc / or_norm_T(j);
  }
}

/* Coefficients of the characteristic function chi_[xi,eta] (Sec. 2.4, App. A eq. (app.3)). */
void or_chi_coeffs(double xi, double eta, int32_t m, double *gam) {
  double a = xi < -1.0 ? -1.0 : xi, b = eta > 1.0 ? 1.0 : eta;
  for (int32_t j = 0; j <= m; ++j) gam[j] = (a < b) ? or_int_T(j, a, b) / or_norm_T(j) : 0.0;
}

/*
 * Damping factors g_0..g_k for truncation at degree k, Sec. 2.3:
 *   kind 0: none (g_j = 1);
 *   kind 1: Jackson, eq. (jackson_smoothing), alpha_k = pi / (k + 2);
 *   kind 2: Lanczos sigma, eq. (lanczos_smoothing), theta_k = pi / (k + 1).
 */
void or_damping(int kind, int32_t k, double *g) {
  for (int32_t j = 0; j <= k; ++j) {
    if (kind == 1) {
      double al = OR_PI / (double)(k + 2);
      g[j] = (1.0 - (double)j / (double)(k + 2)) * cos(j * al) +
             (1.0 / (double)(k + 2)) * (cos(al) / sin(al)) * sin(j * al);
    } else if (kind == 2) {
      double th = OR_PI / (double)(k + 1);
      g[j] = (j == 0) ? 1.0 : sin(j * th) / (j * th);
    } else {
      g[j] = 1.0;
    }
  }
}

/* sum_{j=0}^k c_j T_j(x) with the three-term recurrence T_{j+1} = 2x T_j - T_{j-1}. */
double or_series_value(const double *c, int32_t k, double x) {
  double tpp = 1.0, y = c[0] * tpp;
  if (k < 1) return y;
  double tp = x;
  y += c[1] * tp;
  for (int32_t j = 2; j <= k; ++j) {
    double t = 2.0 * x * tp - tpp;
    tpp = tp;
    tp = t;
    y += c[j] * t;
  }
  return y;
}

/*
 * Smallest degree k >= 1 satisfying eq. (thresh) for the damped series of p:
 *   max{pi_k(xi - eps), pi_k(eta + eps)} <= r * min{pi_k(xi), pi_k(eta)}.
 * Returns -1 if no k <= kmax satisfies it.
 */
int32_t or_select_degree(double xi, double eta, double eps, double r, int kind, int32_t kmax) {
  double *gam = (double *)malloc(sizeof(double) * (size_t)(kmax + 1));
  double *g = (double *)malloc(sizeof(double) * (size_t)(kmax + 1));
  double *c = (double *)malloc(sizeof(double) * (size_t)(kmax + 1));
  or_pq_coeffs(xi, eta, eps, kmax, gam);
  int32_t found = -1;
  for (int32_t k = 1; k <= kmax; ++k) {
    or_damping(kind, k, g);
    for (int32_t j = 0; j <= k; ++j) c[j] = g[j] * gam[j];
    double vl = or_series_value(c, k, xi - eps), vr = or_series_value(c, k, eta + eps);
    double vxi = or_series_value(c, k, xi), veta = or_series_value(c, k, eta);
    double lhs = vl > vr ? vl : vr, rhs = r * (vxi < veta ? vxi : veta);
    if (lhs <= rhs) {
      found = k;
      break;
    }
  }
  free(gam);
  free(g);
  free(c);
  return found;
}

/*
 * Alg. 2: y = p_m(Ht) x for each of the k columns, with the spectral transform of
 * eq. (transf.1) folded in: Ht = (H - cI)/d, so Ht t = (H t - c t) / d.
 *   t'' = x; y = g0 t''; t' = Ht x; y += g1 t'; for j = 2..m: t = 2 Ht t' - t''; rotate; y += gj t.
 * Returns the number of single-vector products with H (k * m).
 */
int64_t or_cheb_filter(const or_csr *H, double c, double d, const double *coef, int32_t m, int32_t k,
                       const double *X, int64_t ldx, double *Y, int64_t ldy) {
  int64_t n = H->n;
  double *tpp = (double *)malloc(sizeof(double) * (size_t)n);
  double *tp = (double *)malloc(sizeof(double) * (size_t)n);
  double *t = (double *)malloc(sizeof(double) * (size_t)n);
  double *ht = (double *)malloc(sizeof(double) * (size_t)n);
  int64_t mv = 0;
  for (int32_t col = 0; col < k; ++col) {
    const double *x = X + (int64_t)col * ldx;
    double *y = Y + (int64_t)col * ldy;
    for (int64_t i = 0; i < n; ++i) {
      tpp[i] = x[i];
      y[i] = coef[0] * tpp[i];
    }
    if (m >= 1) {
      or_spmm(H, 1, x, n, ht, n);
      ++mv;
      for (int64_t i = 0; i < n; ++i) {
        tp[i] = (ht[i] - c * x[i]) / d;
        y[i] += coef[1] * tp[i];
      }
    }
    for (int32_t j = 2; j <= m; ++j) {
      or_spmm(H, 1, tp, n, ht, n);
      ++mv;
      for (int64_t i = 0; i < n; ++i) {
        t[i] = 2.0 * (ht[i] - c * tp[i]) / d - tpp[i];
        y[i] += coef[j] * t[i];
      }
      double *sw = tpp;
      tpp = tp;
      tp = t;
      t = sw;
    }
  }
  free(tpp);
  free(tp);
  free(t);
  free(ht);
  return mv;
}

/* ======================================================================================
 * Random blocks: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) + Box-Muller.
 * Element (row, col) of stream s under seed: counter (row, col, s, 0), key (seed lo, seed hi).
 * u1 = (top 53 bits of words 0,1 + 1) 2^-53 in (0, 1], u2 = top 53 bits of words 2,3 * 2^-53,
 * z = sqrt(-2 ln u1) cos(2 pi u2).
 * ==================================================================================== */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3], k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t m0 = (uint64_t)x0 * 0xD2511F53ull, m1 = (uint64_t)x2 * 0xCD9E8D57ull;
    uint32_t y0 = (uint32_t)(m1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)m1;
    uint32_t y2 = (uint32_t)(m0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)m0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double or_normal(uint64_t seed, uint32_t stream, uint32_t row, uint32_t col) {
  uint32_t ctr[4] = {row, col, stream, 0u}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)}, w[4];
  or_philox4x32_10(ctr, key, w);
  uint64_t a = ((uint64_t)w[0] << 21) ^ (uint64_t)(w[1] >> 11);
  uint64_t b = ((uint64_t)w[2] << 21) ^ (uint64_t)(w[3] >> 11);
  double u1 = ((double)a + 1.0) * 0x1.0p-53, u2 = (double)b * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cos(2.0 * OR_PI * u2);
}

void or_normal_block(uint64_t seed, uint32_t stream, int64_t n, int32_t k, int32_t col0, double *X, int64_t ldx) {
  for (int32_t c = 0; c < k; ++c)
    for (int64_t i = 0; i < n; ++i) X[(int64_t)c * ldx + i] = or_normal(seed, stream, (uint32_t)i, (uint32_t)(col0 + c));
}

/* ======================================================================================
 * Dense linear algebra (own code, column-major)
 * ==================================================================================== */

/* Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (Golub & Van Loan, Sec. 8.5).
 * A is destroyed; w ascending; V columns are the eigenvectors. */
void or_jacobi_eig(int32_t n, double *A, double *w, double *V) {
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < n; ++j) V[(int64_t)j * n + i] = (i == j) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int64_t i = 0; i < (int64_t)n * n; ++i) fro += A[i] * A[i];
  fro = sqrt(fro);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int32_t j = 0; j < n; ++j)
      for (int32_t i = 0; i < j; ++i) off += 2.0 * A[(int64_t)j * n + i] * A[(int64_t)j * n + i];
    if (sqrt(off) <= 1e-17 * fro || fro == 0.0) break;
    for (int32_t p = 0; p < n - 1; ++p)
      for (int32_t q = p + 1; q < n; ++q) {
        double apq = A[(int64_t)q * n + p];
        if (apq == 0.0) continue;
        double app = A[(int64_t)p * n + p], aqq = A[(int64_t)q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int32_t r = 0; r < n; ++r) { /* columns p, q */
          double arp = A[(int64_t)p * n + r], arq = A[(int64_t)q * n + r];
          A[(int64_t)p * n + r] = cs * arp - sn * arq;
          A[(int64_t)q * n + r] = sn * arp + cs * arq;
        }
        for (int32_t r = 0; r < n; ++r) { /* rows p, q */
          double apr = A[(int64_t)r * n + p], aqr = A[(int64_t)r * n + q];
          A[(int64_t)r * n + p] = cs * apr - sn * aqr;
          A[(int64_t)r * n + q] = sn * apr + cs * aqr;
        }
        A[(int64_t)q * n + p] = 0.0;
        A[(int64_t)p * n + q] = 0.0;
        for (int32_t r = 0; r < n; ++r) {
          double vrp = V[(int64_t)p * n + r], vrq = V[(int64_t)q * n + r];
          V[(int64_t)p * n + r] = cs * vrp - sn * vrq;
          V[(int64_t)q * n + r] = sn * vrp + cs * vrq;
        }
      }
  }
  for (int32_t i = 0; i < n; ++i) w[i] = A[(int64_t)i * n + i];
  /* selection sort, ascending */
  for (int32_t i = 0; i < n; ++i) {
    int32_t m = i;
    for (int32_t j = i + 1; j < n; ++j)
      if (w[j] < w[m]) m = j;
    if (m != i) {
      double t = w[i]; w[i] = w[m]; w[m] = t;
      for (int32_t r = 0; r < n; ++r) {
        double s = V[(int64_t)i * n + r];
        V[(int64_t)i * n + r] = V[(int64_t)m * n + r];
        V[(int64_t)m * n + r] = s;
      }
    }
  }
}

/*
 * Householder QR of an n x q block (n >= q): on return X holds the thin Q (n x q) and,
 * if R != NULL, R (q x q, upper triangular) holds the triangular factor, X_in = Q R.
 */
int or_householder_qr(int64_t n, int32_t q, double *X, int64_t ldx, double *R) {
  if (n < q) return -1;
  double *vs = (double *)calloc((size_t)n * (size_t)(q > 0 ? q : 1), sizeof(double));
  double *beta = (double *)calloc((size_t)(q > 0 ? q : 1), sizeof(double));
  for (int32_t j = 0; j < q; ++j) {
    double *x = X + (int64_t)j * ldx;
    double nrm = 0.0;
    for (int64_t i = j; i < n; ++i) nrm += x[i] * x[i];
    nrm = sqrt(nrm);
    double *v = vs + (int64_t)j * n;
    double alpha = (x[j] >= 0 ? -nrm : nrm);
    for (int64_t i = j; i < n; ++i) v[i] = x[i];
    v[j] -= alpha;
    double vn = 0.0;
    for (int64_t i = j; i < n; ++i) vn += v[i] * v[i];
    beta[j] = vn > 0 ? 2.0 / vn : 0.0;
    for (int32_t c = j; c < q; ++c) {
      double *xc = X + (int64_t)c * ldx, s = 0.0;
      for (int64_t i = j; i < n; ++i) s += v[i] * xc[i];
      s *= beta[j];
      for (int64_t i = j; i < n; ++i) xc[i] -= s * v[i];
    }
  }
  if (R) {
    for (int32_t c = 0; c < q; ++c)
      for (int32_t r = 0; r < q; ++r) R[(int64_t)c * q + r] = (r <= c) ? X[(int64_t)c * ldx + r] : 0.0;
  }
  /* form Q = H_0 ... H_{q-1} [I; 0] */
  for (int32_t c = 0; c < q; ++c)
    for (int64_t i = 0; i < n; ++i) X[(int64_t)c * ldx + i] = (i == c) ? 1.0 : 0.0;
  for (int32_t j = q - 1; j >= 0; --j) {
    double *v = vs + (int64_t)j * n;
    for (int32_t c = j; c < q; ++c) {
      double *xc = X + (int64_t)c * ldx, s = 0.0;
      for (int64_t i = j; i < n; ++i) s += v[i] * xc[i];
      s *= beta[j];
      for (int64_t i = j; i < n; ++i) xc[i] -= s * v[i];
    }
  }
  free(vs);
  free(beta);
  return 0;
}

/*
 * Householder reduction of a dense symmetric matrix to tridiagonal form (Golub & Van Loan,
 * Alg. 8.3.1).  A (n x n, column-major) is destroyed; diag[n], off[n-1] receive T.
 */
void or_tridiagonalize(int32_t n, double *A, double *diag, double *off) {
  double *v = (double *)malloc(sizeof(double) * (size_t)n);
  double *p = (double *)malloc(sizeof(double) * (size_t)n);
  for (int32_t k = 0; k < n - 2; ++k) {
    /* x = A[k+1:, k] */
    double nrm = 0.0;
    for (int32_t i = k + 1; i < n; ++i) nrm += A[(int64_t)k * n + i] * A[(int64_t)k * n + i];
    nrm = sqrt(nrm);
    double x0 = A[(int64_t)k * n + k + 1];
    double alpha = (x0 >= 0 ? -nrm : nrm);
    for (int32_t i = k + 1; i < n; ++i) v[i] = A[(int64_t)k * n + i];
    v[k + 1] -= alpha;
    double vn = 0.0;
    for (int32_t i = k + 1; i < n; ++i) vn += v[i] * v[i];
    if (vn == 0.0) continue;
    double beta = 2.0 / vn;
    /* p = beta A22 v */
    for (int32_t i = k + 1; i < n; ++i) p[i] = 0.0;
    for (int32_t j = k + 1; j < n; ++j) {
      double vj = v[j];
      const double *aj = A + (int64_t)j * n;
      for (int32_t i = k + 1; i < n; ++i) p[i] += aj[i] * vj;
    }
    double pv = 0.0;
    for (int32_t i = k + 1; i < n; ++i) {
      p[i] *= beta;
      pv += p[i] * v[i];
    }
    /* w = p - (beta/2)(p^T v) v ; A22 -= v w^T + w v^T */
    double hh = 0.5 * beta * pv;
    for (int32_t i = k + 1; i < n; ++i) p[i] -= hh * v[i];
    for (int32_t j = k + 1; j < n; ++j) {
      double *aj = A + (int64_t)j * n;
      double vj = v[j], wj = p[j];
      for (int32_t i = k + 1; i < n; ++i) aj[i] -= v[i] * wj + p[i] * vj;
    }
    A[(int64_t)k * n + k + 1] = alpha;
    A[(int64_t)(k + 1) * n + k] = alpha;
    for (int32_t i = k + 2; i < n; ++i) {
      A[(int64_t)k * n + i] = 0.0;
      A[(int64_t)i * n + k] = 0.0;
    }
  }
  for (int32_t i = 0; i < n; ++i) diag[i] = A[(int64_t)i * n + i];
  for (int32_t i = 0; i + 1 < n; ++i) off[i] = A[(int64_t)i * n + i + 1];
  free(v);
  free(p);
}

/*
 * Number of eigenvalues of the tridiagonal T below sigma, by Sylvester's law of inertia on
 * the LDL^T factorisation of T - sigma I (the pivots of the Sturm sequence), Sec. 2.4.
 */
int64_t or_count_below(int32_t n, const double *diag, const double *off, double sigma) {
  int64_t cnt = 0;
  double dprev = 1.0;
  for (int32_t i = 0; i < n; ++i) {
    double d = diag[i] - sigma;
    if (i > 0) d -= off[i - 1] * off[i - 1] / dprev;
    if (d == 0.0) d = 1e-300;
    if (d < 0) ++cnt;
    dprev = d;
  }
  return cnt;
}

/* ======================================================================================
 * Extremal eigenvalue estimate (Alg. 3, a few Lanczos steps): Lanczos with full reorthogonalisation.
 * lmax_est = max(1.01 theta_max, theta_max + |beta_s s_s|), s the Ritz vector of theta_max.
 * The start vector is column 0 of random stream 1.
 * ==================================================================================== */
int or_lanczos_lmax(const or_csr *H, int32_t steps, uint64_t seed, double *theta_max, double *resid_bound,
                    double *lmax_est) {
  int64_t n = H->n;
  if (steps < 1) return -1;
  if (steps > n) steps = (int32_t)n;
  double *V = (double *)calloc((size_t)n * (size_t)(steps + 1), sizeof(double));
  double *w = (double *)malloc(sizeof(double) * (size_t)n);
  double *al = (double *)calloc((size_t)steps, sizeof(double));
  double *be = (double *)calloc((size_t)steps, sizeof(double));
  or_normal_block(seed, 1u, n, 1, 0, V, n);
  double nv = 0.0;
  for (int64_t i = 0; i < n; ++i) nv += V[i] * V[i];
  nv = sqrt(nv);
  for (int64_t i = 0; i < n; ++i) V[i] /= nv;
  int32_t s = steps;
  for (int32_t j = 0; j < steps; ++j) {
    double *vj = V + (int64_t)j * n;
    or_spmm(H, 1, vj, n, w, n);
    if (j > 0)
      for (int64_t i = 0; i < n; ++i) w[i] -= be[j - 1] * V[(int64_t)(j - 1) * n + i];
    double a = 0.0;
    for (int64_t i = 0; i < n; ++i) a += w[i] * vj[i];
    al[j] = a;
    for (int64_t i = 0; i < n; ++i) w[i] -= a * vj[i];
    for (int pass = 0; pass < 2; ++pass)
      for (int32_t l = 0; l <= j; ++l) {
        double *vl = V + (int64_t)l * n, h = 0.0;
        for (int64_t i = 0; i < n; ++i) h += vl[i] * w[i];
        for (int64_t i = 0; i < n; ++i) w[i] -= h * vl[i];
      }
    double b = 0.0;
    for (int64_t i = 0; i < n; ++i) b += w[i] * w[i];
    b = sqrt(b);
    be[j] = b;
    if (b == 0.0) {
      s = j + 1;
      break;
    }
    for (int64_t i = 0; i < n; ++i) V[(int64_t)(j + 1) * n + i] = w[i] / b;
  }
  double *T = (double *)calloc((size_t)s * s, sizeof(double));
  double *ev = (double *)malloc(sizeof(double) * s);
  double *EV = (double *)malloc(sizeof(double) * (size_t)s * s);
  for (int32_t i = 0; i < s; ++i) {
    T[(int64_t)i * s + i] = al[i];
    if (i + 1 < s) {
      T[(int64_t)(i + 1) * s + i] = be[i];
      T[(int64_t)i * s + i + 1] = be[i];
    }
  }
  or_jacobi_eig(s, T, ev, EV);
  double th = ev[s - 1];
  double rb = fabs(be[s - 1] * EV[(int64_t)(s - 1) * s + (s - 1)]);
  *theta_max = th;
  *resid_bound = rb;
  double e1 = 1.01 * th, e2 = th + rb;
  *lmax_est = e1 > e2 ? e1 : e2;
  free(V); free(w); free(al); free(be); free(T); free(ev); free(EV);
  return 0;
}

/* ======================================================================================
 * Eigenvalue count estimator, Sec. 2.4 eq. (eigval_count_estimator):
 *   T_M = (n / M) sum_l v_l^T psi(Ht) v_l, v_l = g_l / ||g_l||, g_l Gaussian (stream 2),
 *   psi the (optionally damped) Chebyshev series of chi_[xi, eta] of the given degree.
 * ==================================================================================== */
double or_count_estimate(const or_csr *H, double c, double d, double xi, double eta, int32_t degree,
                         int damping, int32_t M, uint64_t seed) {
  int64_t n = H->n;
  double *gam = (double *)malloc(sizeof(double) * (size_t)(degree + 1));
  double *g = (double *)malloc(sizeof(double) * (size_t)(degree + 1));
  or_chi_coeffs(xi, eta, degree, gam);
  or_damping(damping, degree, g);
  for (int32_t j = 0; j <= degree; ++j) gam[j] *= g[j];
  double *v = (double *)malloc(sizeof(double) * (size_t)n);
  double *y = (double *)malloc(sizeof(double) * (size_t)n);
  double sum = 0.0;
  for (int32_t l = 0; l < M; ++l) {
    or_normal_block(seed, 2u, n, 1, l, v, n);
    double nv = 0.0;
    for (int64_t i = 0; i < n; ++i) nv += v[i] * v[i];
    nv = sqrt(nv);
    for (int64_t i = 0; i < n; ++i) v[i] /= nv;
    or_cheb_filter(H, c, d, gam, degree, 1, v, n, y, n);
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += v[i] * y[i];
    sum += s;
  }
  free(gam); free(g); free(v); free(y);
  return (double)n / (double)M * sum;
}

/* ======================================================================================
 * Filtered subspace iteration with Rayleigh-Ritz on H and locking (Sec. 2.6, the Rayleigh-Ritz step of Alg. 1,
 * Alg. 4 with n_RR = 1, and the locking paragraph after Alg. 4).
 *
 * Per iteration, on the active (unlocked) columns:
 *   Y = p(Ht) X                         (Alg. 2)
 *   Y -= L (L^T Y), twice               (keep the active block orthogonal to locked vectors)
 *   X = Q of the Householder QR of Y    (Alg. 4, "QR factorization")
 *   W = H X; A = X^T W; A = Q Theta Q^T (Jacobi); X = X Q; W = W Q   (Rayleigh-Ritz, Alg. 1)
 *   r_i = ||w_i - theta_i x_i|| / lmax
 *   lock every pair with r_i <= tol.
 * Stop once no unconverged active Ritz pair certifies an eigenvalue inside [a, b] (its residual
 * interval [theta - r, theta + r] inside [a, b]), the number of converged pairs in [a, b] equals
 * that of the previous iteration, and at least two iterations ran.
 *
 * Inputs: X0 (n x q, column-major).  Outputs (capacity cap): the pairs with eigenvalue in
 * [a, b], ascending, residuals relative to lmax.  Returns 0 on convergence, 1 if max_iter was
 * reached, 2 if the capacity was exceeded (n_found set), 3 if every active Ritz value lay in
 * [a, b] (the subspace is too narrow to prove completeness), <0 on bad input.
 * ==================================================================================== */
int or_si_solve(const or_csr *H, double a, double b, double lmin, double lmax, const double *coef, int32_t m,
                int32_t q, const double *X0, double tol, int32_t max_iter, int32_t cap, int32_t *n_found,
                double *lam_out, double *vec_out, double *res_out, int32_t *iters_out, int64_t *matvecs_out) {
  int64_t n = H->n;
  if (q < 1 || q > n || m < 0) return -1;
  double c = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
  double *L = (double *)malloc(sizeof(double) * (size_t)n * q);   /* locked vectors */
  double *Lam = (double *)malloc(sizeof(double) * (size_t)q);      /* locked values */
  double *Lres = (double *)malloc(sizeof(double) * (size_t)q);
  double *X = (double *)malloc(sizeof(double) * (size_t)n * q);
  double *Y = (double *)malloc(sizeof(double) * (size_t)n * q);
  double *W = (double *)malloc(sizeof(double) * (size_t)n * q);
  double *A = (double *)malloc(sizeof(double) * (size_t)q * q);
  double *Q = (double *)malloc(sizeof(double) * (size_t)q * q);
  double *th = (double *)malloc(sizeof(double) * (size_t)q);
  double *rr = (double *)malloc(sizeof(double) * (size_t)q);
  double *h = (double *)malloc(sizeof(double) * (size_t)q);
  int32_t nl = 0, act = q;
  int64_t mv = 0;
  memcpy(X, X0, sizeof(double) * (size_t)n * q);
  or_householder_qr(n, act, X, n, NULL);
  int status = 1, prev_count = -1, it = 0;
  for (it = 1; it <= max_iter; ++it) {
    /* filter */
    mv += or_cheb_filter(H, c, d, coef, m, act, X, n, Y, n);
    /* orthogonalise against locked vectors (classical Gram-Schmidt, two passes) */
    for (int pass = 0; pass < 2 && nl > 0; ++pass)
      for (int32_t col = 0; col < act; ++col) {
        double *y = Y + (int64_t)col * n;
        for (int32_t l = 0; l < nl; ++l) {
          double s = 0.0;
          for (int64_t i = 0; i < n; ++i) s += L[(int64_t)l * n + i] * y[i];
          h[l] = s;
        }
        for (int32_t l = 0; l < nl; ++l)
          for (int64_t i = 0; i < n; ++i) y[i] -= h[l] * L[(int64_t)l * n + i];
      }
    /* QR */
    memcpy(X, Y, sizeof(double) * (size_t)n * act);
    or_householder_qr(n, act, X, n, NULL);
    /* Rayleigh-Ritz with H */
    or_spmm(H, act, X, n, W, n);
    mv += act;
    for (int32_t j = 0; j < act; ++j)
      for (int32_t i = 0; i < act; ++i) {
        double s = 0.0;
        for (int64_t r = 0; r < n; ++r) s += X[(int64_t)i * n + r] * W[(int64_t)j * n + r];
        A[(int64_t)j * act + i] = s;
      }
    for (int32_t j = 0; j < act; ++j)
      for (int32_t i = 0; i < j; ++i) {
        double s = 0.5 * (A[(int64_t)j * act + i] + A[(int64_t)i * act + j]);
        A[(int64_t)j * act + i] = s;
        A[(int64_t)i * act + j] = s;
      }
    or_jacobi_eig(act, A, th, Q);
    /* X = X Q, W = W Q (through Y as scratch) */
    for (int32_t j = 0; j < act; ++j)
      for (int64_t r = 0; r < n; ++r) {
        double s = 0.0;
        for (int32_t i = 0; i < act; ++i) s += X[(int64_t)i * n + r] * Q[(int64_t)j * act + i];
        Y[(int64_t)j * n + r] = s;
      }
    memcpy(X, Y, sizeof(double) * (size_t)n * act);
    for (int32_t j = 0; j < act; ++j)
      for (int64_t r = 0; r < n; ++r) {
        double s = 0.0;
        for (int32_t i = 0; i < act; ++i) s += W[(int64_t)i * n + r] * Q[(int64_t)j * act + i];
        Y[(int64_t)j * n + r] = s;
      }
    memcpy(W, Y, sizeof(double) * (size_t)n * act);
    /* residuals */
    for (int32_t j = 0; j < act; ++j) {
      double s = 0.0;
      for (int64_t r = 0; r < n; ++r) {
        double e = W[(int64_t)j * n + r] - th[j] * X[(int64_t)j * n + r];
        s += e * e;
      }
      rr[j] = sqrt(s) / lmax;
    }
    /* convergence bookkeeping: an unconverged Ritz pair (theta, r) certifies a not yet locked
       eigenvalue in [a, b] only if [theta - r, theta + r] lies inside [a, b] (the Krylov-Weinstein
       bound on the complement of the locked invariant subspace); other unconverged Ritz values in
       [a, b] may be mixtures of eigenvectors from both sides of the interval */
    int32_t unconv_in = 0, count_in = 0;
    for (int32_t j = 0; j < act; ++j) {
      double rabs = rr[j] * lmax;
      if (rr[j] > tol && th[j] - rabs >= a && th[j] + rabs <= b) ++unconv_in;
      if (rr[j] <= tol && th[j] >= a && th[j] <= b) ++count_in;
    }
    for (int32_t l = 0; l < nl; ++l)
      if (Lam[l] >= a && Lam[l] <= b) ++count_in;
    /* lock converged pairs; compact the active block */
    int32_t keep = 0;
    for (int32_t j = 0; j < act; ++j) {
      if (rr[j] <= tol && nl < q) {
        memcpy(L + (int64_t)nl * n, X + (int64_t)j * n, sizeof(double) * (size_t)n);
        Lam[nl] = th[j];
        Lres[nl] = rr[j];
        ++nl;
      } else {
        if (keep != j) memcpy(X + (int64_t)keep * n, X + (int64_t)j * n, sizeof(double) * (size_t)n);
        ++keep;
      }
    }
    act = keep;
    if ((unconv_in == 0 && count_in == prev_count && it >= 2) || act == 0) {
      status = (count_in >= q) ? 3 : 0;
      break;
    }
    prev_count = count_in;
  }
  if (it > max_iter) it = max_iter;
  /* gather pairs in [a, b], ascending */
  int32_t nf = 0;
  for (int32_t l = 0; l < nl; ++l)
    if (Lam[l] >= a && Lam[l] <= b) ++nf;
  *n_found = nf;
  int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nf > 0 ? nf : 1));
  int32_t t = 0;
  for (int32_t l = 0; l < nl; ++l)
    if (Lam[l] >= a && Lam[l] <= b) ord[t++] = l;
  for (int32_t i = 1; i < nf; ++i) { /* insertion sort by eigenvalue */
    int32_t key = ord[i], j = i - 1;
    while (j >= 0 && Lam[ord[j]] > Lam[key]) {
      ord[j + 1] = ord[j];
      --j;
    }
    ord[j + 1] = key;
  }
  if (nf > cap) {
    status = 2;
  } else {
    for (int32_t i = 0; i < nf; ++i) {
      lam_out[i] = Lam[ord[i]];
      if (res_out) res_out[i] = Lres[ord[i]];
      if (vec_out) memcpy(vec_out + (int64_t)i * n, L + (int64_t)ord[i] * n, sizeof(double) * (size_t)n);
    }
  }
  if (iters_out) *iters_out = it;
  if (matvecs_out) *matvecs_out = mv;
  free(ord); free(L); free(Lam); free(Lres); free(X); free(Y); free(W); free(A); free(Q); free(th); free(rr); free(h);
  return status;
}

/* ======================================================================================
 * Alg. 4 as printed (Rutishauser's subspace iteration with an SVD Ritz step), applied to a
 * DIAGONAL operator pi(H) = diag(pd) -- the synthetic problems of Sec. 4.1, where applying
 * Alg. 2 to a diagonal H reduces to multiplying row i by pi(lambda_i).
 *   k = 1 mod n_RR, k > 1: Y = op X; R = Y - X Lambda; n_conv = #{||r_i|| < tau};
 *                          return if n_conv >= p; X = Y
 *   k = -1 mod n_RR:       X R = op X (QR)
 *   k = 0 mod n_RR:        Y = op X; X R = Y; R = U Lambda V^T (SVD); X = X U
 *   otherwise:             X = op X
 * Returns the step k at which it returned (number of operator applications), or -1.
 * ==================================================================================== */
int32_t or_si_alg4_diag(int64_t n, const double *pd, int32_t q, int32_t p, int32_t n_rr, double tau,
                        const double *X0, int32_t max_k) {
  double *X = (double *)malloc(sizeof(double) * (size_t)n * q);
  double *Y = (double *)malloc(sizeof(double) * (size_t)n * q);
  double *R = (double *)malloc(sizeof(double) * (size_t)q * q);
  double *RRt = (double *)malloc(sizeof(double) * (size_t)q * q);
  double *U = (double *)malloc(sizeof(double) * (size_t)q * q);
  double *sv = (double *)malloc(sizeof(double) * (size_t)q);
  double *Lam = (double *)calloc((size_t)q, sizeof(double));
  memcpy(X, X0, sizeof(double) * (size_t)n * q);
  or_householder_qr(n, q, X, n, NULL);
  int32_t result = -1;
  for (int32_t k = 1; k <= max_k; ++k) {
    for (int32_t c = 0; c < q; ++c)
      for (int64_t i = 0; i < n; ++i) Y[(int64_t)c * n + i] = pd[i] * X[(int64_t)c * n + i];
    int32_t km = k % n_rr;
    if (km == 1 % n_rr && k > 1) {
      int32_t nconv = 0;
      for (int32_t c = 0; c < q; ++c) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) {
          double e = Y[(int64_t)c * n + i] - Lam[c] * X[(int64_t)c * n + i];
          s += e * e;
        }
        if (sqrt(s) < tau) ++nconv;
      }
      if (nconv >= p) {
        result = k;
        break;
      }
      memcpy(X, Y, sizeof(double) * (size_t)n * q);
    } else if (km == (n_rr - 1) % n_rr) {
      memcpy(X, Y, sizeof(double) * (size_t)n * q);
      or_householder_qr(n, q, X, n, NULL);
    } else if (km == 0) {
      memcpy(X, Y, sizeof(double) * (size_t)n * q);
      or_householder_qr(n, q, X, n, R);
      /* left singular vectors of R: eigenvectors of R R^T, singular values descending */
      for (int32_t j = 0; j < q; ++j)
        for (int32_t i = 0; i < q; ++i) {
          double s = 0.0;
          for (int32_t l = 0; l < q; ++l) s += R[(int64_t)l * q + i] * R[(int64_t)l * q + j];
          RRt[(int64_t)j * q + i] = s;
        }
      or_jacobi_eig(q, RRt, sv, U);
      for (int32_t j = 0; j < q; ++j) Lam[j] = sqrt(sv[q - 1 - j] > 0 ? sv[q - 1 - j] : 0.0);
      for (int32_t j = 0; j < q; ++j) /* X U with U's columns reversed (descending) */
        for (int64_t r = 0; r < n; ++r) {
          double s = 0.0;
          for (int32_t i = 0; i < q; ++i) s += X[(int64_t)i * n + r] * U[(int64_t)(q - 1 - j) * q + i];
          Y[(int64_t)j * n + r] = s;
        }
      memcpy(X, Y, sizeof(double) * (size_t)n * q);
    } else {
      memcpy(X, Y, sizeof(double) * (size_t)n * q);
    }
  }
  free(X); free(Y); free(R); free(RRt); free(U); free(sv); free(Lam);
  return result;
}

/* ======================================================================================
 * Adjoint of Alg. 2 (reverse sweep through the three-term recurrence).
 * For L = <Ybar, Y>, Y = sum_j gamma_j T_j(Ht) X, Ht = (H - cI)/d with c, d held fixed:
 *   adjoints a_j = dL/dt_j: a_m = g_m Ybar, a_{m-1} = g_{m-1} Ybar + 2 Ht a_m,
 *   a_j = g_j Ybar + 2 Ht a_{j+1} - a_{j+2} (j >= 1), a_0 = g_0 Ybar + Ht a_1 - a_2,
 *   Xbar = a_0,
 *   dL/dHt = a_1 t_0^T + sum_{j=1}^{m-1} 2 a_{j+1} t_j^T (summed over columns),
 *   dL/dH = dL/dHt / d, restricted to the stored pattern: vbar[p] for each CSR entry p.
 * Every t_j is stored (no checkpointing): memory (m+1) n k doubles.
 * ==================================================================================== */
int or_filter_adjoint(const or_csr *H, double c, double d, const double *coef, int32_t m, int32_t k,
                      const double *X, int64_t ldx, const double *Yb, int64_t ldyb, double *Xb, int64_t ldxb,
                      double *vbar) {
  int64_t n = H->n;
  double *T = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(m + 1));
  double *a = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(m + 2 > 3 ? m + 2 : 3));
  double *ht = (double *)malloc(sizeof(double) * (size_t)n);
  if (!T || !a || !ht) {
    free(T); free(a); free(ht);
    return -4;
  }
  for (int64_t p = 0; p < H->nnz; ++p) vbar[p] = 0.0;
  for (int32_t col = 0; col < k; ++col) {
    const double *x = X + (int64_t)col * ldx;
    const double *yb = Yb + (int64_t)col * ldyb;
    /* forward: t_0 .. t_m */
    memcpy(T, x, sizeof(double) * (size_t)n);
    if (m >= 1) {
      or_spmm(H, 1, T, n, ht, n);
      for (int64_t i = 0; i < n; ++i) T[n + i] = (ht[i] - c * T[i]) / d;
    }
    for (int32_t j = 2; j <= m; ++j) {
      or_spmm(H, 1, T + (int64_t)(j - 1) * n, n, ht, n);
      for (int64_t i = 0; i < n; ++i)
        T[(int64_t)j * n + i] = 2.0 * (ht[i] - c * T[(int64_t)(j - 1) * n + i]) / d - T[(int64_t)(j - 2) * n + i];
    }
    /* reverse: a_j stored at a + j n, with a_{m+1} = 0 */
    for (int64_t i = 0; i < n; ++i) a[(int64_t)(m + 1) * n + i] = 0.0;
    for (int32_t j = m; j >= 0; --j) {
      double *aj = a + (int64_t)j * n;
      for (int64_t i = 0; i < n; ++i) aj[i] = coef[j] * yb[i];
      if (j + 1 <= m) {
        /* coefficient of Ht a_{j+1}: 2 when t_{j+1} = 2 Ht t_j - t_{j-1} (j >= 1), 1 for t_1 = Ht t_0 */
        double f = (j >= 1) ? 2.0 : 1.0;
        or_spmm(H, 1, a + (int64_t)(j + 1) * n, n, ht, n);
        for (int64_t i = 0; i < n; ++i) aj[i] += f * (ht[i] - c * a[(int64_t)(j + 1) * n + i]) / d;
      }
      if (j + 2 <= m)
        for (int64_t i = 0; i < n; ++i) aj[i] -= a[(int64_t)(j + 2) * n + i];
    }
    double *xb = Xb + (int64_t)col * ldxb;
    for (int64_t i = 0; i < n; ++i) xb[i] = a[i];
    /* dL/dH entries */
    for (int64_t row = 0; row < n; ++row)
      for (int64_t p = H->rp[row]; p < H->rp[row + 1]; ++p) {
        int32_t cc = H->ci[p];
        double s = 0.0;
        if (m >= 1) s += a[n + row] * T[cc];
        for (int32_t j = 1; j <= m - 1; ++j) s += 2.0 * a[(int64_t)(j + 1) * n + row] * T[(int64_t)j * n + cc];
        vbar[p] += s / d;
      }
  }
  free(T);
  free(a);
  free(ht);
  return 0;
}

static int64_t or_find(const or_csr *H, int64_t row, int32_t col) {
  int64_t lo = H->rp[row], hi = H->rp[row + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    if (H->ci[mid] == col) return mid;
    if (H->ci[mid] < col) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

/*
 * Chain rule from dL/dH (per stored entry of the mass-weighted Hessian built by
 * or_csr_from_springs) to the spring constants and masses (Sec. 1 eq. (2)):
 *   H_ij = -k r r^T / sqrt(m_i m_j) (both off-diagonal blocks), H_ii += k r r^T / m_i,
 *   dL/dk_e = sum over the four blocks touched by bond e of <Hbar_block, dH_block/dk_e>,
 *   dL/dm_i = -1/(2 m_i) sum_{j != i} (<Hbar_ij, H_ij> + <Hbar_ji, H_ji>) - <Hbar_ii, H_ii> / m_i.
 */
void or_chain_springs(const or_csr *H, int32_t N, int64_t nb, const int32_t *bi, const int32_t *bj,
                      const double *k, const double *rhat, const double *mass, const double *vbar, double *kbar,
                      double *mbar) {
  (void)k;
  for (int64_t e = 0; e < nb; ++e) {
    int32_t i = bi[e], j = bj[e];
    const double *r = rhat + 3 * e;
    double sij = 0.0, sji = 0.0, sii = 0.0, sjj = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double rr = r[a] * r[b];
        sij += vbar[or_find(H, 3 * (int64_t)i + a, 3 * j + b)] * rr;
        sji += vbar[or_find(H, 3 * (int64_t)j + a, 3 * i + b)] * rr;
        sii += vbar[or_find(H, 3 * (int64_t)i + a, 3 * i + b)] * rr;
        sjj += vbar[or_find(H, 3 * (int64_t)j + a, 3 * j + b)] * rr;
      }
    kbar[e] = -(sij + sji) / sqrt(mass[i] * mass[j]) + sii / mass[i] + sjj / mass[j];
  }
  for (int32_t i = 0; i < N; ++i) {
    double off = 0.0, dia = 0.0;
    for (int a = 0; a < 3; ++a) {
      int64_t row = 3 * (int64_t)i + a;
      for (int64_t p = H->rp[row]; p < H->rp[row + 1]; ++p) {
        int32_t blk = H->ci[p] / 3;
        double hv = vbar[p] * H->v[p];
        if (blk == i) dia += hv;
        else off += hv;
      }
    }
    /* the column side: entries (j, i) in rows of the neighbours j -- by symmetry of the
       pattern, walk row i's neighbour blocks and read their (j, i) entries */
    for (int a = 0; a < 3; ++a) {
      int64_t row = 3 * (int64_t)i + a;
      for (int64_t p = H->rp[row]; p < H->rp[row + 1]; ++p) {
        int32_t cc = H->ci[p], blk = cc / 3;
        if (blk == i) continue;
        int64_t q = or_find(H, cc, 3 * i + a);
        off += vbar[q] * H->v[q];
      }
    }
    mbar[i] = -off / (2.0 * mass[i]) - dia / mass[i];
  }
}

/* ======================================================================================
 * Thick-restart block Lanczos on the filter operator Op = p(Ht) (Sec. 2.5 and Sec. 3: the block
 * Krylov-Schur / thick-restart Lanczos eigensolver applied to the matrix polynomial), followed by
 * Rayleigh-Ritz with H on the converged wanted Op-eigenvectors (Sec. 2.5: "the correct
 * eigenvalue-eigenvector relations can be found by a Rayleigh-Ritz procedure applied to H").
 *
 * Krylov basis V (orthonormal, block size bs) and OV = Op V for its first nv columns.
 *   expand:  OV_j = Op V_j; W = OV_j - V (V^T OV_j) (twice); V_{j+1} = QR(W) (twice against V)
 *   restart: T = V^T OV (nv x nv), T = S Theta S^T (Jacobi), Y = V S, OY = OV S,
 *            r_i = ||OY_i - theta_i Y_i||; keep the `keep` largest Ritz pairs as the new basis and
 *            the last block V_{j+1} (orthogonal to all of V) as the continuation block.
 *   stop:    every Ritz pair with theta >= theta_cut has r_i <= tol_op * max|theta|, at least one
 *            block of Ritz values lies below theta_cut (the wanted set is not truncated), and the
 *            number of wanted Ritz pairs equals that of the previous restart.
 * Final:    A = Yw^T H Yw for the wanted converged Yw, A = Q Lambda Q^T, U = Yw Q; pairs with lambda
 *            in [a, b] and residual ||H u - lambda u|| / lmax <= tol are returned, ascending.  If a
 *            returned residual exceeds tol, tol_op is divided by 100 and the iteration continues.
 * Returns 0 on success, 1 iteration limit, 2 capacity exceeded, <0 bad input.
 * ==================================================================================== */
static void or_cgs2(int64_t n, const double *V, int32_t nv, double *W, int32_t k, double *h) {
  for (int pass = 0; pass < 2; ++pass)
    for (int32_t c = 0; c < k; ++c) {
      double *w = W + (int64_t)c * n;
      for (int32_t l = 0; l < nv; ++l) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += V[(int64_t)l * n + i] * w[i];
        h[l] = s;
      }
      for (int32_t l = 0; l < nv; ++l)
        for (int64_t i = 0; i < n; ++i) w[i] -= h[l] * V[(int64_t)l * n + i];
    }
}

int or_bks_solve(const or_csr *H, double a, double b, double lmin, double lmax, const double *coef, int32_t m,
                 int32_t bs, int32_t maxbasis, int32_t keep_min, const double *X0, double theta_cut, double tol,
                 int32_t max_restarts, int32_t cap, int32_t *n_found, double *lam_out, double *vec_out,
                 double *res_out, int32_t *restarts_out, int64_t *matvecs_out) {
  const int64_t n = H->n;
  if (bs < 1 || maxbasis < 3 * bs || maxbasis + bs > n) return -1;
  const double c = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
  double *V = (double *)calloc((size_t)n * (size_t)(maxbasis + bs), sizeof(double));
  double *OV = (double *)calloc((size_t)n * (size_t)maxbasis, sizeof(double));
  double *Y = (double *)malloc(sizeof(double) * (size_t)n * maxbasis);
  double *OY = (double *)malloc(sizeof(double) * (size_t)n * maxbasis);
  double *T = (double *)malloc(sizeof(double) * (size_t)maxbasis * maxbasis);
  double *S = (double *)malloc(sizeof(double) * (size_t)maxbasis * maxbasis);
  double *th = (double *)malloc(sizeof(double) * (size_t)maxbasis);
  double *rr = (double *)malloc(sizeof(double) * (size_t)maxbasis);
  double *h = (double *)malloc(sizeof(double) * (size_t)(maxbasis + bs));
  int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)maxbasis);
  if (!V || !OV || !Y || !OY || !T || !S || !th || !rr || !h || !ord) {
    free(V); free(OV); free(Y); free(OY); free(T); free(S); free(th); free(rr); free(h); free(ord);
    return -4;
  }
  memcpy(V, X0, sizeof(double) * (size_t)n * bs);
  or_householder_qr(n, bs, V, n, NULL);
  int32_t nv = 0, restarts = 0, status = 1, nf = 0, prev_nwant = -1;
  int64_t mv = 0;
  double tol_op = 1e-10;
  for (;;) {
    /* expand the basis (with Op applied) while another block fits into maxbasis columns */
    while (nv + bs <= maxbasis) {
      double *Vj = V + (int64_t)nv * n, *OVj = OV + (int64_t)nv * n;
      mv += or_cheb_filter(H, c, d, coef, m, bs, Vj, n, OVj, n);
      double *Wn = V + (int64_t)(nv + bs) * n;
      memcpy(Wn, OVj, sizeof(double) * (size_t)n * bs);
      or_cgs2(n, V, nv + bs, Wn, bs, h);
      or_householder_qr(n, bs, Wn, n, NULL);
      or_cgs2(n, V, nv + bs, Wn, bs, h);
      or_householder_qr(n, bs, Wn, n, NULL);
      nv += bs;
    }
    /* Rayleigh-Ritz of Op on span(V) */
    for (int32_t j = 0; j < nv; ++j)
      for (int32_t i = 0; i < nv; ++i) {
        double s = 0.0;
        for (int64_t r = 0; r < n; ++r) s += V[(int64_t)i * n + r] * OV[(int64_t)j * n + r];
        T[(int64_t)j * nv + i] = s;
      }
    for (int32_t j = 0; j < nv; ++j)
      for (int32_t i = 0; i < j; ++i) {
        double s = 0.5 * (T[(int64_t)j * nv + i] + T[(int64_t)i * nv + j]);
        T[(int64_t)j * nv + i] = s;
        T[(int64_t)i * nv + j] = s;
      }
    or_jacobi_eig(nv, T, th, S);
    for (int32_t i = 0; i < nv; ++i) ord[i] = nv - 1 - i; /* descending theta */
    for (int32_t jj = 0; jj < nv; ++jj) {
      int32_t j = ord[jj];
      for (int64_t r = 0; r < n; ++r) {
        double sy = 0.0, so = 0.0;
        for (int32_t i = 0; i < nv; ++i) {
          double sij = S[(int64_t)j * nv + i];
          sy += V[(int64_t)i * n + r] * sij;
          so += OV[(int64_t)i * n + r] * sij;
        }
        Y[(int64_t)jj * n + r] = sy;
        OY[(int64_t)jj * n + r] = so;
      }
      double s2 = 0.0;
      for (int64_t r = 0; r < n; ++r) {
        double e = OY[(int64_t)jj * n + r] - th[j] * Y[(int64_t)jj * n + r];
        s2 += e * e;
      }
      rr[jj] = sqrt(s2);
    }
    double thmax = fabs(th[ord[0]]);
    int32_t nwant = 0, nconv = 0;
    for (int32_t jj = 0; jj < nv; ++jj)
      if (th[ord[jj]] >= theta_cut) {
        ++nwant;
        if (rr[jj] <= tol_op * thmax) ++nconv;
      }
    int done = (nwant == nconv) && (nwant <= nv - bs) && (nwant == prev_nwant);
    prev_nwant = nwant;
    if (done) {
      /* Rayleigh-Ritz with H on the wanted Op-eigenvectors (the first nwant columns of Y) */
      int32_t k = nwant;
      double *HY = OY; /* reuse */
      or_spmm(H, k, Y, n, HY, n);
      mv += k;
      double *A = T, *Q = S;
      for (int32_t j = 0; j < k; ++j)
        for (int32_t i = 0; i < k; ++i) {
          double s = 0.0;
          for (int64_t r = 0; r < n; ++r) s += Y[(int64_t)i * n + r] * HY[(int64_t)j * n + r];
          A[(int64_t)j * k + i] = s;
        }
      for (int32_t j = 0; j < k; ++j)
        for (int32_t i = 0; i < j; ++i) {
          double s = 0.5 * (A[(int64_t)j * k + i] + A[(int64_t)i * k + j]);
          A[(int64_t)j * k + i] = s;
          A[(int64_t)i * k + j] = s;
        }
      double *ev = rr; /* k <= maxbasis */
      or_jacobi_eig(k, A, ev, Q);
      double *U = OV; /* n x k */
      for (int32_t j = 0; j < k; ++j)
        for (int64_t r = 0; r < n; ++r) {
          double s = 0.0;
          for (int32_t i = 0; i < k; ++i) s += Y[(int64_t)i * n + r] * Q[(int64_t)j * k + i];
          U[(int64_t)j * n + r] = s;
        }
      double *w = (double *)malloc(sizeof(double) * (size_t)n);
      int bad = 0;
      nf = 0;
      for (int32_t j = 0; j < k; ++j) {
        if (ev[j] < a || ev[j] > b) continue;
        or_spmm(H, 1, U + (int64_t)j * n, n, w, n);
        double s2 = 0.0;
        for (int64_t r = 0; r < n; ++r) {
          double e = w[r] - ev[j] * U[(int64_t)j * n + r];
          s2 += e * e;
        }
        double res = sqrt(s2) / lmax;
        if (res > tol) bad = 1;
        if (nf < cap) {
          lam_out[nf] = ev[j];
          if (res_out) res_out[nf] = res;
          if (vec_out) memcpy(vec_out + (int64_t)nf * n, U + (int64_t)j * n, sizeof(double) * (size_t)n);
        }
        ++nf;
      }
      free(w);
      if (!bad || tol_op < 1e-15) {
        status = (nf > cap) ? 2 : (bad ? 1 : 0);
        break;
      }
      tol_op *= 1e-2; /* the Op-residuals were not small enough for the H-residuals: iterate on */
      /* the basis was overwritten by the final Rayleigh-Ritz: restore it from Y (kept below) */
    }
    if (++restarts > max_restarts) {
      status = 1;
      nf = 0;
      break;
    }
    /* thick restart: keep the `keep` largest Ritz pairs plus the continuation block */
    int32_t keep = nwant + bs;
    if (keep < keep_min) keep = keep_min;
    if (keep > nv - bs) keep = nv - bs;
    if (done) {
      /* OY was reused for H Y: recompute Op Y for the kept columns from the stored basis is not
         possible, so rebuild OY = OV_old S is lost; fall back to re-applying Op to the kept block */
      memcpy(V, Y, sizeof(double) * (size_t)n * keep);
      mv += or_cheb_filter(H, c, d, coef, m, keep, V, n, OV, n);
    } else {
      memcpy(V, Y, sizeof(double) * (size_t)n * keep);
      memcpy(OV, OY, sizeof(double) * (size_t)n * keep);
    }
    /* continuation block: the last Krylov block, orthogonal to the old basis */
    memmove(V + (int64_t)keep * n, V + (int64_t)nv * n, sizeof(double) * (size_t)n * bs);
    or_cgs2(n, V, keep, V + (int64_t)keep * n, bs, h);
    or_householder_qr(n, bs, V + (int64_t)keep * n, n, NULL);
    nv = keep;
  }
  *n_found = nf;
  if (restarts_out) *restarts_out = restarts;
  if (matvecs_out) *matvecs_out = mv;
  /* ascending order of the returned pairs (Jacobi already returns ascending eigenvalues) */
  free(V); free(OV); free(Y); free(OY); free(T); free(S); free(th); free(rr); free(h); free(ord);
  return status;
}

/* ======================================================================================
 * Analysis of the computed modes, Sec. 4.4
 * ==================================================================================== */

/* Participation ratio, eq. (PR_def): PR = 1 / sum_i |q_i|^4 for a mode of unit 2-norm, q_i the
 * 3-vector of atom i.  The paper then reads PR = 1 for |q_i| = 1/sqrt(N) and PR = 1/N for a
 * single atom, which is the printed formula divided by N; this routine returns that normalised
 * value, with the unit-norm assumption written out: (sum |q_i|^2)^2 / (N sum |q_i|^4).
 * V: n x k column-major (n = 3 n_atoms), ld ldv. */
void or_participation_ratio(int64_t n_atoms, int32_t k, const double *V, int64_t ldv, double *pr) {
  for (int32_t c = 0; c < k; ++c) {
    const double *q = V + (int64_t)c * ldv;
    double s2 = 0.0, s4 = 0.0;
    for (int64_t i = 0; i < n_atoms; ++i) {
      double w = q[3 * i] * q[3 * i] + q[3 * i + 1] * q[3 * i + 1] + q[3 * i + 2] * q[3 * i + 2];
      s2 += w;
      s4 += w * w;
    }
    pr[c] = (s4 > 0.0) ? s2 * s2 / ((double)n_atoms * s4) : 0.0;
  }
}

/* Plane-wave content of each mode for wave vectors kvec[w] (Sec. 4.4: a plane wave of wave
 * vector k and polarisation zeta is q_i = sqrt(2/N) zeta sin(k . r_i), r_i the atom position):
 * the squared projections onto sqrt(2/N) zeta sin(k . r_i) and sqrt(2/N) zeta cos(k . r_i), summed
 * over both and over the polarisations along k (out[.. 0]) and across k (out[.. 1]), divided by
 * |q|^2.  Written with A_d = sum_i q_{i,d} (cos + i sin)(k . r_i):
 *   longitudinal (2/N) |khat . A|^2 / |q|^2, transverse (2/N) (|A|^2 - |khat . A|^2) / |q|^2.
 * out[(c * nk + w) * 2 + {0, 1}].  pos: 3 n_atoms; kvec: 3 nk, each nonzero. */
void or_plane_wave_content(int64_t n_atoms, int32_t k, const double *V, int64_t ldv, const double *pos, int32_t nk,
                           const double *kvec, double *out) {
  for (int32_t c = 0; c < k; ++c) {
    const double *q = V + (int64_t)c * ldv;
    double nrm2 = 0.0;
    for (int64_t i = 0; i < 3 * n_atoms; ++i) nrm2 += q[i] * q[i];
    for (int32_t w = 0; w < nk; ++w) {
      const double *kv = kvec + 3 * w;
      double re[3] = {0.0, 0.0, 0.0}, im[3] = {0.0, 0.0, 0.0};
      for (int64_t i = 0; i < n_atoms; ++i) {
        double ph = kv[0] * pos[3 * i] + kv[1] * pos[3 * i + 1] + kv[2] * pos[3 * i + 2];
        double cs = cos(ph), sn = sin(ph);
        for (int d = 0; d < 3; ++d) {
          re[d] += q[3 * i + d] * cs;
          im[d] += q[3 * i + d] * sn;
        }
      }
      double kn = sqrt(kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2]);
      double lre = 0.0, lim = 0.0, tot = 0.0;
      for (int d = 0; d < 3; ++d) {
        lre += kv[d] / kn * re[d];
        lim += kv[d] / kn * im[d];
        tot += re[d] * re[d] + im[d] * im[d];
      }
      double l2 = lre * lre + lim * lim;
      double sc = (nrm2 > 0.0) ? 2.0 / ((double)n_atoms * nrm2) : 0.0;
      out[((int64_t)c * nk + w) * 2] = sc * l2;
      out[((int64_t)c * nk + w) * 2 + 1] = sc * (tot - l2);
    }
  }
}

/* ======================================================================================
 * The Dirac polynomial filter, Sec. 2.5, eq. (cheby-delta.1)
 * ==================================================================================== */

/* Damped Chebyshev coefficients of the degree-k representative of delta(t - gamma):
 * c_j = g_j T_j(gamma) / <T_j, T_j>, <T_0, T_0> = pi, <T_j, T_j> = pi / 2 (eq. (cheby-delta.1)),
 * with the damping factors g_j of or_damping. */
void or_dirac_coeffs(double gamma, int32_t k, int kind, double *c) {
  double *g = (double *)malloc(sizeof(double) * (size_t)(k + 1));
  or_damping(kind, k, g);
  double th = acos(gamma);
  for (int32_t j = 0; j <= k; ++j) c[j] = g[j] * cos((double)j * th) / (j == 0 ? OR_PI : OR_PI / 2.0);
  free(g);
}

/* gamma in (xi, eta) with rho_k(xi) = rho_k(eta) (Sec. 2.5 and Sec. 3: gamma close to the midpoint),
 * by bisection on rho_k(xi) - rho_k(eta), which is positive while gamma sits too close to xi. */
double or_dirac_gamma(double xi, double eta, int32_t k, int kind) {
  double *c = (double *)malloc(sizeof(double) * (size_t)(k + 1));
  double lo = xi, hi = eta;
  for (int it = 0; it < 100; ++it) {
    double mid = 0.5 * (lo + hi);
    or_dirac_coeffs(mid, k, kind, c);
    double f = or_series_value(c, k, xi) - or_series_value(c, k, eta);
    if (f > 0.0) lo = mid;
    else hi = mid;
  }
  free(c);
  return 0.5 * (lo + hi);
}

/* Degree of the Dirac filter: the smallest k >= 2 whose balanced filter has
 * rho_k(xi) / rho_k(gamma) <= phi (the parameter phi of Tables 1-3: the filter value at the interval
 * edges relative to its peak).  Returns -1 if no k <= kmax qualifies. */
int32_t or_dirac_degree(double xi, double eta, double phi, int kind, int32_t kmax) {
  double *c = (double *)malloc(sizeof(double) * (size_t)(kmax + 1));
  int32_t found = -1;
  for (int32_t k = 2; k <= kmax; ++k) {
    double gm = or_dirac_gamma(xi, eta, k, kind);
    or_dirac_coeffs(gm, k, kind, c);
    if (or_series_value(c, k, xi) / or_series_value(c, k, gm) <= phi) {
      found = k;
      break;
    }
  }
  free(c);
  return found;
}
