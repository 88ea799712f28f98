/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the inverse-factorization path.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this code; the library's compute path never does.
 * It shares no code, header or helper with the CUDA path.
 *
 * What it computes (paper: Artemov, Rudberg, Rubensson, "Parallelization and
 * scalability analysis of inverse factorization using the Chunks and Tasks
 * programming model", arXiv:1901.07993):
 *
 *  - om_truncate: removal of blocks whose Frobenius norm is below tau
 *    (Section 5: blocks with norm smaller than the threshold are removed).
 *  - om_gemm: C = alpha * op(A) op(B) on stored blocks, then truncation of
 *    the output blocks (Section 5: truncation after every product).
 *  - om_add: alpha A + beta B + gamma I on the union of patterns (no
 *    truncation: the paper truncates after products and leaf routines only).
 *  - om_gershgorin: beta = max_i sum_j |S_ij| (Section 2.2, Eq. for c with
 *    the Gershgorin estimate of the spectral radius).
 *  - om_irsi: iterative refinement from a scaled identity, Eq. (2.1) with
 *    delta_i = I - Z_i^T S Z_i evaluated directly each sweep (or, with
 *    local_delta, updated by Eq. (2.2) after a direct delta_0), Z_0 = c I,
 *    and the automatic stop ||delta_{i+1}||_F > ||delta_i||_F^{m+1}
 *    (Section 2.2).
 *  - om_lif: localized inverse factorization, Algorithm 2, with the localized
 *    refinement of Eq. (2.2) and the stop rule as in Algorithm 4.
 *  - om_invchol_dense: the leaf routine "factorize S^-1 = Z Z^T" of
 *    Algorithms 1-2, as Cholesky S = L L^T and Z = L^-T.
 *  - om_rinch: recursive inverse Cholesky, Algorithm 1 (left-looking, two
 *    blocks per dimension), with the leaf routine above at the lowest level.
 *
 * Every loop is the definition written out; there is no blocking, fusion or
 * reordering beyond the block structure the paper's storage itself has.
 * om_gemm forms its output block rows independently; with OpenMP they are
 * spread over threads (om_set_threads), which changes no result: every
 * block row is summed in the same order by whichever thread forms it.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int64_t n;       /* logical dimension */
  int32_t bs;      /* block size */
  int32_t nb;      /* block rows = block cols = ceil(n / bs) */
  int64_t nnzb;    /* stored blocks */
  int32_t* row_ptr;  /* [nb + 1] */
  int32_t* col_idx;  /* [nnzb], increasing within each row */
  double* val;       /* [nnzb * bs * bs], block p row-major at val + p*bs*bs */
} om_mat;

typedef struct {
  int m;            /* refinement order (number of delta powers), >= 1 */
  double tau;       /* block truncation threshold */
  double target;    /* stop once ||delta||_F <= target */
  int max_iter;     /* hard cap on sweeps per refinement */
  int fixed_iters;  /* IRSI only: if > 0, run exactly this many corrections */
  int c_rule;       /* IRSI start: 0 -> c = 1/sqrt(beta), 1 -> c = sqrt(2/beta) */
  int leaf_size;    /* LIF, RINCH: recurse while a sub-problem has more rows */
  int rinch_rows;   /* LIF: sub-problems with at most this many rows (> leaf_size)
                       are factorized by RINCH instead of split further; 0 = off */
  int local_delta;  /* IRSI: 0 direct delta each sweep, 1 the local update of
                       Eq. (2.2) after a direct delta_0 */
} om_opts;

enum { OM_STOP_RULE = 1, OM_STOP_TARGET = 2, OM_STOP_MAXITER = 3, OM_STOP_FIXED = 4 };

typedef struct {
  int sweeps;          /* corrections applied (IRSI) / total over levels (LIF) */
  int stop_reason;     /* of the last refinement (IRSI) / of the top level (LIF) */
  int levels;          /* LIF: recursion levels above the leaves */
  double beta;         /* IRSI: Gershgorin bound */
  double delta_fro[64];  /* IRSI: ||delta_i||_F per evaluation; LIF: top level */
  int n_delta;
  int64_t products;    /* number of block-sparse products performed */
  int64_t block_pairs; /* stored-block pairs multiplied over all products */
  int status;          /* 0 ok; -2 leaf not positive definite; -1 alloc */
} om_report;

/* ------------------------------------------------------------------ */
/* Storage helpers                                                      */
/* ------------------------------------------------------------------ */

static om_mat* om_new(int64_t n, int bs, int nb, int64_t nnzb) {
  om_mat* a = (om_mat*)calloc(1, sizeof(om_mat));
  a->n = n; a->bs = bs; a->nb = nb; a->nnzb = nnzb;
  a->row_ptr = (int32_t*)calloc((size_t)nb + 1, sizeof(int32_t));
  a->col_idx = (int32_t*)malloc((size_t)(nnzb > 0 ? nnzb : 1) * sizeof(int32_t));
  a->val = (double*)malloc((size_t)(nnzb > 0 ? nnzb : 1) * bs * bs * sizeof(double));
  return a;
}

void om_free(om_mat* a) {
  if (!a) return;
  free(a->row_ptr); free(a->col_idx); free(a->val); free(a);
}

/* Wrap caller arrays (copied, so the oracle owns its matrices). */
om_mat* om_from_arrays(int64_t n, int bs, int nb, int64_t nnzb, const int32_t* row_ptr,
                       const int32_t* col_idx, const double* val) {
  om_mat* a = om_new(n, bs, nb, nnzb);
  memcpy(a->row_ptr, row_ptr, ((size_t)nb + 1) * sizeof(int32_t));
  memcpy(a->col_idx, col_idx, (size_t)nnzb * sizeof(int32_t));
  memcpy(a->val, val, (size_t)nnzb * bs * bs * sizeof(double));
  return a;
}

int64_t om_nnzb(const om_mat* a) { return a->nnzb; }
int32_t om_nb(const om_mat* a) { return a->nb; }
int64_t om_n(const om_mat* a) { return a->n; }

void om_to_arrays(const om_mat* a, int32_t* row_ptr, int32_t* col_idx, double* val) {
  memcpy(row_ptr, a->row_ptr, ((size_t)a->nb + 1) * sizeof(int32_t));
  memcpy(col_idx, a->col_idx, (size_t)a->nnzb * sizeof(int32_t));
  memcpy(val, a->val, (size_t)a->nnzb * a->bs * a->bs * sizeof(double));
}

/* Growable builder: blocks are appended row by row in increasing column. */
typedef struct {
  om_mat* m;
  int64_t cap;
} om_builder;

static om_builder ob_begin(int64_t n, int bs, int nb) {
  om_builder b;
  b.cap = (int64_t)nb * 4 + 8;
  b.m = om_new(n, bs, nb, b.cap);
  b.m->nnzb = 0;
  return b;
}

static double* ob_push(om_builder* b, int32_t col) {
  size_t bsz = (size_t)b->m->bs * b->m->bs;
  if (b->m->nnzb == b->cap) {
    b->cap *= 2;
    b->m->col_idx = (int32_t*)realloc(b->m->col_idx, (size_t)b->cap * sizeof(int32_t));
    b->m->val = (double*)realloc(b->m->val, (size_t)b->cap * bsz * sizeof(double));
  }
  b->m->col_idx[b->m->nnzb] = col;
  return b->m->val + (size_t)(b->m->nnzb++) * bsz;
}

static void ob_end_row(om_builder* b, int row) { b->m->row_ptr[row + 1] = (int32_t)b->m->nnzb; }

/* Frobenius norm of one bs x bs block: sqrt of the plain sum of squares. */
static double block_fro(const double* blk, int bs) {
  double s = 0.0;
  for (int i = 0; i < bs * bs; ++i) s += blk[i] * blk[i];
  return sqrt(s);
}

double om_block_fro(const om_mat* a, int64_t p) {
  return block_fro(a->val + (size_t)p * a->bs * a->bs, a->bs);
}

/* ------------------------------------------------------------------ */
/* Truncation, transpose, sub-matrices                                  */
/* ------------------------------------------------------------------ */

/* Keep the blocks with ||B||_F >= tau (drop when strictly below). */
om_mat* om_truncate(const om_mat* a, double tau) {
  size_t bsz = (size_t)a->bs * a->bs;
  om_builder b = ob_begin(a->n, a->bs, a->nb);
  for (int i = 0; i < a->nb; ++i) {
    for (int p = a->row_ptr[i]; p < a->row_ptr[i + 1]; ++p) {
      const double* blk = a->val + (size_t)p * bsz;
      if (block_fro(blk, a->bs) < tau) continue;
      memcpy(ob_push(&b, a->col_idx[p]), blk, bsz * sizeof(double));
    }
    ob_end_row(&b, i);
  }
  return b.m;
}

/* Explicit transpose: block (i, j) of A^T is (block (j, i) of A)^T.  Rows of
 * A^T are filled by scanning A's rows in increasing order, so the columns of
 * each row of A^T come out increasing. */
om_mat* om_transpose(const om_mat* a) {
  int bs = a->bs, nb = a->nb;
  size_t bsz = (size_t)bs * bs;
  om_mat* t = om_new(a->n, bs, nb, a->nnzb);
  int32_t* next = (int32_t*)calloc((size_t)nb + 1, sizeof(int32_t));
  for (int64_t p = 0; p < a->nnzb; ++p) t->row_ptr[a->col_idx[p] + 1]++;
  for (int i = 0; i < nb; ++i) t->row_ptr[i + 1] += t->row_ptr[i];
  for (int i = 0; i < nb; ++i) next[i] = t->row_ptr[i];
  for (int j = 0; j < nb; ++j)
    for (int p = a->row_ptr[j]; p < a->row_ptr[j + 1]; ++p) {
      int i = a->col_idx[p];
      int q = next[i]++;
      t->col_idx[q] = j;
      const double* src = a->val + (size_t)p * bsz;
      double* dst = t->val + (size_t)q * bsz;
      for (int r = 0; r < bs; ++r)
        for (int c = 0; c < bs; ++c) dst[r * bs + c] = src[c * bs + r];
    }
  free(next);
  return t;
}

/* Square sub-matrix on block rows [r0, r1) x block cols [c0, c1). */
static om_mat* om_sub(const om_mat* a, int r0, int r1, int c0, int c1) {
  size_t bsz = (size_t)a->bs * a->bs;
  int64_t n = (int64_t)(r1 - r0) * a->bs;
  om_builder b = ob_begin(n, a->bs, r1 - r0);
  b.m->n = n;
  for (int i = r0; i < r1; ++i) {
    for (int p = a->row_ptr[i]; p < a->row_ptr[i + 1]; ++p) {
      int j = a->col_idx[p];
      if (j < c0 || j >= c1) continue;
      memcpy(ob_push(&b, j - c0), a->val + (size_t)p * bsz, bsz * sizeof(double));
    }
    ob_end_row(&b, i - r0);
  }
  return b.m;
}

/* Rectangular-as-square helper: the oracle keeps every matrix square with nb
 * block rows; for the off-diagonal coupling block B of S = [A B; B^T C] we
 * embed it in the sub-problem's full index space instead (rows [0, na),
 * cols [na, na + nc)), so every product is between square matrices of the
 * sub-problem's dimension. */
static om_mat* om_sub_embedded(const om_mat* a, int b0, int b1, int r0, int r1, int c0, int c1) {
  size_t bsz = (size_t)a->bs * a->bs;
  int nbs = b1 - b0;
  om_builder b = ob_begin((int64_t)nbs * a->bs, a->bs, nbs);
  for (int i = b0; i < b1; ++i) {
    if (i >= r0 && i < r1) {
      for (int p = a->row_ptr[i]; p < a->row_ptr[i + 1]; ++p) {
        int j = a->col_idx[p];
        if (j < c0 || j >= c1) continue;
        memcpy(ob_push(&b, j - b0), a->val + (size_t)p * bsz, bsz * sizeof(double));
      }
    }
    ob_end_row(&b, i - b0);
  }
  return b.m;
}

/* ------------------------------------------------------------------ */
/* Products, sums, norms                                                */
/* ------------------------------------------------------------------ */

static int64_t g_products = 0, g_pairs = 0;

/*
 * C = alpha * op(A) op(B), then drop output blocks with ||C_IJ||_F < tau.
 * op(X) = X^T when tX != 0.  C_IJ = alpha * sum over K of op(A)_IK op(B)_KJ,
 * summed over the stored blocks only; the output pattern is every (I, J) for
 * which some K has both blocks stored.
 */
om_mat* om_gemm(const om_mat* A, int tA, const om_mat* B, int tB, double alpha, double tau) {
  const om_mat* a = A;
  const om_mat* b = B;
  om_mat* at = NULL;
  om_mat* bt = NULL;
  if (tA) a = at = om_transpose(A);
  if (tB) b = bt = om_transpose(B);
  int bs = a->bs, nb = a->nb;
  size_t bsz = (size_t)bs * bs;
  /* Output block rows are independent: each is formed on its own (by one
   * thread when OpenMP is on) into a row buffer, and the rows are then
   * appended in order.  A row's arithmetic is the same whatever the thread
   * count, so results are identical with one thread or many. */
  int32_t** row_cols = (int32_t**)calloc((size_t)nb, sizeof(int32_t*));
  double** row_vals = (double**)calloc((size_t)nb, sizeof(double*));
  int* row_n = (int*)calloc((size_t)nb, sizeof(int));
  int64_t pairs = 0;
  g_products++;
#pragma omp parallel reduction(+ : pairs)
  {
    double* acc = (double*)malloc((size_t)nb * bsz * sizeof(double));
    char* touched = (char*)calloc((size_t)nb, 1);
#pragma omp for schedule(dynamic, 4)
    for (int I = 0; I < nb; ++I) {
      int ncols = 0;
      for (int p = a->row_ptr[I]; p < a->row_ptr[I + 1]; ++p) {
        int K = a->col_idx[p];
        const double* aik = a->val + (size_t)p * bsz;
        for (int q = b->row_ptr[K]; q < b->row_ptr[K + 1]; ++q) {
          int J = b->col_idx[q];
          const double* bkj = b->val + (size_t)q * bsz;
          double* cij = acc + (size_t)J * bsz;
          if (!touched[J]) {
            touched[J] = 1;
            ++ncols;
            memset(cij, 0, bsz * sizeof(double));
          }
          pairs++;
          for (int i = 0; i < bs; ++i)
            for (int k = 0; k < bs; ++k) {
              double x = aik[i * bs + k];
              for (int j = 0; j < bs; ++j) cij[i * bs + j] += x * bkj[k * bs + j];
            }
        }
      }
      /* scale, truncate and keep in increasing J */
      int32_t* cols = (int32_t*)malloc((size_t)(ncols ? ncols : 1) * sizeof(int32_t));
      double* vals = (double*)malloc((size_t)(ncols ? ncols : 1) * bsz * sizeof(double));
      int kept = 0;
      for (int J = 0, left = ncols; J < nb && left > 0; ++J) {
        if (!touched[J]) continue;
        --left;
        touched[J] = 0;
        double* cij = acc + (size_t)J * bsz;
        for (size_t e = 0; e < bsz; ++e) cij[e] *= alpha;
        if (block_fro(cij, bs) < tau) continue;
        cols[kept] = J;
        memcpy(vals + (size_t)kept * bsz, cij, bsz * sizeof(double));
        ++kept;
      }
      row_cols[I] = cols;
      row_vals[I] = vals;
      row_n[I] = kept;
    }
    free(acc);
    free(touched);
  }
  g_pairs += pairs;
  om_builder out = ob_begin(A->n, bs, nb);
  for (int I = 0; I < nb; ++I) {
    for (int e = 0; e < row_n[I]; ++e) memcpy(ob_push(&out, row_cols[I][e]), row_vals[I] + (size_t)e * bsz,
                                              bsz * sizeof(double));
    ob_end_row(&out, I);
    free(row_cols[I]);
    free(row_vals[I]);
  }
  free(row_cols); free(row_vals); free(row_n);
  om_free(at); om_free(bt);
  return out.m;
}

/* Threads of the parallel loops (OpenMP builds; 1 otherwise). */
#ifdef _OPENMP
#include <omp.h>
void om_set_threads(int t) { omp_set_num_threads(t > 0 ? t : 1); }
int om_max_threads(void) { return omp_get_max_threads(); }
#else
void om_set_threads(int t) { (void)t; }
int om_max_threads(void) { return 1; }
#endif

/* C = alpha A + beta B + gamma I on the union pattern (B may be NULL).
 * Per row, the sorted column lists of A, B and the diagonal are merged. */
om_mat* om_add(double alpha, const om_mat* A, double beta, const om_mat* B, double gamma) {
  int bs = A->bs, nb = A->nb;
  size_t bsz = (size_t)bs * bs;
  om_builder out = ob_begin(A->n, bs, nb);
  for (int I = 0; I < nb; ++I) {
    int pa = A->row_ptr[I], ea = A->row_ptr[I + 1];
    int pb = B ? B->row_ptr[I] : 0, eb = B ? B->row_ptr[I + 1] : 0;
    int need_diag = (gamma != 0.0);
    for (;;) {
      int ja = (pa < ea) ? A->col_idx[pa] : nb;
      int jb = (pb < eb) ? B->col_idx[pb] : nb;
      int jd = need_diag ? I : nb;
      int J = ja < jb ? ja : jb;
      if (jd < J) J = jd;
      if (J >= nb) break;
      const double* a = (ja == J) ? A->val + (size_t)pa++ * bsz : NULL;
      const double* b = (jb == J) ? B->val + (size_t)pb++ * bsz : NULL;
      if (jd == J) need_diag = 0;
      double* c = ob_push(&out, J);
      for (int r = 0; r < bs; ++r)
        for (int s = 0; s < bs; ++s) {
          double v = 0.0;
          if (a) v += alpha * a[r * bs + s];
          if (b) v += beta * b[r * bs + s];
          if (I == J && r == s) v += gamma;
          c[r * bs + s] = v;
        }
    }
    ob_end_row(&out, I);
  }
  return out.m;
}

double om_fro(const om_mat* a) {
  double s = 0.0;
  size_t tot = (size_t)a->nnzb * a->bs * a->bs;
  for (size_t e = 0; e < tot; ++e) s += a->val[e] * a->val[e];
  return sqrt(s);
}

/* beta = max over rows i of sum_j |S_ij| (Gershgorin bound on lambda_max). */
double om_gershgorin(const om_mat* s) {
  int bs = s->bs;
  double best = 0.0;
  for (int I = 0; I < s->nb; ++I)
    for (int r = 0; r < bs; ++r) {
      double row = 0.0;
      for (int p = s->row_ptr[I]; p < s->row_ptr[I + 1]; ++p)
        for (int c = 0; c < bs; ++c) row += fabs(s->val[(size_t)p * bs * bs + (size_t)r * bs + c]);
      if (row > best) best = row;
    }
  return best;
}

static om_mat* om_scaled_identity(int64_t n, int bs, int nb, double c) {
  om_builder out = ob_begin(n, bs, nb);
  for (int I = 0; I < nb; ++I) {
    double* blk = ob_push(&out, I);
    memset(blk, 0, (size_t)bs * bs * sizeof(double));
    for (int r = 0; r < bs; ++r) blk[r * bs + r] = c;
    ob_end_row(&out, I);
  }
  return out.m;
}

/* Refinement coefficients b_0 = 1, b_k = (2k-1)/(2k) b_{k-1}. */
static double coef_b(int k) {
  double b = 1.0;
  for (int j = 1; j <= k; ++j) b = b * (double)(2 * j - 1) / (double)(2 * j);
  return b;
}

double om_coef_b(int k) { return coef_b(k); }

/* P = sum_{k=1}^{m} b_k delta^k; powers by successive truncated products. */
static om_mat* poly_P(const om_mat* delta, int m, double tau) {
  om_mat* P = om_add(coef_b(1), delta, 0.0, NULL, 0.0);
  om_mat* D = NULL;
  for (int k = 2; k <= m; ++k) {
    om_mat* Dn = om_gemm(k == 2 ? delta : D, 0, delta, 0, 1.0, tau);
    om_free(D);
    D = Dn;
    om_mat* Pn = om_add(1.0, P, coef_b(k), D, 0.0);
    om_free(P);
    P = Pn;
  }
  om_free(D);
  return P;
}

static void rep_reset_counters(void) { g_products = 0; g_pairs = 0; }

/* ------------------------------------------------------------------ */
/* IRSI: iterative refinement from a scaled identity                    */
/* ------------------------------------------------------------------ */

/* delta = I - Z^T (S Z), both products truncated */
static om_mat* irsi_direct_delta(const om_mat* S, const om_mat* Z, double tau) {
  om_mat* X = om_gemm(S, 0, Z, 0, 1.0, tau);        /* S Z */
  om_mat* Y = om_gemm(Z, 1, X, 0, 1.0, tau);        /* Z^T (S Z) */
  om_mat* delta = om_add(-1.0, Y, 0.0, NULL, 1.0);  /* I - Z^T S Z */
  om_free(X); om_free(Y);
  return delta;
}

om_mat* om_irsi(const om_mat* S_in, const om_opts* o, om_report* rep) {
  memset(rep, 0, sizeof(*rep));
  rep_reset_counters();
  om_mat* S = om_truncate(S_in, o->tau);
  double beta = om_gershgorin(S);
  rep->beta = beta;
  double c = (o->c_rule == 1) ? sqrt(2.0 / beta) : 1.0 / sqrt(beta);
  om_mat* Z = om_scaled_identity(S->n, S->bs, S->nb, c);
  double e_prev = INFINITY;
  om_mat* delta = irsi_direct_delta(S, Z, o->tau);
  for (int it = 0;; ++it) {
    double e = om_fro(delta);
    if (rep->n_delta < 64) rep->delta_fro[rep->n_delta++] = e;
    int stop = 0;
    if (o->fixed_iters > 0) {
      if (it == o->fixed_iters) stop = OM_STOP_FIXED;
    } else if (e <= o->target) {
      stop = OM_STOP_TARGET;
    } else if (e > pow(e_prev, (double)(o->m + 1))) {
      stop = OM_STOP_RULE;
    } else if (it == o->max_iter) {
      stop = OM_STOP_MAXITER;
    }
    if (stop) {
      rep->stop_reason = stop;
      rep->sweeps = it;
      om_free(delta);
      break;
    }
    om_mat* P = poly_P(delta, o->m, o->tau);
    om_mat* M = om_gemm(Z, 0, P, 0, 1.0, o->tau);       /* M = Z sum b_k delta^k */
    om_mat* Zn = om_add(1.0, Z, 1.0, M, 0.0);           /* Z + M */
    om_free(P);
    if (o->local_delta) {
      /* Eq. (2.2): delta' = delta - Z_{i+1}^T (S M) - (M^T S) Z_i, M^T S = (S M)^T */
      om_mat* T = om_gemm(S, 0, M, 0, 1.0, o->tau);
      om_mat* U = om_gemm(Zn, 1, T, 0, 1.0, o->tau);
      om_mat* V = om_gemm(T, 1, Z, 0, 1.0, o->tau);
      om_mat* d1 = om_add(1.0, delta, -1.0, U, 0.0);
      om_mat* dn = om_add(1.0, d1, -1.0, V, 0.0);
      om_free(T); om_free(U); om_free(V); om_free(d1); om_free(delta);
      delta = dn;
    }
    om_free(M); om_free(Z);
    Z = Zn;
    if (!o->local_delta) {
      om_free(delta);
      delta = irsi_direct_delta(S, Z, o->tau);
    }
    e_prev = e;
  }
  om_free(S);
  rep->products = g_products;
  rep->block_pairs = g_pairs;
  return Z;
}

/* ------------------------------------------------------------------ */
/* Leaf routine: dense inverse Cholesky                                 */
/* ------------------------------------------------------------------ */

/* S (n x n, row-major, SPD) -> Z = L^-T with S = L L^T.  Z is upper
 * triangular with positive diagonal.  Returns 0, or -2 when a pivot is not
 * positive (S not positive definite). */
int om_invchol_dense(int n, const double* S, double* Z) {
  double* L = (double*)calloc((size_t)n * n, sizeof(double));
  double* W = (double*)calloc((size_t)n * n, sizeof(double));
  for (int j = 0; j < n; ++j) {
    double d = S[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(d > 0.0)) { free(L); free(W); return -2; }
    double ljj = sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double v = S[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = v / ljj;
    }
  }
  /* W = L^-1 by forward substitution, column by column of the identity. */
  for (int c = 0; c < n; ++c) {
    for (int i = c; i < n; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) v -= L[(size_t)i * n + k] * W[(size_t)k * n + c];
      W[(size_t)i * n + c] = v / L[(size_t)i * n + i];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Z[(size_t)i * n + j] = W[(size_t)j * n + i];
  free(L); free(W);
  return 0;
}

/* Leaf routine on the principal sub-matrix [b0, b1) of S: the dense inverse
 * Cholesky factor Z = L^-T, its blocks on and above the diagonal kept, then
 * truncated (Section 5: truncation after leaf-level routines).  Returned in
 * the sub-matrix's own index space; *status = -2 when a pivot fails. */
static om_mat* leaf_factor(const om_mat* S, int b0, int b1, double tau, int* status) {
  int bs = S->bs, nbs = b1 - b0, nl = nbs * bs;
  size_t bsz = (size_t)bs * bs;
  double* dS = (double*)calloc((size_t)nl * nl, sizeof(double));
  double* dZ = (double*)calloc((size_t)nl * nl, sizeof(double));
  for (int I = b0; I < b1; ++I)
    for (int p = S->row_ptr[I]; p < S->row_ptr[I + 1]; ++p) {
      int J = S->col_idx[p];
      if (J < b0 || J >= b1) continue;
      for (int r = 0; r < bs; ++r)
        for (int c = 0; c < bs; ++c)
          dS[(size_t)((I - b0) * bs + r) * nl + (J - b0) * bs + c] = S->val[(size_t)p * bsz + r * bs + c];
    }
  if (om_invchol_dense(nl, dS, dZ) != 0) *status = -2;
  om_builder out = ob_begin((int64_t)nl, bs, nbs);
  double* tmp = (double*)malloc(bsz * sizeof(double));
  for (int I = 0; I < nbs; ++I) {
    for (int J = I; J < nbs; ++J) {
      for (int r = 0; r < bs; ++r)
        for (int c = 0; c < bs; ++c) tmp[r * bs + c] = dZ[(size_t)(I * bs + r) * nl + J * bs + c];
      if (!(block_fro(tmp, bs) < tau)) memcpy(ob_push(&out, J), tmp, bsz * sizeof(double));
    }
    ob_end_row(&out, I);
  }
  free(tmp); free(dS); free(dZ);
  return out.m;
}

/* A (na x na, own index space) placed at block offset off of an nbs-block
 * square matrix, zero elsewhere. */
static om_mat* om_embed(const om_mat* A, int nbs, int off) {
  size_t bsz = (size_t)A->bs * A->bs;
  om_builder b = ob_begin((int64_t)nbs * A->bs, A->bs, nbs);
  for (int I = 0; I < nbs; ++I) {
    int li = I - off;
    if (li >= 0 && li < A->nb)
      for (int p = A->row_ptr[li]; p < A->row_ptr[li + 1]; ++p)
        memcpy(ob_push(&b, A->col_idx[p] + off), A->val + (size_t)p * bsz, bsz * sizeof(double));
    ob_end_row(&b, I);
  }
  return b.m;
}

/* ------------------------------------------------------------------ */
/* LIF: localized inverse factorization (Algorithm 2)                   */
/* ------------------------------------------------------------------ */

typedef struct {
  const om_opts* o;
  int depth_max;
  int status;
} rinch_ctx;
static om_mat* rinch_rec(rinch_ctx* R, const om_mat* S, int b0, int b1, int depth);

typedef struct {
  const om_opts* o;
  om_report* rep;
  int depth_max;
  int status;
} lif_ctx;

/* Localized refinement, Eq. (2.2) in the form of Algorithm 2:
 *   M_i = Z_i sum_{k>=1} b_k delta_i^k,  Z_{i+1} = Z_i + M_i,
 *   delta_{i+1} = delta_i - Z_{i+1}^T (S M_i) - (M_i^T S) Z_i,
 * with (M_i^T S) = (S M_i)^T because S is symmetric.  Stops as Algorithm 4:
 * after computing e = ||delta_{i+1}||_F, stop when e > e_prev^{m+1} (e_prev
 * starts at +inf, so the first check never stops), or e <= target, or the
 * sweep cap is hit; the last iterate Z_{i+1} is returned. */
static om_mat* refine_local(lif_ctx* L, const om_mat* S, om_mat* Z, om_mat* delta, int top) {
  const om_opts* o = L->o;
  double e_prev = INFINITY;
  for (int it = 0;; ++it) {
    om_mat* P = poly_P(delta, o->m, o->tau);
    om_mat* M = om_gemm(Z, 0, P, 0, 1.0, o->tau);
    om_free(P);
    om_mat* Zn = om_add(1.0, Z, 1.0, M, 0.0);
    om_mat* T = om_gemm(S, 0, M, 0, 1.0, o->tau);          /* S M */
    om_mat* U = om_gemm(Zn, 1, T, 0, 1.0, o->tau);         /* Z_{i+1}^T (S M) */
    om_mat* V = om_gemm(T, 1, Z, 0, 1.0, o->tau);          /* (M^T S) Z_i */
    om_mat* d1 = om_add(1.0, delta, -1.0, U, 0.0);
    om_mat* dn = om_add(1.0, d1, -1.0, V, 0.0);
    om_free(M); om_free(T); om_free(U); om_free(V); om_free(d1);
    om_free(Z); om_free(delta);
    Z = Zn;
    delta = dn;
    double e = om_fro(delta);
    L->rep->sweeps++;
    if (top && L->rep->n_delta < 64) L->rep->delta_fro[L->rep->n_delta++] = e;
    int stop = 0;
    if (e <= o->target) stop = OM_STOP_TARGET;
    else if (e > pow(e_prev, (double)(o->m + 1))) stop = OM_STOP_RULE;
    else if (it + 1 >= o->max_iter) stop = OM_STOP_MAXITER;
    if (stop) {
      if (top) L->rep->stop_reason = stop;
      break;
    }
    e_prev = e;
  }
  om_free(delta);
  return Z;
}

/* Inverse factor of the principal sub-matrix on block range [b0, b1). */
static om_mat* lif_rec(lif_ctx* L, const om_mat* S, int b0, int b1, int depth) {
  const om_opts* o = L->o;
  int bs = S->bs, nbs = b1 - b0;
  size_t bsz = (size_t)bs * bs;
  if (depth > L->depth_max) L->depth_max = depth;
  if ((int64_t)nbs * bs <= o->leaf_size || nbs == 1) return leaf_factor(S, b0, b1, o->tau, &L->status);
  if ((int64_t)nbs * bs <= o->rinch_rows) {  /* the switch to RINCH for small sub-problems */
    rinch_ctx R = {o, 0, 0};
    om_mat* Z = rinch_rec(&R, S, b0, b1, 0);
    if (R.status) L->status = R.status;
    return Z;
  }
  int bm = b0 + nbs / 2;
  om_mat* ZA = lif_rec(L, S, b0, bm, depth + 1);
  om_mat* ZC = lif_rec(L, S, bm, b1, depth + 1);
  int na = bm - b0;
  /* Z_0 = diag(Z_A, Z_C) in the sub-problem's index space */
  om_builder zb = ob_begin((int64_t)nbs * bs, bs, nbs);
  for (int I = 0; I < nbs; ++I) {
    const om_mat* src = (I < na) ? ZA : ZC;
    int li = (I < na) ? I : I - na, off = (I < na) ? 0 : na;
    for (int p = src->row_ptr[li]; p < src->row_ptr[li + 1]; ++p)
      memcpy(ob_push(&zb, src->col_idx[p] + off), src->val + (size_t)p * bsz, bsz * sizeof(double));
    ob_end_row(&zb, I);
  }
  om_mat* Z0 = zb.m;
  /* X = -Z_A^T B Z_C, formed in the sub-problem's index space: with
   * Bhat holding B at rows [0, na), cols [na, nbs) and Z_0 = diag(Z_A, Z_C),
   * Bhat Z_0 = [0, B Z_C; 0, 0] and Z_0^T (Bhat Z_0) = [0, Z_A^T B Z_C; 0, 0]. */
  om_mat* Bh = om_sub_embedded(S, b0, b1, b0, bm, bm, b1);
  om_mat* T = om_gemm(Bh, 0, Z0, 0, 1.0, o->tau);        /* B Z_C */
  om_mat* X = om_gemm(Z0, 1, T, 0, -1.0, o->tau);        /* -Z_A^T B Z_C */
  om_mat* Xt = om_transpose(X);
  om_mat* delta0 = om_add(1.0, X, 1.0, Xt, 0.0);         /* [0 X; X^T 0] */
  om_free(Bh); om_free(T); om_free(X); om_free(Xt);
  om_free(ZA); om_free(ZC);
  om_mat* Ssub = om_sub(S, b0, b1, b0, b1);
  om_mat* Z = refine_local(L, Ssub, Z0, delta0, depth == 0);
  om_free(Ssub);
  return Z;
}

om_mat* om_lif(const om_mat* S_in, const om_opts* o, om_report* rep) {
  memset(rep, 0, sizeof(*rep));
  rep_reset_counters();
  om_mat* S = om_truncate(S_in, o->tau);
  lif_ctx L = {o, rep, 0, 0};
  om_mat* Z = lif_rec(&L, S, 0, S->nb, 0);
  Z->n = S_in->n;
  om_free(S);
  rep->levels = L.depth_max;
  rep->status = L.status;
  rep->products = g_products;
  rep->block_pairs = g_pairs;
  return Z;
}

/* ------------------------------------------------------------------ */
/* Direct factorization error                                           */
/* ------------------------------------------------------------------ */

/* ||I - Z^T S Z||_F with untruncated products. */
/* ------------------------------------------------------------------ */
/* RINCH: recursive inverse Cholesky (Algorithm 1)                      */
/* ------------------------------------------------------------------ */

/* Inverse factor of the principal sub-matrix on block range [b0, b1) of S,
 * in the sub-matrix's own index space.  With S = [S00 S01; S01^T S11] split
 * at the block-aligned midpoint (the same split as LIF):
 *   Z00 = rinch(S00),  R = Z00^T S01,  Q = -R^T R + S11,  Z11 = rinch(Q),
 *   Z01 = -(Z00 R) Z11,  Z10 = 0,
 * every product truncated at tau, sums not truncated.  The off-diagonal
 * pieces live embedded in the sub-problem's index space (rows [0, na), cols
 * [na, nbs)), so every product is between square matrices. */
static om_mat* rinch_rec(rinch_ctx* R, const om_mat* S, int b0, int b1, int depth) {
  const om_opts* o = R->o;
  int bs = S->bs, nbs = b1 - b0;
  if (depth > R->depth_max) R->depth_max = depth;
  if ((int64_t)nbs * bs <= o->leaf_size || nbs == 1) return leaf_factor(S, b0, b1, o->tau, &R->status);
  int bm = b0 + nbs / 2, na = bm - b0;
  om_mat* Z00 = rinch_rec(R, S, b0, bm, depth + 1);
  om_mat* Z00e = om_embed(Z00, nbs, 0);
  om_free(Z00);
  om_mat* S01 = om_sub_embedded(S, b0, b1, b0, bm, bm, b1);
  om_mat* Rm = om_gemm(Z00e, 1, S01, 0, 1.0, o->tau);     /* R = Z00^T S01 */
  om_free(S01);
  om_mat* RtR = om_gemm(Rm, 1, Rm, 0, 1.0, o->tau);       /* R^T R */
  om_mat* S11 = om_sub_embedded(S, b0, b1, bm, b1, bm, b1);
  om_mat* Q = om_add(-1.0, RtR, 1.0, S11, 0.0);           /* Q = -R^T R + S11 */
  om_free(RtR); om_free(S11);
  om_mat* Z11 = rinch_rec(R, Q, na, nbs, depth + 1);
  om_free(Q);
  om_mat* Z11e = om_embed(Z11, nbs, na);
  om_free(Z11);
  om_mat* T = om_gemm(Z00e, 0, Rm, 0, 1.0, o->tau);       /* Z00 R */
  om_mat* Z01 = om_gemm(T, 0, Z11e, 0, -1.0, o->tau);     /* Z01 = -(Z00 R) Z11 */
  om_free(T); om_free(Rm);
  om_mat* Zu = om_add(1.0, Z00e, 1.0, Z01, 0.0);
  om_mat* Z = om_add(1.0, Zu, 1.0, Z11e, 0.0);
  om_free(Z00e); om_free(Z01); om_free(Zu); om_free(Z11e);
  return Z;
}

om_mat* om_rinch(const om_mat* S_in, const om_opts* o, om_report* rep) {
  memset(rep, 0, sizeof(*rep));
  rep_reset_counters();
  om_mat* S = om_truncate(S_in, o->tau);
  rinch_ctx R = {o, 0, 0};
  om_mat* Z = rinch_rec(&R, S, 0, S->nb, 0);
  Z->n = S_in->n;
  om_free(S);
  rep->levels = R.depth_max;
  rep->status = R.status;
  rep->products = g_products;
  rep->block_pairs = g_pairs;
  return Z;
}

double om_resid(const om_mat* S, const om_mat* Z) {
  om_mat* X = om_gemm(S, 0, Z, 0, 1.0, 0.0);
  om_mat* Y = om_gemm(Z, 1, X, 0, 1.0, 0.0);
  om_mat* d = om_add(-1.0, Y, 0.0, NULL, 1.0);
  double e = om_fro(d);
  om_free(X); om_free(Y); om_free(d);
  return e;
}

int64_t om_counter_products(void) { return g_products; }
int64_t om_counter_pairs(void) { return g_pairs; }

/* ------------------------------------------------------------------ */
/* Adjoint of the refinement on a frozen block pattern                  */
/* ------------------------------------------------------------------ */
/*
 * The differentiated function: K sweeps of Eq. (2.1) with m = 2 from
 * Z_0 = c I (c held constant), every intermediate restricted to a block
 * pattern that is fixed in advance (the patterns a tau-truncated run
 * produced), and L = tr(Z_K^T F Z_K).  With Pi_X the projection onto the
 * frozen pattern of X, one sweep is
 *   X = Pi_X(S Z), Y = Pi_Y(Z^T X), delta = I - Y, D = Pi_D(delta delta),
 *   P = delta/2 + 3 D/8, M = Pi_M(Z P), Z' = Z + M.
 * Its reverse-mode derivative, applied step by step in reverse order:
 *   Mh = Pi_M(Zh'),  Zh = Pi_Z(Zh') + Pi_Z(Mh P^T),  Ph = Pi_P(Z^T Mh),
 *   Dh = 3/8 Pi_D(Ph),  deltah = 1/2 Pi_delta(Ph) + Pi_delta(Dh delta^T + delta^T Dh),
 *   Yh = -Pi_Y(deltah),  Zh += Pi_Z(X Yh^T),  Xh = Pi_X(Z Yh),
 *   Zh += Pi_Z(S^T Xh),  Sh += Pi_S(Xh Z^T),
 * starting from Zh_K = Pi_{Z_K}((F + F^T) Z_K).
 */

/* C = alpha op(A) op(B) restricted to the pattern of P (blocks of P absent
 * from the product are zero blocks). */
static om_mat* om_gemm_masked(const om_mat* A, int tA, const om_mat* B, int tB, double alpha, const om_mat* P) {
  om_mat* full = om_gemm(A, tA, B, tB, alpha, 0.0);
  size_t bsz = (size_t)A->bs * A->bs;
  om_builder out = ob_begin(A->n, A->bs, A->nb);
  for (int I = 0; I < P->nb; ++I) {
    int q = full->row_ptr[I];
    for (int p = P->row_ptr[I]; p < P->row_ptr[I + 1]; ++p) {
      int J = P->col_idx[p];
      while (q < full->row_ptr[I + 1] && full->col_idx[q] < J) ++q;
      double* dst = ob_push(&out, J);
      if (q < full->row_ptr[I + 1] && full->col_idx[q] == J) memcpy(dst, full->val + (size_t)q * bsz, bsz * sizeof(double));
      else memset(dst, 0, bsz * sizeof(double));
    }
    ob_end_row(&out, I);
  }
  om_free(full);
  return out.m;
}

/* Pi_P(A): A restricted to the pattern of P. */
static om_mat* om_project(const om_mat* A, const om_mat* P) {
  size_t bsz = (size_t)A->bs * A->bs;
  om_builder out = ob_begin(A->n, A->bs, A->nb);
  for (int I = 0; I < P->nb; ++I) {
    int q = A->row_ptr[I];
    for (int p = P->row_ptr[I]; p < P->row_ptr[I + 1]; ++p) {
      int J = P->col_idx[p];
      while (q < A->row_ptr[I + 1] && A->col_idx[q] < J) ++q;
      double* dst = ob_push(&out, J);
      if (q < A->row_ptr[I + 1] && A->col_idx[q] == J) memcpy(dst, A->val + (size_t)q * bsz, bsz * sizeof(double));
      else memset(dst, 0, bsz * sizeof(double));
    }
    ob_end_row(&out, I);
  }
  return out.m;
}

/* sum over stored blocks of <A_blk, B_blk> on A's pattern (B looked up) */
static double om_dot_on(const om_mat* A, const om_mat* B) {
  om_mat* Bp = om_project(B, A);
  double s = 0.0;
  size_t tot = (size_t)A->nnzb * A->bs * A->bs;
  for (size_t e = 0; e < tot; ++e) s += A->val[e] * Bp->val[e];
  om_free(Bp);
  return s;
}

typedef struct {
  int K;
  om_mat** X;  /* frozen patterns (and values of the recording run) per sweep */
  om_mat** Y;
  om_mat** D;
  om_mat** M;
  om_mat** Z;  /* Z_0 .. Z_K */
  om_mat* S;   /* truncated S */
} om_tape;

void om_tape_free(om_tape* t) {
  if (!t) return;
  for (int k = 0; k < t->K; ++k) {
    om_free(t->X[k]); om_free(t->Y[k]); om_free(t->D[k]); om_free(t->M[k]);
  }
  for (int k = 0; k <= t->K; ++k) om_free(t->Z[k]);
  free(t->X); free(t->Y); free(t->D); free(t->M); free(t->Z);
  om_free(t->S);
  free(t);
}

/* Recording run: K truncated sweeps (m = 2) from Z_0 = c I; keeps every
 * intermediate (its pattern is the frozen pattern). */
om_tape* om_tape_record(const om_mat* S_in, double c, int K, double tau) {
  om_tape* t = (om_tape*)calloc(1, sizeof(om_tape));
  t->K = K;
  t->X = (om_mat**)calloc((size_t)K, sizeof(om_mat*));
  t->Y = (om_mat**)calloc((size_t)K, sizeof(om_mat*));
  t->D = (om_mat**)calloc((size_t)K, sizeof(om_mat*));
  t->M = (om_mat**)calloc((size_t)K, sizeof(om_mat*));
  t->Z = (om_mat**)calloc((size_t)K + 1, sizeof(om_mat*));
  t->S = om_truncate(S_in, tau);
  t->Z[0] = om_scaled_identity(t->S->n, t->S->bs, t->S->nb, c);
  for (int k = 0; k < K; ++k) {
    om_mat* Z = t->Z[k];
    t->X[k] = om_gemm(t->S, 0, Z, 0, 1.0, tau);
    t->Y[k] = om_gemm(Z, 1, t->X[k], 0, 1.0, tau);
    om_mat* delta = om_add(-1.0, t->Y[k], 0.0, NULL, 1.0);
    t->D[k] = om_gemm(delta, 0, delta, 0, 1.0, tau);
    om_mat* P = om_add(0.5, delta, 0.375, t->D[k], 0.0);
    t->M[k] = om_gemm(Z, 0, P, 0, 1.0, tau);
    t->Z[k + 1] = om_add(1.0, Z, 1.0, t->M[k], 0.0);
    om_free(delta); om_free(P);
  }
  return t;
}

/* Frozen-pattern forward for a (possibly perturbed) S on the tape's patterns;
 * returns L = tr(Z_K^T F Z_K).  S_val must have the tape's S pattern. */
double om_frozen_loss(const om_tape* t, const om_mat* S, const om_mat* F, double c) {
  om_mat* Z = om_scaled_identity(S->n, S->bs, S->nb, c);
  for (int k = 0; k < t->K; ++k) {
    om_mat* X = om_gemm_masked(S, 0, Z, 0, 1.0, t->X[k]);
    om_mat* Y = om_gemm_masked(Z, 1, X, 0, 1.0, t->Y[k]);
    om_mat* delta = om_add(-1.0, Y, 0.0, NULL, 1.0);
    om_mat* D = om_gemm_masked(delta, 0, delta, 0, 1.0, t->D[k]);
    om_mat* P = om_add(0.5, delta, 0.375, D, 0.0);
    om_mat* M = om_gemm_masked(Z, 0, P, 0, 1.0, t->M[k]);
    om_mat* Zn = om_add(1.0, Z, 1.0, M, 0.0);
    om_free(X); om_free(Y); om_free(delta); om_free(D); om_free(P); om_free(M); om_free(Z);
    Z = Zn;
  }
  om_mat* FZ = om_gemm(F, 0, Z, 0, 1.0, 0.0);
  double L = om_dot_on(Z, FZ);
  om_free(FZ); om_free(Z);
  return L;
}

/* Reverse pass: returns Sh = dL/dS on the pattern of the tape's S. */
om_mat* om_adjoint(const om_tape* t, const om_mat* F) {
  const int K = t->K;
  const om_mat* S = t->S;
  om_mat* ZK = t->Z[K];
  om_mat* FZ = om_gemm(F, 0, ZK, 0, 1.0, 0.0);
  om_mat* FtZ = om_gemm(F, 1, ZK, 0, 1.0, 0.0);
  om_mat* G = om_add(1.0, FZ, 1.0, FtZ, 0.0);
  om_mat* Zh = om_project(G, ZK);
  om_free(FZ); om_free(FtZ); om_free(G);
  om_mat* Sh = om_project(S, S);
  memset(Sh->val, 0, (size_t)Sh->nnzb * S->bs * S->bs * sizeof(double));
  for (int k = K - 1; k >= 0; --k) {
    const om_mat* Z = t->Z[k];
    const om_mat* X = t->X[k];
    om_mat* delta = om_add(-1.0, t->Y[k], 0.0, NULL, 1.0);
    om_mat* P = om_add(0.5, delta, 0.375, t->D[k], 0.0);
    om_mat* Mh = om_project(Zh, t->M[k]);
    om_mat* Zn = om_project(Zh, Z);
    om_mat* t1 = om_gemm_masked(Mh, 0, P, 1, 1.0, Z);               /* Pi_Z(Mh P^T) */
    om_mat* Zacc = om_add(1.0, Zn, 1.0, t1, 0.0);
    om_free(Zn); om_free(t1);
    om_mat* Ph = om_gemm_masked(Z, 1, Mh, 0, 1.0, P);                /* Pi_P(Z^T Mh) */
    om_mat* Dh = om_project(Ph, t->D[k]);
    om_mat* Dh38 = om_add(0.375, Dh, 0.0, NULL, 0.0);
    om_mat* a1 = om_gemm_masked(Dh38, 0, delta, 1, 1.0, delta);      /* Pi_delta(Dh delta^T) */
    om_mat* a2 = om_gemm_masked(delta, 1, Dh38, 0, 1.0, delta);      /* Pi_delta(delta^T Dh) */
    om_mat* Phd = om_project(Ph, delta);
    om_mat* s1 = om_add(0.5, Phd, 1.0, a1, 0.0);
    om_mat* deltah = om_add(1.0, s1, 1.0, a2, 0.0);
    om_mat* Yh0 = om_project(deltah, t->Y[k]);
    om_mat* Yh = om_add(-1.0, Yh0, 0.0, NULL, 0.0);
    om_mat* t2 = om_gemm_masked(X, 0, Yh, 1, 1.0, Z);                /* Pi_Z(X Yh^T) */
    om_mat* Zacc2 = om_add(1.0, Zacc, 1.0, t2, 0.0);
    om_mat* Xh = om_gemm_masked(Z, 0, Yh, 0, 1.0, X);                /* Pi_X(Z Yh) */
    om_mat* t3 = om_gemm_masked(S, 1, Xh, 0, 1.0, Z);                /* Pi_Z(S^T Xh) */
    om_mat* Zacc3 = om_add(1.0, Zacc2, 1.0, t3, 0.0);
    om_mat* t4 = om_gemm_masked(Xh, 0, Z, 1, 1.0, S);                /* Pi_S(Xh Z^T) */
    om_mat* Shn = om_add(1.0, Sh, 1.0, t4, 0.0);
    om_free(Sh); Sh = Shn;
    om_free(delta); om_free(P); om_free(Mh); om_free(Zacc); om_free(Ph); om_free(Dh); om_free(Dh38);
    om_free(a1); om_free(a2); om_free(Phd); om_free(s1); om_free(deltah); om_free(Yh0); om_free(Yh);
    om_free(t2); om_free(Zacc2); om_free(Xh); om_free(t3); om_free(t4);
    om_free(Zh);
    Zh = Zacc3;
  }
  om_free(Zh);
  return Sh;
}

double om_tape_loss(const om_tape* t, const om_mat* F) {
  om_mat* FZ = om_gemm(F, 0, t->Z[t->K], 0, 1.0, 0.0);
  double L = om_dot_on(t->Z[t->K], FZ);
  om_free(FZ);
  return L;
}

const om_mat* om_tape_S(const om_tape* t) { return t->S; }
const om_mat* om_tape_Z(const om_tape* t, int k) { return t->Z[k]; }
