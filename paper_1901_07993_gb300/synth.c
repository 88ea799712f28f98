/*
 * synth.c -- seeded synthetic inputs for the inverse-factorization path.
 *
 * This file generates INPUTS only: point geometries (a jittered 1D chain and
 * a random-sequential-addition cluster in a cube), a recursive coordinate
 * bisection (RCB) ordering of the points, and the overlap matrix S of
 * normalized s-type Gaussians on those points, stored block-sparse.  It holds
 * none of the factorization method's arithmetic (no products, no refinement,
 * no truncation at the method's threshold tau); both the CPU oracle and the
 * CUDA path receive the matrices this file writes.
 *
 * The paper factorizes STO-3G overlap matrices of Glu-Ala helices and water
 * clusters produced by the Ergo program (Section 5); those matrices are not
 * available, so these synthetic Gaussian-overlap matrices stand in for them:
 * the chain mimics the quasi-linear helices, the 3D cluster the water clusters.
 *
 * Overlap of two normalized s-type Gaussians with exponents a, b at distance r:
 *     S = (2 sqrt(a b) / (a + b))^(3/2) * exp(-a b / (a + b) * r^2)
 * so S_ii = 1 exactly and S is symmetric positive definite.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): the state starts at the
 * seed and draw k (k >= 1) is mix64(seed + k * 0x9E3779B97F4A7C15), so it is
 * counter-based.  Doubles take the top 53 bits.  Integer arithmetic only, so the draws are the same on
 * every machine.  Build with -ffp-contract=off so that geometry decisions do
 * not change with FMA contraction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct { uint64_t state; } rng_t;

static rng_t rng_make(uint64_t seed) {
  rng_t r;
  r.state = seed; /* plain SplitMix64 seeding */
  return r;
}
static uint64_t rng_next(rng_t* r) {
  r->state += GOLDEN;
  return mix64(r->state);
}
static double rng_uniform(rng_t* r) { /* [0, 1) */
  return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0);
}

/* Exported for tests: the k-th raw draw of stream `seed` (k >= 1). */
uint64_t synth_rng_draw(uint64_t seed, int64_t k) {
  rng_t r = rng_make(seed);
  uint64_t v = 0;
  for (int64_t i = 0; i < k; ++i) v = rng_next(&r);
  return v;
}

/* ------------------------------------------------------------------ */
/* Geometries                                                           */
/* ------------------------------------------------------------------ */

/* 1D chain: x_i = spacing * i + U(-jitter, jitter), y = z = 0. */
void synth_chain(int64_t n, double spacing, double jitter, uint64_t seed, double* xyz) {
  rng_t r = rng_make(seed);
  for (int64_t i = 0; i < n; ++i) {
    double u = rng_uniform(&r);
    xyz[3 * i + 0] = spacing * (double)i + (2.0 * u - 1.0) * jitter;
    xyz[3 * i + 1] = 0.0;
    xyz[3 * i + 2] = 0.0;
  }
}

/*
 * Random sequential addition in the open cube [0, L)^3 with L = (n/density)^(1/3):
 * candidate points are drawn uniformly and accepted when no accepted point is
 * closer than dmin.  A cell grid with cells of side >= dmin limits the search
 * to the 27 neighbouring cells.  Returns the number of points placed (n on
 * success; fewer if max_attempts ran out).
 */
int64_t synth_rsa_cube(int64_t n, double density, double dmin, uint64_t seed,
                       int64_t max_attempts, double* xyz) {
  const double L = cbrt((double)n / density);
  int g = (int)floor(L / dmin);
  if (g < 1) g = 1;
  const double cell = L / (double)g;
  const int64_t ncell = (int64_t)g * g * g;
  const int cap = 16; /* a cell of side >= dmin holds at most 8 points */
  int32_t* cnt = (int32_t*)calloc((size_t)ncell, sizeof(int32_t));
  int32_t* idx = (int32_t*)malloc((size_t)ncell * cap * sizeof(int32_t));
  if (!cnt || !idx) { free(cnt); free(idx); return -1; }
  rng_t r = rng_make(seed);
  const double d2 = dmin * dmin;
  int64_t placed = 0, attempts = 0;
  while (placed < n && attempts < max_attempts) {
    ++attempts;
    double p[3];
    for (int c = 0; c < 3; ++c) p[c] = rng_uniform(&r) * L;
    int ci[3];
    for (int c = 0; c < 3; ++c) {
      ci[c] = (int)(p[c] / cell);
      if (ci[c] >= g) ci[c] = g - 1;
    }
    int ok = 1;
    for (int dx = -1; dx <= 1 && ok; ++dx)
      for (int dy = -1; dy <= 1 && ok; ++dy)
        for (int dz = -1; dz <= 1 && ok; ++dz) {
          int x = ci[0] + dx, y = ci[1] + dy, z = ci[2] + dz;
          if (x < 0 || y < 0 || z < 0 || x >= g || y >= g || z >= g) continue;
          int64_t cid = ((int64_t)x * g + y) * g + z;
          for (int k = 0; k < cnt[cid]; ++k) {
            const double* q = xyz + 3 * (int64_t)idx[cid * cap + k];
            double ex = p[0] - q[0], ey = p[1] - q[1], ez = p[2] - q[2];
            if (ex * ex + ey * ey + ez * ez < d2) { ok = 0; break; }
          }
        }
    if (!ok) continue;
    int64_t cid = ((int64_t)ci[0] * g + ci[1]) * g + ci[2];
    if (cnt[cid] >= cap) continue; /* cannot happen for cell >= dmin */
    idx[cid * cap + cnt[cid]++] = (int32_t)placed;
    for (int c = 0; c < 3; ++c) xyz[3 * placed + c] = p[c];
    ++placed;
  }
  free(cnt);
  free(idx);
  return placed;
}

/* ------------------------------------------------------------------ */
/* Recursive coordinate bisection ordering                              */
/* ------------------------------------------------------------------ */

static const double* g_sort_xyz;
static int g_sort_axis;
static int cmp_axis(const void* pa, const void* pb) {
  int64_t a = *(const int64_t*)pa, b = *(const int64_t*)pb;
  double va = g_sort_xyz[3 * a + g_sort_axis], vb = g_sort_xyz[3 * b + g_sort_axis];
  if (va < vb) return -1;
  if (va > vb) return 1;
  return (a < b) ? -1 : (a > b);
}

/* perm[p0..p1) holds point ids; nblk blocks of bs points cover them. */
static void rcb_rec(const double* xyz, int64_t* perm, int64_t p0, int64_t p1, int64_t nblk, int bs) {
  if (nblk <= 1 || p1 - p0 <= 1) return;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = p0; i < p1; ++i)
    for (int c = 0; c < 3; ++c) {
      double v = xyz[3 * perm[i] + c];
      if (v < lo[c]) lo[c] = v;
      if (v > hi[c]) hi[c] = v;
    }
  int axis = 0;
  for (int c = 1; c < 3; ++c)
    if (hi[c] - lo[c] > hi[axis] - lo[axis]) axis = c;
  g_sort_xyz = xyz;
  g_sort_axis = axis;
  qsort(perm + p0, (size_t)(p1 - p0), sizeof(int64_t), cmp_axis);
  int64_t lblk = nblk / 2;
  int64_t lcount = lblk * bs;
  if (lcount > p1 - p0) lcount = p1 - p0;
  rcb_rec(xyz, perm, p0, p0 + lcount, lblk, bs);
  rcb_rec(xyz, perm, p0 + lcount, p1, nblk - lblk, bs);
}

/* perm[k] = generation index of the point placed k-th in RCB order.  The
 * block-aligned halving of the index range then follows the geometric cuts. */
void synth_rcb_order(int64_t n, const double* xyz, int bs, int64_t* perm) {
  for (int64_t i = 0; i < n; ++i) perm[i] = i;
  int64_t nblk = (n + bs - 1) / bs;
  rcb_rec(xyz, perm, 0, n, nblk, bs);
}

/* ------------------------------------------------------------------ */
/* Gaussian overlap matrix in block-sparse row (BSR) storage           */
/* ------------------------------------------------------------------ */

typedef struct {
  int64_t nb, nnzb;
  int32_t* row_ptr;
  int32_t* col_idx;
  double* val;
} synth_bsr;

static double overlap(const double* p, double a, const double* q, double b) {
  double ex = p[0] - q[0], ey = p[1] - q[1], ez = p[2] - q[2];
  double r2 = ex * ex + ey * ey + ez * ez;
  double s = a + b;
  double pre = 2.0 * sqrt(a * b) / s;
  return pre * sqrt(pre) * exp(-(a * b / s) * r2);
}

/*
 * Build S for points xyz[n] (already in the wanted order) with exponents
 * alpha[n], as an nb x nb block matrix of bs x bs blocks (nb = ceil(n/bs)).
 * Rows/columns beyond n (padding of the last block) carry a unit diagonal.
 * A block is stored when its Frobenius norm is >= drop (a generation cutoff
 * far below any truncation threshold the method uses; exact-zero blocks are
 * never stored).  Blocks whose bounding boxes are so far apart that
 * bs * exp(-pmin * dist^2) < drop are skipped without evaluation, where
 * pmin = min_i alpha_i / 2 bounds a b / (a + b) from below and the prefactor
 * is <= 1.  Returns a handle (NULL on allocation failure).
 */
void* synth_overlap_bsr(int64_t n, const double* xyz, const double* alpha, int bs, double drop) {
  int64_t nb = (n + bs - 1) / bs;
  double* bmin = (double*)malloc((size_t)nb * 3 * sizeof(double));
  double* bmax = (double*)malloc((size_t)nb * 3 * sizeof(double));
  synth_bsr* out = (synth_bsr*)calloc(1, sizeof(synth_bsr));
  if (!bmin || !bmax || !out) { free(bmin); free(bmax); free(out); return NULL; }
  double amin = INFINITY;
  for (int64_t i = 0; i < n; ++i) if (alpha[i] < amin) amin = alpha[i];
  const double pmin = 0.5 * amin;
  for (int64_t I = 0; I < nb; ++I) {
    for (int c = 0; c < 3; ++c) { bmin[3 * I + c] = INFINITY; bmax[3 * I + c] = -INFINITY; }
    for (int64_t i = I * bs; i < (I + 1) * bs && i < n; ++i)
      for (int c = 0; c < 3; ++c) {
        double v = xyz[3 * i + c];
        if (v < bmin[3 * I + c]) bmin[3 * I + c] = v;
        if (v > bmax[3 * I + c]) bmax[3 * I + c] = v;
      }
  }
  const size_t bsz = (size_t)bs * bs;
  int64_t cap = nb * 8 + 16;
  out->nb = nb;
  out->row_ptr = (int32_t*)malloc((size_t)(nb + 1) * sizeof(int32_t));
  out->col_idx = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
  out->val = (double*)malloc((size_t)cap * bsz * sizeof(double));
  double* tile = (double*)malloc(bsz * sizeof(double));
  if (!out->row_ptr || !out->col_idx || !out->val || !tile) goto fail;
  out->row_ptr[0] = 0;
  for (int64_t I = 0; I < nb; ++I) {
    for (int64_t J = 0; J < nb; ++J) {
      int emptyI = (I * bs >= n), emptyJ = (J * bs >= n);
      if (I != J && (emptyI || emptyJ)) continue;
      if (!emptyI && !emptyJ && I != J) {
        double d2 = 0.0;
        for (int c = 0; c < 3; ++c) {
          double gap = 0.0;
          if (bmax[3 * I + c] < bmin[3 * J + c]) gap = bmin[3 * J + c] - bmax[3 * I + c];
          else if (bmax[3 * J + c] < bmin[3 * I + c]) gap = bmin[3 * I + c] - bmax[3 * J + c];
          d2 += gap * gap;
        }
        if ((double)bs * exp(-pmin * d2) < drop) continue;
      }
      double fro2 = 0.0;
      for (int r = 0; r < bs; ++r)
        for (int c = 0; c < bs; ++c) {
          int64_t i = I * bs + r, j = J * bs + c;
          double v;
          if (i >= n || j >= n) v = (i == j) ? 1.0 : 0.0;
          else if (i == j) v = 1.0;
          else v = overlap(xyz + 3 * i, alpha[i], xyz + 3 * j, alpha[j]);
          tile[(size_t)r * bs + c] = v;
          fro2 += v * v;
        }
      if (fro2 == 0.0 || sqrt(fro2) < drop) continue;
      if (out->nnzb == cap) {
        cap *= 2;
        int32_t* ci = (int32_t*)realloc(out->col_idx, (size_t)cap * sizeof(int32_t));
        if (!ci) goto fail;
        out->col_idx = ci;
        double* v = (double*)realloc(out->val, (size_t)cap * bsz * sizeof(double));
        if (!v) goto fail;
        out->val = v;
      }
      out->col_idx[out->nnzb] = (int32_t)J;
      memcpy(out->val + (size_t)out->nnzb * bsz, tile, bsz * sizeof(double));
      out->nnzb++;
    }
    out->row_ptr[I + 1] = (int32_t)out->nnzb;
  }
  free(tile); free(bmin); free(bmax);
  return out;
fail:
  free(tile); free(bmin); free(bmax);
  free(out->row_ptr); free(out->col_idx); free(out->val); free(out);
  return NULL;
}

int64_t synth_bsr_nnzb(void* h) { return ((synth_bsr*)h)->nnzb; }

/* Copy the matrix out and release the handle. */
void synth_bsr_take(void* h, int bs, int32_t* row_ptr, int32_t* col_idx, double* val) {
  synth_bsr* s = (synth_bsr*)h;
  memcpy(row_ptr, s->row_ptr, (size_t)(s->nb + 1) * sizeof(int32_t));
  memcpy(col_idx, s->col_idx, (size_t)s->nnzb * sizeof(int32_t));
  memcpy(val, s->val, (size_t)s->nnzb * bs * bs * sizeof(double));
  free(s->row_ptr); free(s->col_idx); free(s->val); free(s);
}

void synth_bsr_release(void* h) {
  synth_bsr* s = (synth_bsr*)h;
  if (!s) return;
  free(s->row_ptr); free(s->col_idx); free(s->val); free(s);
}
