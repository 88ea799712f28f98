/*
 * ifac.h -- C ABI of the GB300 (sm_103a) inverse-factorization library.
 *
 * Computes Z with Z^T S Z = I (so S^-1 = Z Z^T) for a block-sparse symmetric
 * positive definite S, following Artemov, Rudberg, Rubensson, "Parallelization
 * and scalability analysis of inverse factorization using the Chunks and
 * Tasks programming model" (arXiv:1901.07993): iterative refinement from a
 * scaled identity (Section 2.2, Eq. 2.1) and localized inverse factorization
 * (Section 2.3, Algorithm 2), both driven by block-sparse products with
 * norm-based block truncation (Section 5).
 *
 * Conventions shared by every entry point:
 *  - Matrices are square, n x n, stored as ifac_bsr: nb = ceil(n/bs) block
 *    rows and columns of bs x bs blocks, CSR order of blocks, columns strictly
 *    increasing within a block row, each block row-major, FP64.  Rows and
 *    columns past n (padding of the last block) must hold a unit diagonal; the
 *    library treats the padded matrix as the one to factor, and the padding
 *    part of Z is the identity.
 *  - Every pointer inside an ifac_bsr is DEVICE memory of the context's
 *    device.  Inputs are borrowed: they must stay valid and unmodified until
 *    the call returns.  Outputs (ifac_bsr* out parameters) are allocated by the
 *    library through the context's allocator; the caller owns them and
 *    releases them with ifac_bsr_free.
 *  - All work is issued on the context's stream.  Calls that produce a
 *    matrix synchronise that stream (output sizes are data dependent); scalar
 *    results are valid on return.
 *  - Return codes: 0 = success; > 0 = success with a warning (results valid);
 *    < 0 = error, outputs left empty (all pointers NULL).  No C++ exception
 *    crosses this boundary.  ifac_last_error() gives a message for the last
 *    non-zero code on that context.
 *  - A context must not be used from two host threads at once.
 */
#ifndef IFAC_H
#define IFAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- */
/* Status codes                                                      */
/* ---------------------------------------------------------------- */
#define IFAC_OK 0
#define IFAC_WARN_TARGET_NOT_MET 1  /* stopped by the automatic rule above the target */
#define IFAC_ERR_INVALID (-1)       /* malformed BSR or argument */
#define IFAC_ERR_NOT_SPD (-2)       /* a leaf pivot was not positive */
#define IFAC_ERR_NO_CONVERGENCE (-3)/* max_iter reached */
#define IFAC_ERR_OOM (-4)           /* allocator returned NULL */
#define IFAC_ERR_CUDA (-5)          /* a CUDA call failed */
#define IFAC_ERR_TIMEOUT (-6)       /* a bounded device-side wait expired */
#define IFAC_ERR_UNSUPPORTED (-7)   /* block size / precision not built */
#define IFAC_ERR_TOO_LARGE (-8)     /* request exceeds a fixed scratch area */

/* Product precision (the arithmetic of the block products). */
#define IFAC_FP64 0 /* FP64 inputs, FP64 accumulation (FP64 pipe) */
#define IFAC_TF32 1 /* inputs rounded to TF32, FP32 accumulation (tensor cores, bs 32/64/128) */
#define IFAC_BF16 2 /* inputs rounded to BF16, FP32 accumulation (tensor cores, bs 32/64/128) */
#define IFAC_FP64_SPLIT 3 /* FP64-accurate: error-free splitting into BF16 slices on the
                             tensor cores (Ozaki et al. 2012), FP64 accumulation, bs 32/64/128 */

/* Stop reasons reported by the refinement drivers. */
#define IFAC_STOP_RULE 1     /* ||delta_{i+1}||_F > ||delta_i||_F^(m+1) (Section 2.2) */
#define IFAC_STOP_TARGET 2   /* ||delta||_F <= target */
#define IFAC_STOP_MAXITER 3  /* max_iter sweeps done */
#define IFAC_STOP_FIXED 4    /* fixed_iters corrections done */

typedef struct {
  int64_t n;        /* logical dimension */
  int32_t bs;       /* block size */
  int32_t nb;       /* block rows = block columns = ceil(n / bs) */
  int64_t nnzb;     /* number of stored blocks */
  int32_t* row_ptr; /* device [nb + 1], row_ptr[0] = 0, row_ptr[nb] = nnzb */
  int32_t* col_idx; /* device [nnzb] */
  double* val;      /* device [nnzb * bs * bs] */
  double* norms;    /* device [nnzb] block Frobenius norms, or NULL (inputs);
                       always filled on library outputs */
} ifac_bsr;

/* Device memory provider.  alloc returns NULL on failure; both are called
 * with the context's stream.  Pass NULL to ifac_create to use the device's
 * stream-ordered pool (cudaMallocAsync / cudaFreeAsync). */
typedef struct {
  void* (*alloc)(void* user, size_t bytes, void* stream);
  void (*free)(void* user, void* ptr, void* stream);
  void* user;
} ifac_allocator;

typedef struct ifac_ctx ifac_ctx;

/* Result of ifac_autotune_batched. */
typedef struct {
  int32_t bs;                /* chosen block size: 32, 64 or 128 */
  int32_t narrow_kmax;       /* chosen tile schedule of bs-64 TF32/BF16 products */
  int32_t narrow_kmax_split; /* and of bs-64 split products (ifac_set_schedule) */
  int32_t low_sweeps_est;    /* sweeps and FP64-accurate delta evaluations */
  int32_t split_evals_est;   /* the prediction assumes */
  double probe_ms[3];        /* predicted product time of a batch refinement at bs 32,
                                64, 128 (best schedules), from the timed probes */
  double probe64_lp_ms[3];   /* at bs 64, the low-precision and the split share of */
  double probe64_split_ms[3];/* it per schedule: default, super-tiles only, narrow only */
} ifac_tune_result;

/* Options of the factorization drivers.  ifac_opts_default fills:
 * m = 2, max_iter = 50, fixed_iters = 0, c_rule = 0, leaf_size = 512,
 * prec = IFAC_FP64, profile = 0, delta_prec = IFAC_FP64_SPLIT, rinch_rows = 0,
 * local_delta = 0. */
typedef struct {
  int m;           /* refinement order: Z_{i+1} = Z_i sum_{k=0}^{m} b_k delta_i^k,
                      b_0 = 1, b_k = (2k-1)/(2k) b_{k-1} (Eq. 2.1); 1..8 */
  int max_iter;    /* cap on sweeps of one refinement */
  int fixed_iters; /* inv_factor_refine only: > 0 runs exactly this many
                      corrections and ignores the stop rule and target */
  int c_rule;      /* inv_factor_refine start Z_0 = c I with beta the
                      Gershgorin bound of S (Section 2.2):
                      0 -> c = 1/sqrt(beta), 1 -> c = sqrt(2/beta) */
  int leaf_size;   /* inv_factor_localized: sub-problems with more rows are
                      split at the block-aligned midpoint (Algorithm 2) */
  int prec;        /* IFAC_FP64; or IFAC_FP64_SPLIT (bs 32, 64 or 128): the FP64
                      schedule with every block product on the split
                      tensor-core kernel; inv_factor_refine and the batched
                      call also take IFAC_TF32 or IFAC_BF16: the
                      mixed-precision schedule below */
  int profile;     /* != 0: time every numeric block-product launch with CUDA
                      events on the context's stream (fills gemm_ms) */
  int delta_prec;  /* products of the FP64-accurate delta evaluations that
                      follow low-precision sweeps (inv_factor_refine with
                      prec TF32/BF16: the FP64 phase; batched: the final
                      residual): IFAC_FP64 (FP64 pipe) or IFAC_FP64_SPLIT
                      (tensor cores; used when bs is 32, 64 or 128,
                      else IFAC_FP64) */
  int rinch_rows;  /* inv_factor_localized: sub-problems with at most this
                      many rows (when above leaf_size) are factorized by
                      recursive inverse Cholesky (Algorithm 1, leaf_size
                      leaves) instead of being split further -- the paper
                      switches to RINCH below 16384 rows; 0 = off */
  int local_delta; /* inv_factor_refine (FP64): 0 evaluates delta = I - Z^T S Z
                      directly every sweep; 1 evaluates delta_0 directly and
                      then updates it locally by Eq. (2.2),
                      delta' = delta - Z'^T (S M) - (S M)^T Z, as the paper's
                      runs do for all methods */
} ifac_opts;

typedef struct {
  int sweeps;          /* corrections applied (localized: summed over sub-problems) */
  int stop_reason;     /* IFAC_STOP_* of the (top-level) refinement */
  int levels;          /* localized: depth of the bisection tree */
  int n_delta;         /* entries used in delta_fro */
  double beta;         /* refine: Gershgorin bound of the truncated S */
  double delta_fro[64];/* refine: ||delta_i||_F per evaluation;
                          localized: top level, per sweep */
  int64_t products;    /* block-sparse products performed */
  int64_t block_pairs; /* stored-block pairs multiplied, over all products */
  int64_t nnzb_Z;      /* stored blocks of the returned Z */
  double flops;        /* 2 bs^3 block_pairs */
  int fp64_delta_evals;/* refine, mixed precision: delta evaluations with FP64 products */
  int low_sweeps;      /* refine, mixed precision: corrections made in the low-precision phase */
  int64_t launches;    /* kernels this call launched */
  int64_t gemm_launches; /* FP64 numeric block-product launches */
  double gemm_ms;      /* their summed device time (opts.profile != 0) */
  int64_t fp64_pairs;  /* block pairs multiplied by them */
  int64_t tc_launches; /* tensor-core (TF32/BF16) block-product launches */
  double tc_ms;        /* their summed device time (opts.profile != 0) */
  int64_t tc_pairs;    /* stored block pairs multiplied by them */
  double resid_fro;    /* batched: ||I - Z^T S Z||_F with FP64 products (else 0) */
  int64_t split_launches; /* FP64-accurate split tensor-core block-product launches */
  double split_ms;     /* their summed device time (opts.profile != 0) */
  int64_t split_pairs; /* stored block pairs multiplied by them */
  int64_t split_slice_pairs; /* sum over those block pairs of the BF16 slice
                                pairs each took: s (s + 1) / 2 with s slices
                                per operand (the mixed schedule lowers s for
                                early delta evaluations) */
  double fp64_bytes;   /* algorithmic bytes of the FP64 product launches: per
                          product (nnzb(A) + nnzb(B) + nnzb(C)) bs^2 8, C before
                          truncation (each block read or written once) */
  double tc_bytes;     /* the same for the TF32/BF16 launches: operands at 4 / 2
                          bytes (the converted copies), C at 8 (FP64), or at 4
                          where a mixed refinement keeps it in FP32
                          (ifac_set_fp32_intermediates) */
  double split_bytes;  /* the same for the split launches: s BF16 slices of
                          each operand (2 s bytes), C as 64-bit sums (8) */
} ifac_report;

/* ---------------------------------------------------------------- */
/* Context                                                           */
/* ---------------------------------------------------------------- */

/* Create a context on the current CUDA device.  stream: a cudaStream_t (NULL
 * = legacy default stream).  alloc: NULL for the built-in pool, else copied.
 * With the built-in pool the context keeps device blocks of up to 4 GB that
 * it frees (24 GB in all at most) and hands them out again in the order of
 * its stream; ifac_destroy returns them, and a failed allocation returns
 * them before it is retried.  ifac_set_stream waits for the old stream. */
int ifac_create(ifac_ctx** ctx, void* stream, const ifac_allocator* alloc);
void ifac_destroy(ifac_ctx* ctx);
int ifac_set_stream(ifac_ctx* ctx, void* stream);
/* Slices per operand of the context's IFAC_FP64_SPLIT products, 3..8
 * (default 7): s slices keep about 7 s bits of every scaled row and column,
 * the product uses the s (s + 1) / 2 slice pairs with s_a + s_b <= s + 1,
 * and the element error is about 2^-(7 s - 3) K max|op(A)_i.| max|op(B)_.j|.
 * IFAC_ERR_INVALID outside 3..8.  The mixed-precision refinement takes this
 * count as its maximum and uses fewer slices for delta evaluations whose
 * result only needs to resolve the next sweep (see inv_factor_refine). */
int ifac_set_split_slices(ifac_ctx* ctx, int slices);
/* Whether the mixed-precision refinements (inv_factor_refine and
 * inv_factor_refine_batched with TF32/BF16) keep the results of their
 * low-precision products -- X = S Z, the upper triangle of Z^T X, delta^2
 * and M = Z P -- in FP32 (on, the default) or in FP64 (off).  These results
 * are FP32 accumulators, so both settings give bitwise the same factors; FP32
 * halves the bytes these intermediates take in memory and move through HBM.
 * Returns IFAC_ERR_INVALID for a NULL context. */
int ifac_set_fp32_intermediates(ifac_ctx* ctx, int on);
const char* ifac_last_error(const ifac_ctx* ctx);
void ifac_opts_default(ifac_opts* opts);

/* ---------------------------------------------------------------- */
/* Storage helpers                                                   */
/* ---------------------------------------------------------------- */

/* Copy a host BSR (arrays as in ifac_bsr) to a new library-owned device
 * matrix; block norms are computed.  Validates the pattern (row_ptr
 * monotone, columns in range and strictly increasing): IFAC_ERR_INVALID. */
int ifac_bsr_upload(ifac_ctx* ctx, int64_t n, int32_t bs, int32_t nb, int64_t nnzb,
                    const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                    ifac_bsr* out);

/* Copy a device BSR to host arrays of sizes nb+1, nnzb, nnzb*bs*bs (any of
 * the three may be NULL to skip it).  Synchronises the stream. */
int ifac_bsr_download(ifac_ctx* ctx, const ifac_bsr* a, int32_t* row_ptr, int32_t* col_idx,
                      double* val);

/* Release a library-allocated matrix and zero the struct.  NULL-safe. */
void ifac_bsr_free(ifac_ctx* ctx, ifac_bsr* a);

/* ---------------------------------------------------------------- */
/* Block-sparse operations                                           */
/* ---------------------------------------------------------------- */

/* C = alpha * op(A) * op(B), op(X) = X^T when transX != 0; then every output
 * block with Frobenius norm strictly below tau is removed (Section 5: blocks
 * with norm smaller than the threshold are removed after every product).
 * The output pattern before truncation is every (I, J) for which some K has
 * op(A)_IK and op(B)_KJ stored.  A and B: same n and bs.  prec: IFAC_FP64 (any
 * bs in {16, 32, 64}), or IFAC_TF32 / IFAC_BF16 (bs 32, 64 or 128): the
 * operands are
 * rounded to that format (BF16 round-to-nearest-even from FP64; TF32 via FP32,
 * round-to-nearest-even, then round-half-away; magnitudes below 2^-126 become
 * zero), products are accumulated in
 * FP32 on the tensor cores, and the result, its norms and the truncation are
 * FP64.  IFAC_FP64_SPLIT (bs 32, 64 or 128): an FP64-accurate product on the tensor
 * cores (error-free splitting, Ozaki et al. 2012): each scalar row i of op(A)
 * and column j of op(B) is scaled by a power of two sigma_i, tau_j above its
 * largest magnitude and split into s slices of 7-bit integers held exactly in
 * BF16 (s = 7 unless ifac_set_split_slices); slice products accumulate
 * exactly in FP32 over windows of at most 1024 scalar K terms (16 blocks at
 * bs 64), pairs of slice orders
 * s_a + s_b <= s + 1, and are summed in 64-bit fixed point at 2^-f sigma_i
 * tau_j, f <= 56 chosen so that no partial sum can overflow; the result is
 * converted to FP64 once.  Element error about 2^-(7 s - 3) K_ij sigma_i tau_j
 * (2^-46 for s = 7) plus 2^-f sigma_i tau_j per window.  IFAC_ERR_TIMEOUT if
 * a device pipeline wait expired; IFAC_ERR_CUDA if a fixed-point sum
 * overflowed (not expected: the scale is bounded from the operands). */
int bsr_gemm_trunc(ifac_ctx* ctx, const ifac_bsr* A, int transA, const ifac_bsr* B, int transB,
                   double alpha, double tau, int prec, ifac_bsr* C);

/* The same product for a result the caller knows to be symmetric, such as
 * Z^T (S Z) with S symmetric (delta = I - Z^T S Z, Eq. 2.1) or delta delta:
 * only the output blocks (I, J) with J >= I are formed (same pattern rule,
 * arithmetic and truncation as bsr_gemm_trunc) and block (J, I) is set to the
 * transpose of block (I, J); a diagonal block is the product's own
 * (symmetric up to rounding).  Nothing checks that op(A) op(B) is symmetric:
 * otherwise the strict lower triangle is simply the transposed upper one.
 * bs = 64 (IFAC_ERR_UNSUPPORTED otherwise); the other arguments, ownership
 * and errors as bsr_gemm_trunc. */
int bsr_gemm_sym_trunc(ifac_ctx* ctx, const ifac_bsr* A, int transA, const ifac_bsr* B, int transB,
                       double alpha, double tau, int prec, ifac_bsr* C);

/* C = alpha A + beta B + gamma I on the union pattern (B may be NULL; the
 * diagonal blocks are added when gamma != 0).  No truncation: the paper
 * truncates after products and leaf routines only (Section 5). */
int bsr_add(ifac_ctx* ctx, double alpha, const ifac_bsr* A, double beta, const ifac_bsr* B,
            double gamma, ifac_bsr* C);

/* C = A without its blocks of Frobenius norm < tau (the truncation of S,
 * Section 5). */
int bsr_truncate(ifac_ctx* ctx, const ifac_bsr* A, double tau, ifac_bsr* C);

/* ||A||_F and the Gershgorin bound max_i sum_j |A_ij| (Section 2.2). */
int bsr_fro(ifac_ctx* ctx, const ifac_bsr* A, double* out);
int bsr_gershgorin(ifac_ctx* ctx, const ifac_bsr* A, double* out);

/* Batched dense leaf routine of Algorithms 1-2 ("factorize S^-1 = Z Z^T"):
 * for each of `count` row-major nl x nl SPD matrices at S + k*nl*nl (device),
 * writes the upper-triangular Z = L^-T (S = L L^T, positive diagonal) to
 * Z + k*nl*nl (device; may equal S for in-place).  info[k] (device int) is 0,
 * or j+1 when pivot j of matrix k was not positive (that Z is undefined).
 * Returns IFAC_ERR_NOT_SPD when any info is non-zero.  nl <= 1024. */
int leaf_invchol_batched(ifac_ctx* ctx, int count, int nl, const double* S, double* Z, int* info);

/* The same batched leaf inverse Cholesky for callers that cannot allocate
 * device memory when they call it: frameworks that own the whole
 * device-memory budget and forbid allocations behind their allocator's back,
 * or loops that cannot afford an allocation's synchronisation with the
 * device.  The paper has no counterpart; this is a library convenience.
 *
 * Arguments as leaf_invchol_batched, except that `stream` (a cudaStream_t)
 * replaces the context.  It allocates nothing: its scratch (the diagonal-tile
 * inverses, count * ceil(nl/32) * 1024 doubles, plus count * np * np doubles
 * of identity-padded copies when nl is not a multiple of 32, np = nl rounded
 * up to 32) lives in one fixed 32 MiB device array (4 Mi doubles) that every
 * GPU loading the library holds until exit.  Larger requests return
 * IFAC_ERR_TOO_LARGE and touch nothing.
 *  - S and Z must be equal (in place) or not overlap at all; a partial
 *    overlap returns IFAC_ERR_INVALID and touches nothing.
 *  - The first call on a device looks up that array's device address
 *    (cudaGetSymbolAddress, with that device current); make this first call
 *    before any stream capture.  The address is kept for the process, so a
 *    device reset (cudaDeviceReset) between calls is not supported.
 *  - The call is asynchronous on `stream`: it returns after enqueueing and
 *    does not read info back; info[k] (device) is set as in
 *    leaf_invchol_batched once the stream reaches it.
 *  - Every call uses the same scratch array, so calls whose work overlaps on
 *    the GPU (other streams, other host threads) race; serialise them.  The
 *    scratch keeps the previous call's contents; nothing in it needs to start
 *    at zero, since every element is written before it is read.
 * Returns IFAC_OK, IFAC_ERR_INVALID (bad arguments), IFAC_ERR_TOO_LARGE or
 * IFAC_ERR_CUDA (a launch or copy failed). */
int leaf_invchol_batched_noalloc(void* stream, int count, int nl, const double* S, double* Z, int* info);

/* The same matrix stored with block size bs (32, 64 or 128): exact.  Block
 * (I', J') of the result holds rows [I' bs, (I'+1) bs) and columns
 * [J' bs, (J'+1) bs) of the padded input, gathered from every stored input
 * block that overlaps it; result blocks that come out all zero are dropped,
 * except diagonal blocks; padding rows that the new block size adds past the
 * input's padded size get a unit diagonal.  No truncation.  The paper stores
 * its matrices with one block size throughout; this serves the block-size
 * choice of ifac_autotune_batched.  IFAC_ERR_UNSUPPORTED for another bs. */
int bsr_reblock(ifac_ctx* ctx, const ifac_bsr* A, int32_t bs, ifac_bsr* out);

/* Tile schedules of the context's bs-64 tensor-core products, one for the
 * TF32/BF16 products (narrow_kmax) and one for the split FP64-accurate ones
 * (narrow_kmax_split): -1 (default) narrow 128 x 64 tiles for TF32/BF16
 * products whose longest tile has at most 16 K blocks and super-tiles for
 * the others, narrow tiles for every split product; 0 super-tiles for every
 * product; k > 0 narrow tiles for every product whose longest tile has at
 * most k K blocks.
 * Results are the same products either way (TF32/BF16 up to FP32 summation
 * order; split products within their error bound).  Products at bs 32 and
 * 128 always use narrow tiles.  IFAC_ERR_INVALID below -1. */
int ifac_set_schedule(ifac_ctx* ctx, int32_t narrow_kmax, int32_t narrow_kmax_split);

/* Autotuner of the batched refinement (config 4's block size and tile
 * schedule): for each block size 32, 64 and 128 the members are re-blocked
 * (bsr_reblock) and placed on the diagonal of one matrix, truncated at tau,
 * and a probe is timed with CUDA events on the context's stream -- two
 * low-precision products (X = S S and X X, in opts->prec, TF32 unless that
 * is BF16; X has about the pattern of the later iterates) and one split
 * FP64-accurate product X X, best of two runs;
 * at bs 64 each tile schedule of ifac_set_schedule (-1, 0, and narrow for
 * all) is probed for each of the two kinds of product.  The predicted batch
 * time weighs the probes by a typical
 * sweep count (4 products in each of 6 low-precision sweeps, 2 in each of 4
 * FP64-accurate delta evaluations); the fastest block size and schedules are
 * returned in out, and the schedules are set on the context.  The caller
 * re-blocks its members to out->bs (bsr_reblock) before
 * inv_factor_refine_batched.  Synchronises the stream; allocates the probe's
 * matrices through the context's allocator and frees them. */
int ifac_autotune_batched(ifac_ctx* ctx, int count, const ifac_bsr* const* S, double tau, const ifac_opts* opts,
                          ifac_tune_result* out);

/* ---------------------------------------------------------------- */
/* Factorizations                                                    */
/* ---------------------------------------------------------------- */

/* Iterative refinement with a scaled identity start (IRSI), Section 2.2:
 * S is truncated at tau; beta = Gershgorin bound; Z_0 = c I; per sweep
 * delta = I - Z^T (S Z) (two truncated products), the stop tests, then
 * M = Z sum_{k=1}^{m} b_k delta^k and Z <- Z + M (Eq. 2.1).  Stops when
 * ||delta||_F <= target, or ||delta_{i+1}||_F > ||delta_i||_F^(m+1), or after
 * max_iter corrections; returns the last iterate (whose delta was last
 * evaluated).  Returns IFAC_WARN_TARGET_NOT_MET when the rule stopped it
 * above the target, IFAC_ERR_NO_CONVERGENCE at max_iter.  rep may be NULL.
 *
 * Mixed precision (opts->prec = IFAC_TF32 or IFAC_BF16, bs 32, 64 or 128;
 * at bs 128 delta_prec must be IFAC_FP64_SPLIT; at bs 64 the symmetric
 * products Z^T (S Z) and delta delta form their upper block triangle only): every
 * block product of a sweep runs on the tensor cores with inputs rounded to
 * that format and FP32 accumulation (the products' results are kept as those
 * FP32 values, ifac_set_fp32_intermediates), while sums, block norms,
 * truncation and delta = I - Y stay FP64, until the automatic rule of Section 2.2
 * (||delta_{i+1}||_F > ||delta_i||_F^(m+1): rounding dominates) fires or
 * ||delta||_F stops decreasing (the rule cannot fire once the rounding floor
 * of ||delta||_F, which grows like sqrt(n), lies above 1).  From
 * then on delta is evaluated with FP64 products for the same Z and after each
 * correction (the correction M stays low precision, so convergence becomes
 * linear with a rate near the format's unit roundoff), stopping at
 * ||delta||_F <= target or when ||delta||_F no longer decreases.  The returned
 * Z is the last one whose delta was evaluated with FP64 products.  With low-
 * precision corrections Z converges to an inverse factor S^-1/2 Q with Q close
 * to orthogonal, not to S^-1/2 itself.  In the mixed schedule Z^T (S Z) and
 * delta^k are formed on their upper block triangle and completed by symmetry
 * (as bsr_gemm_sym_trunc).  With split FP64-accurate evaluations
 * (opts->delta_prec = IFAC_FP64_SPLIT) each evaluation takes the fewest
 * slices s (at least 3, at most the context's count) whose error level
 * 2^-(7 s - 3) sqrt(n) is at most max(target, u e) / 10, with u the low
 * format's unit roundoff (TF32 2^-11, BF16 2^-8) and e the predicted
 * ||delta||_F: a tenth of the last low-precision value for the first, u times
 * the previous value after that (a sweep with low-precision M reduces
 * ||delta||_F by about u).  An evaluation whose own ||delta||_F shows that it
 * needed more slices is repeated with all of them, so the error stays below
 * a tenth of the target at the stop test. */
int inv_factor_refine(ifac_ctx* ctx, const ifac_bsr* S, double tau, double target,
                      const ifac_opts* opts, ifac_bsr* Z, ifac_report* rep);

/* Localized inverse factorization, Algorithm 2: the block range is halved
 * (block-aligned midpoint, left half floor(nb/2)) until a range has at most
 * leaf_size rows (or one block); leaves get Z = L^-T, truncated at tau; each
 * parent forms Z_0 = diag(Z_A, Z_C), delta_0 = [0 X; X^T 0] with
 * X = -Z_A^T (B Z_C), and refines with the localized update of Eq. (2.2):
 * M = Z sum_{k>=1} b_k delta^k, Z' = Z + M, T = S M,
 * delta' = delta - Z'^T T - T^T Z, stopping as Algorithm 4 (the first
 * check never stops; then ||delta'|| > ||delta||^(m+1), or target, or
 * max_iter).  All sub-problems of one depth are refined together.  S must
 * already be in the wanted order (e.g. recursive coordinate bisection). */
int inv_factor_localized(ifac_ctx* ctx, const ifac_bsr* S, double tau, double target,
                         const ifac_opts* opts, ifac_bsr* Z, ifac_report* rep);

/* Recursive inverse Cholesky (Algorithm 1, left-looking, two blocks per
 * dimension): S = [S00 S01; S01^T S11] split at the block-aligned midpoint
 * while the range has more than opts->leaf_size rows,
 *   Z00 = rinch(S00), R = Z00^T S01, Q = -R^T R + S11, Z11 = rinch(Q),
 *   Z01 = -(Z00 R) Z11, Z10 = 0,
 * and at the lowest level the dense leaf routine Z = L^-T (S = L L^T).  S is
 * truncated at tau first; every product and every leaf factor is truncated
 * (Section 5).  Without truncation Z is the inverse Cholesky factor (block
 * upper triangular, Z^T S Z = I).  opts: leaf_size; prec IFAC_FP64 or
 * IFAC_FP64_SPLIT (bs 32, 64 or 128).  rep (may be NULL): levels = recursion depth,
 * products, block_pairs, nnzb_Z, flops.  IFAC_ERR_NOT_SPD if a leaf (S00 or
 * a Schur complement Q) is not positive definite. */
int inv_factor_rinch(ifac_ctx* ctx, const ifac_bsr* S, double tau, const ifac_opts* opts, ifac_bsr* Z,
                     ifac_report* rep);

/* Refinement from a scaled identity (as inv_factor_refine, Section 2.2) of
 * `count` independent matrices S[0..count-1] in one launch sequence: the
 * members sit on the diagonal of one block-diagonal matrix, so every block
 * product of a sweep serves all of them.  Each member has its own Gershgorin
 * bound, Z_0 = c_k I, ||delta||_F and stop test (target, the rule of Section
 * 2.2, or max_iter); a stopped member leaves the batch.  With opts->prec
 * TF32/BF16 (tensor cores, bs 32, 64 or 128) every member follows the mixed-precision
 * schedule of inv_factor_refine: low-precision sweeps until its floor, then
 * delta with FP64-accurate products (opts->delta_prec) and M in opts->prec
 * until the target or until ||delta||_F stops falling.  The final residual
 * of every member is evaluated with FP64-accurate products (delta_prec) and
 * returned in rep[k].resid_fro.
 * All members need the same bs.  Z[k] (count entries) receive the factors;
 * rep may be NULL or hold count reports (batch-wide counters are repeated in
 * each).  Returns IFAC_WARN_TARGET_NOT_MET if any member stopped above the
 * target. */
int inv_factor_refine_batched(ifac_ctx* ctx, int count, const ifac_bsr* const* S, double tau, double target,
                              const ifac_opts* opts, ifac_bsr* Z, ifac_report* rep);

/* Reverse-mode derivative of K refinement sweeps of Eq. (2.1) (m = 2, from
 * Z_0 = c I, c = 1/sqrt(beta) of the truncated S, held constant) on a frozen
 * block pattern, for the loss L = tr(Z_K^T F Z_K).  A recording run with
 * truncation at tau (Section 5) fixes the block pattern of every
 * intermediate; the differentiated function restricts every product to its
 * recorded pattern, so L is a polynomial in the stored entries of S and the
 * derivative is exact up to rounding.  The paper has no derivative; this is
 * the hand-written adjoint of those sweeps (all FP64).  F: same n and bs as S
 * (any pattern).  Outputs: *L, and Sbar = dL/dS with every stored entry of S
 * an independent variable (not symmetrized), on the pattern of the caller's
 * S (zero on blocks the truncation removed).  K in 0..64. */
int inv_factor_refine_adjoint(ifac_ctx* ctx, const ifac_bsr* S, const ifac_bsr* F, int K, double tau,
                              double* L, ifac_bsr* Sbar);

/* ||I - Z^T S Z||_F with untruncated products (the factorization error of
 * Table 1). */
int inv_factor_resid(ifac_ctx* ctx, const ifac_bsr* S, const ifac_bsr* Z, double* out);

/* ---------------------------------------------------------------- */
/* Failure-path self-test                                            */
/* ---------------------------------------------------------------- */

/* Exercises the bounded device-side waits of the tensor-core product kernel
 * without a fault: one launch of that kernel (two CTAs, a one-tile product of
 * 64 x 64 zero blocks) whose copy and MMA stages are told to do no work, so
 * the epilogue's first wait for an accumulator never completes and expires
 * after wait_limit polls (1..2^30; about 2^20 polls take milliseconds).  The
 * kernel then records the error flag, releases its tensor memory and
 * returns; nothing was copied or multiplied, so nothing is left in flight.
 * Returns IFAC_ERR_TIMEOUT (the status every library call returns when one
 * of its waits expires) and clears the flag, leaving the context usable;
 * IFAC_ERR_INVALID for a wait_limit outside the range.  Synchronises the
 * context's stream.  Not part of the paper's method: it tests the library's
 * failure handling (the bound on every wait inside the pipeline). */
int ifac_selftest_wait_timeout(ifac_ctx* ctx, int64_t wait_limit);

#ifdef __cplusplus
}
#endif
#endif /* IFAC_H */
