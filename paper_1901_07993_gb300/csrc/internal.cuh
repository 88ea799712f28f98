// internal.cuh -- shared declarations of the CUDA library behind ifac.h.
//
// Errors inside the library are C++ exceptions (ifac::Error) that the
// extern "C" entry points in api.cu turn into status codes; device buffers
// are owned by RAII holders so that an error path frees what it allocated.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <initializer_list>
#include <cstdint>
#include <string>
#include <utility>
#include <unordered_map>
#include <vector>

#include "ifac.h"

struct ifac_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool custom_alloc = false;
  ifac_allocator alloc{};
  std::string err;
  // counters of the current driver call
  int64_t products = 0;
  int64_t pairs = 0;
  int64_t launches = 0;
  int64_t gemm_launches = 0;
  int64_t tc_launches = 0, split_launches = 0;
  int64_t pairs_fp64 = 0, pairs_tc = 0, pairs_split = 0, slice_pairs = 0;
  double bytes_fp64 = 0, bytes_tc = 0, bytes_split = 0;  // algorithmic bytes of the product launches
  std::vector<char> event_kind;  // per recorded event pair: 0 FP64, 1 tensor-core (TF32/BF16), 2 split kernel
  // optional event timing of the numeric product kernels
  bool profile = false;
  std::vector<cudaEvent_t> events;
  size_t events_used = 0;
  // small pinned host buffer for scalar read-backs
  void* pinned = nullptr;
  // device words: [0] error flag set by bounded waits that expired;
  // counters [1] FP64 and [2] tensor-core block pairs of the current call
  int* dev_err = nullptr;
  int split_slices = 7;  // BF16 slices per operand for IFAC_FP64_SPLIT products
  bool fp32_mid = true;  // mixed refinements keep low-precision product results in FP32
  int fp64_prec = IFAC_FP64;  // IFAC_FP64_SPLIT: gemm() runs FP64 products of bs = 64 on the split kernel
  unsigned long long* dev_pairs = nullptr;
  // tile schedule of bs-64 tensor-core products (TF32/BF16, and split): -1
  // narrow tiles when no tile has more than 16 K blocks (split: and one
  // window holds them), 0 super-tiles only, k > 0 narrow tiles when no tile
  // has more than k
  int narrow_kmax = -1;
  int narrow_kmax_split = -1;
  // device blocks up to 4 GB (without a caller allocator): a freed block goes
  // back to a list per size class and is handed out again, in the order of
  // the context's stream, instead of a stream-ordered free and allocation --
  // a factorization of the 262,144-row chain allocates about 1200 blocks, and
  // the pool spent 4.6 ms of host time on them
  std::unordered_map<size_t, std::vector<void*>> cache;
  std::unordered_map<void*, size_t> cache_live;  // handed-out blocks and their size class
  size_t cached_bytes = 0;
};

namespace ifac {

struct Error {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg);
void check_cuda(cudaError_t e, const char* what, const char* file, int line);
#define IFAC_CK(x) ::ifac::check_cuda((x), #x, __FILE__, __LINE__)
#define IFAC_CK_LAUNCH() \
  do { ++ctx->launches; ::ifac::check_cuda(cudaGetLastError(), "kernel launch", __FILE__, __LINE__); } while (0)

void* dalloc(ifac_ctx* ctx, size_t bytes);
void dfree(ifac_ctx* ctx, void* p);

// Typed device buffer owned by a context.
template <typename T>
struct Buf {
  ifac_ctx* ctx = nullptr;
  T* p = nullptr;
  size_t n = 0;
  Buf() = default;
  Buf(ifac_ctx* c, size_t count) : ctx(c), n(count) {
    p = static_cast<T*>(dalloc(c, (count ? count : 1) * sizeof(T)));
  }
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  Buf(Buf&& o) noexcept : ctx(o.ctx), p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  Buf& operator=(Buf&& o) noexcept {
    if (this != &o) { reset(); ctx = o.ctx; p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~Buf() { reset(); }
  void reset() { if (p) dfree(ctx, p); p = nullptr; n = 0; }
  T* release() { T* q = p; p = nullptr; n = 0; return q; }
  T* get() const { return p; }
};

// A library-owned block-sparse matrix (all arrays device, norms always set).
// vmap (optional, internal to the drivers): block p's values are at
// m.val + vmap[p] bs^2 -- a product truncated without moving its kept blocks
// (compact with nocopy); only the consumers that take a value map read it.
// f32 (internal to the mixed drivers): m.val holds FP32 values (bs^2 floats
// per block), the exact results of a TF32/BF16 product; only the consumers
// given a matching flag read them.
struct Mat {
  ifac_ctx* ctx = nullptr;
  ifac_bsr m{};
  Buf<int32_t> vmap;
  bool f32 = false;
  Mat() = default;
  explicit Mat(ifac_ctx* c) : ctx(c) {}
  Mat(const Mat&) = delete;
  Mat& operator=(const Mat&) = delete;
  Mat(Mat&& o) noexcept : ctx(o.ctx), m(o.m), vmap(std::move(o.vmap)), f32(o.f32) {
    o.m = ifac_bsr{};
    o.f32 = false;
  }
  Mat& operator=(Mat&& o) noexcept {
    if (this != &o) {
      reset();
      ctx = o.ctx;
      m = o.m;
      o.m = ifac_bsr{};
      vmap = std::move(o.vmap);
      f32 = o.f32;
      o.f32 = false;
    }
    return *this;
  }
  const int32_t* map() const { return vmap.p; }
  ~Mat() { reset(); }
  void reset();
  ifac_bsr release() { ifac_bsr r = m; m = ifac_bsr{}; return r; }
  const ifac_bsr& operator*() const { return m; }
};

// Allocate the arrays of an n x n matrix with nnzb blocks.
Mat mat_alloc(ifac_ctx* ctx, int64_t n, int bs, int nb, int64_t nnzb);

// Read back a few device ints/int64/doubles (synchronises the stream).
void to_host(ifac_ctx* ctx, void* host, const void* dev, size_t bytes);
// Several small read-backs (4096 bytes in all at most) behind one synchronisation.
struct HostRead {
  void* host;
  const void* dev;
  size_t bytes;
};
void to_host_many(ifac_ctx* ctx, std::initializer_list<HostRead> reads);

// ---- pattern utilities (pattern.cu) ----
int words_per_row(int nb);
// exclusive scan of in[0..n) into out[0..n], out[n] = total; returns total (syncs)
int64_t scan_counts(ifac_ctx* ctx, const int32_t* in, int32_t* out, int n, bool want_total);
// CSR view of op(X): rows of X^T with the index of the source block of X.
struct View {
  const int32_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const int32_t* src = nullptr;  // nullptr = identity
  Buf<int32_t> own_rp, own_ci, own_src;
};
View view_rows(ifac_ctx* ctx, const ifac_bsr& A, bool trans);
// Bitmap (nb x W words) of the pattern of op(A): bit (r, c) set when op(A)_rc is stored.
Buf<uint32_t> pattern_bitmap(ifac_ctx* ctx, const ifac_bsr& A, bool trans);
// Row pattern from a bitmap: allocates and fills rp[nb+1], ci[nnzb].
struct Pattern {
  Buf<int32_t> rp, ci, row;
  int64_t nnzb = 0;
};
// known_nnzb >= 0: the number of set bits is known (e.g. a transposed
// pattern), so it is not read back from the device
Pattern pattern_from_bitmap(ifac_ctx* ctx, const uint32_t* bm, int nb, int64_t known_nnzb = -1);
// Symbolic product pattern of op(A) op(B); upper: only the blocks (I, J)
// with J >= I.
Pattern product_pattern(ifac_ctx* ctx, const View& arows, const ifac_bsr& B, bool transB, int nb,
                        bool upper = false);
// Union pattern of A, B (nullable) and the diagonal (if diag).
Pattern union_pattern(ifac_ctx* ctx, const ifac_bsr& A, const ifac_bsr* B, bool diag);
// Pattern of U + U^T, B (nullable) and the diagonal (if diag).
Pattern sym_pattern(ifac_ctx* ctx, const ifac_bsr& U, const ifac_bsr* B, bool diag);
// Expand row_ptr to a per-block row index.
void expand_rows(ifac_ctx* ctx, const int32_t* rp, int nb, int32_t* row);
// Keep blocks with !(norm < tau) of an (uncompacted) matrix; returns the compacted one.
// nocopy: the kept blocks stay where they are (the result's vmap points to them).
Mat compact(ifac_ctx* ctx, Mat&& full, const int32_t* row, double tau, bool nocopy = false);
// Keep blocks selected by a per-block mask (1 keep / 0 drop).
Mat select_blocks(ifac_ctx* ctx, const ifac_bsr& A, const int32_t* row, const uint8_t* keep);

// ---- numeric kernels ----
// FP64 numeric block product into the pattern (rp/ci/row) of C; writes
// C.val, C.norms; adds the number of block pairs to *pairs_dev.
void gemm_numeric_fp64(ifac_ctx* ctx, const View& arows, bool tA_blocks, const ifac_bsr& A,
                       const View& bcols, bool tB_blocks, const ifac_bsr& B, double alpha,
                       ifac_bsr& C, const int32_t* crow, unsigned long long* pairs_dev);
// Converted copies of an operand that several products share: S as op(A) of
// X = S Z across the sweeps of one refinement (from_b false: the K-major
// copy in op(A)'s view order, filled by the first product that uses it), or
// Z as op(B) of X = S Z and then as op(A) = Z^T of Z^T X (from_b true: filled
// by the op(B) side, transposed blocks in Z's stored order; the Z^T product
// reaches them through its view's source indices).  Holds the K-major
// TF32 / BF16 copy, and the BF16 slices with their row (column) scale
// exponents and scaled 1-norm bound.  Slice k does not depend on the slice
// count, so slices held for s serve any split product with at most s.  The
// owner resets it when the operand changes.
struct OperandCache {
  bool from_b = false;     // filled from an op(B) (see above)
  bool b_ready = false;    // conv is this matrix's op(B) copy (transposed blocks, stored order),
                           // written by its producer (poly2_operand): the product uses it as is
  Buf<int32_t> tpos;       // an exactly symmetric matrix with its op(A) copy in conv: the
                           // position of each block's transpose, so conv serves op(B) too
  int conv_elt = 0;        // bytes per element of conv (4 TF32, 2 BF16); 0 empty
  Buf<uint8_t> conv;       // (nnzb + 1) blocks, the last one zero
  int split_ns = 0;        // slices held (0 empty)
  int want_ns = 0;         // slices to compute when filling (at least the product's)
  Buf<uint8_t> split;      // split_ns slices, slice-major, (nnzb + 1) blocks each
  Buf<int> sexp;           // row scale exponents of op(A)
  float l1 = 0.f;          // scaled row 1-norm bound of op(A)
  float l2 = 0.f;          // scaled row 2-norm bound of op(A)
  void reset() {
    from_b = false;
    b_ready = false;
    tpos.reset();
    conv_elt = 0;
    conv.reset();
    split_ns = 0;
    split.reset();
    sexp.reset();
    l1 = 0.f;
    l2 = 0.f;
  }
};

// Tensor-core (TF32/BF16 in, FP32 accumulate, or split FP64-accurate)
// numeric block product, bs 32, 64 or 128.  brows: rows of op(B).  upper: C
// holds only blocks with J >= I.  pairs_dev[0] counts the block pairs
// multiplied; for split products pairs_dev[1] counts block pairs times slice
// pairs.  TF32/BF16 only: out32, C.val receives FP32 values; b32, B.val holds
// FP32 values.
void gemm_numeric_tc(ifac_ctx* ctx, int prec, const View& arows, bool tA, const ifac_bsr& A, const View& brows,
                     bool tB, const ifac_bsr& B, double alpha, ifac_bsr& C, const int32_t* crow, bool upper,
                     unsigned long long* pairs_dev, OperandCache* acache = nullptr,
                     OperandCache* bcache = nullptr, const OperandCache* bpre = nullptr,
                     const int32_t* avmap = nullptr, const int32_t* bvmap = nullptr, bool out32 = false,
                     bool b32 = false);
// the mixed schedule's P = b1 D + b2 (U + strict_upper(U)^T) at m = 2 written
// as the low-precision (elt 4 TF32, 2 BF16) op(B) copy of P's pattern (row
// index of each block in prow) into out ((P.nnzb + 1) blocks), bs 64; u32:
// U's values are FP32
void poly2_lp(ifac_ctx* ctx, int elt, const ifac_bsr& U, const ifac_bsr& D, double b1, double b2,
              const ifac_bsr& P, const int32_t* prow, void* out, const int32_t* umap = nullptr, bool u32 = false);
// TF32 (elt 4) / BF16 (elt 2) product on narrow tiles of 128 accumulator
// rows (gemm_band.cu), bs 32, 64 or 128.  mapA / mapB: CUtensorMap of the
// K-major low-precision copies of op(A) and op(B), boxes of one swizzle atom
// by bs rows (band_lp_shape); tiles, ntiles, tile_nk, rec, rec_off: the tile
// plan for tmb x tnb blocks (copy indices of op(A)_IK of the tile's block
// rows, then op(B)_KJ of its block columns).
struct BandShape {
  int tmb, tnb;      // block rows and columns of a tile
  int atom_elems;    // elements of one swizzle atom row (the box's inner extent)
  int atom_bytes;    // 128 (128-byte swizzle) or 64 (64-byte swizzle)
};
BandShape band_lp_shape(int elt, int bs);
void band_lp_product(ifac_ctx* ctx, int elt, int bs, const void* mapA, const void* mapB, const int32_t* tiles,
                     const int* ntiles, const int32_t* tile_nk, const int32_t* rec, const int32_t* rec_off,
                     const int32_t* cpos, int tiles_bound, double alpha, ifac_bsr& C, bool out32 = false);
// the same matrix with block size bs (32, 64, 128), exact (reblock.cu)
Mat reblock(ifac_ctx* ctx, const ifac_bsr& A, int bs);
// block size and bs-64 tile schedule of a batch from timed probe products
void autotune(ifac_ctx* ctx, int count, const ifac_bsr* const* S, double tau, const ifac_opts& o,
              ifac_tune_result* out);
// Failure-path self-test: a tensor-core launch whose pipeline never fills, so
// its bounded waits expire after wait_limit polls (sets the device error flag).
void tc_wait_timeout_selftest(ifac_ctx* ctx, long long wait_limit);
// bmap / umap: value maps of B / U (Mat::vmap), or null; b32 / u32: B's / U's
// values are FP32 (Mat::f32)
// lp / lp_elt: a low-precision copy of C in the layout of an op(A) operand
// ((C.nnzb + 1) blocks, the caller zeroes the last), lp_elt 4 TF32, 2 BF16
void add_numeric(ifac_ctx* ctx, double alpha, const ifac_bsr& A, double beta, const ifac_bsr* B,
                 double gamma, ifac_bsr& C, const int32_t* crow, const int32_t* bmap = nullptr, void* lp = nullptr,
                 int lp_elt = 0, bool b32 = false);
// C = alpha (U + strict_upper(U)^T) + beta B + gamma I on the pattern of sym_pattern
// mirror: diagonal blocks are completed from their upper triangle too
void sym_numeric(ifac_ctx* ctx, double alpha, const ifac_bsr& U, double beta, const ifac_bsr* B, double gamma,
                 ifac_bsr& C, const int32_t* crow, const int32_t* umap = nullptr, bool mirror = false,
                 void* lp = nullptr, int lp_elt = 0, bool u32 = false);
// out[q]: the position in A of the transpose (J, I) of A's block q = (I, J)
// (row: each block's row index); A's pattern symmetric
void transposed_positions(ifac_ctx* ctx, const ifac_bsr& A, const int32_t* row, int32_t* out);
void block_norms(ifac_ctx* ctx, const ifac_bsr& A, double* norms);
// per block-row sum of squared block norms
void row_sq_norms(ifac_ctx* ctx, const ifac_bsr& A, double* rowsq);
double fro_host(ifac_ctx* ctx, const ifac_bsr& A);
double gershgorin_host(ifac_ctx* ctx, const ifac_bsr& A);
// precision of the FP64-accurate delta evaluations of the mixed schedule
int delta_prec_of(const ifac_opts& o, int bs);
// unit roundoff of a low-precision product format (TF32 2^-11, BF16 2^-8)
double unit_roundoff(int prec);
// error level of a split delta evaluation of an n-row matrix with s slices
double split_delta_error(int slices, int64_t n);
// the accuracy a delta evaluation of the mixed schedule needs when
// ||delta||_F = e: a tenth of what the next low-precision sweep leaves
double delta_need(double e, double target, double u);
// In the FP64 phase a sweep reduces ||delta||_F by about u (below 1e-2 for
// TF32 and BF16 on every input measured), so a ratio above this one means the
// sweeps now converge toward the zero of the s-slice evaluation, which errs
// by its own error: on block-dense factors far above split_delta_error
// (n = 8192, 3D cluster, TF32: seven slices leave ||I - Z^T S Z||_F at 6e-10
// while they evaluate it as 1.4e-10).  From there on every evaluation takes
// all slices.
constexpr double kStallRatio = 0.25;
// slices for an evaluation whose ||delta||_F is predicted at e_pred
int delta_slices(const ifac_ctx* ctx, double e_pred, double target, double u, int64_t n);
// sets the context's split slice count for the scope's lifetime
struct SlicesScope {
  ifac_ctx* c;
  int old;
  SlicesScope(ifac_ctx* c_, int s) : c(c_), old(c_->split_slices) { c->split_slices = s; }
  ~SlicesScope() { c->split_slices = old; }
  SlicesScope(const SlicesScope&) = delete;
  SlicesScope& operator=(const SlicesScope&) = delete;
};
// true the first time it is called with this flag word for `device` (per
// process): per-device one-time settings such as kernel attributes
inline bool first_on_device(std::atomic<unsigned long long>& seen, int device) {
  const unsigned long long bit = 1ull << (device & 63);
  return !(seen.fetch_or(bit) & bit);
}
// driver report: counters reset at entry, filled (with the device counters) at exit
void report_init(ifac_ctx* ctx, ifac_report* r, const ifac_opts& o);
void report_finish(ifac_ctx* ctx, ifac_report* r, const ifac_bsr& Z);
// Z_leaf = L^-T (upper triangular blocks, truncated) of the principal
// sub-matrices [first, second) of S in one batched leaf launch; other rows empty
Mat leaf_factors_ranges(ifac_ctx* ctx, const ifac_bsr& S, const std::vector<std::pair<int, int>>& ranges,
                        double tau);
int rinch(ifac_ctx* ctx, const ifac_bsr& S, double tau, const ifac_opts& o, ifac_bsr* Zout, ifac_report* rep);
// recursive inverse Cholesky of the disjoint ranges [first, second) of S together
Mat rinch_ranges(ifac_ctx* ctx, const ifac_bsr& S, const std::vector<std::pair<int, int>>& ranges, double tau,
                 int leaf_size, int* levels);
// sum_j |A_ij| for every scalar row i (nb * bs values)
void gershgorin_rows(ifac_ctx* ctx, const ifac_bsr& A, double* rs);
Mat scaled_identity(ifac_ctx* ctx, int64_t n, int bs, int nb, double c);

// ---- operations used by drivers (ops.cu) ----
// nocopy: the truncated result keeps its kept blocks in place (Mat::vmap);
// avmap / bvmap: value maps of A and B (tensor-core and split products only)
// out32 (TF32/BF16 with nocopy): the result's values stay FP32 (Mat::f32),
// exactly as accumulated, at half the bytes; b32: B's values are FP32
Mat gemm(ifac_ctx* ctx, const ifac_bsr& A, bool tA, const ifac_bsr& B, bool tB, double alpha, double tau,
         int prec = IFAC_FP64, bool upper = false, OperandCache* acache = nullptr,
         OperandCache* bcache = nullptr, const OperandCache* bpre = nullptr, bool nocopy = false,
         const int32_t* avmap = nullptr, const int32_t* bvmap = nullptr, bool out32 = false, bool b32 = false);
// P = b1 D + b2 (U + strict_upper(U)^T) (Eq. 2.1 at m = 2, U the upper block
// triangle of delta^2, D = delta) for a following low-precision product
// Z P: the returned matrix holds P's pattern only (no values); its op(B)
// copy in precision prec (TF32 or BF16) is in *pc
Mat poly2_operand(ifac_ctx* ctx, const ifac_bsr& U, const ifac_bsr& D, double b1, double b2, int prec,
                  OperandCache* pc, const int32_t* umap = nullptr, bool u32 = false);
// lp_prec (IFAC_TF32 / IFAC_BF16) with lpc: the result's op(A) copy in that
// format is written into *lpc with the FP64 values (no conversion pass later)
Mat add(ifac_ctx* ctx, double alpha, const ifac_bsr& A, double beta, const ifac_bsr* B, double gamma,
        const int32_t* bmap = nullptr, int lp_prec = 0, OperandCache* lpc = nullptr, bool b32 = false);
// the symmetric matrix whose upper block triangle (J >= I) is held by U,
// times alpha, plus beta B and gamma I: alpha (U + strict_upper(U)^T) +
// beta B + gamma I, rounded as add() rounds alpha A + beta B + gamma I
// mirror: the result is made exactly symmetric (diagonal blocks from their
// upper triangle), and with lpc its copy serves op(B) as well (lpc->tpos)
Mat sym_sum(ifac_ctx* ctx, double alpha, const ifac_bsr& U, double beta, const ifac_bsr* B, double gamma,
            const int32_t* umap = nullptr, bool mirror = false, int lp_prec = 0, OperandCache* lpc = nullptr,
            bool u32 = false);
Mat truncate(ifac_ctx* ctx, const ifac_bsr& A, double tau);
Mat copy_mat(ifac_ctx* ctx, const ifac_bsr& A);
void validate(const ifac_bsr* A, const char* name);

// ---- leaf routine (leaf.cu) ----
void leaf_invchol(ifac_ctx* ctx, int count, int nl, double* A, int* info);

// ---- drivers (drivers.cu) ----
int refine_irsi(ifac_ctx* ctx, const ifac_bsr& S, double tau, double target, const ifac_opts& o,
                ifac_bsr* Z, ifac_report* rep);
int refine_irsi_mixed(ifac_ctx* ctx, const ifac_bsr& S, double tau, double target, const ifac_opts& o,
                      ifac_bsr* Z, ifac_report* rep);
int lif(ifac_ctx* ctx, const ifac_bsr& S, double tau, double target, const ifac_opts& o,
        ifac_bsr* Z, ifac_report* rep);
double resid(ifac_ctx* ctx, const ifac_bsr& S, const ifac_bsr& Z);
int refine_batched(ifac_ctx* ctx, int count, const ifac_bsr* const* S, double tau, double target,
                   const ifac_opts& o, ifac_bsr* Z, ifac_report* reps);
int refine_adjoint(ifac_ctx* ctx, const ifac_bsr& S, const ifac_bsr& F, int K, double tau, double* L,
                   ifac_bsr* Sbar);

// event pair around a profiled launch; prof_collect sums and recycles them
void prof_begin(ifac_ctx* ctx, int kind = 0);
void prof_end(ifac_ctx* ctx);
// summed event time per kind (0: FP64 kernel, 1: tensor-core kernel)
void prof_collect(ifac_ctx* ctx, double* ms_fp64, double* ms_tc, double* ms_split = nullptr);

// Zero the device counters / read them back (read_* synchronises).
void reset_device_counters(ifac_ctx* ctx);
// block pairs multiplied on the FP64 pipe, by TF32/BF16 and by split products
// (split block pairs times slice pairs in slice_pairs, if given)
void read_device_counters(ifac_ctx* ctx, int64_t* pairs_fp64, int64_t* pairs_tc, int64_t* pairs_split = nullptr,
                          int64_t* slice_pairs = nullptr);
// Fails with IFAC_ERR_TIMEOUT (and clears the flag) if a device wait expired.
void check_device_error(ifac_ctx* ctx);

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace ifac
