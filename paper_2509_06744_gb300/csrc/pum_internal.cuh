// Internal definitions of the PUM / block-FSAI / Chebyshev-4 library (sm_103a).
//
// Device data layout (HBM):
//  * BSR matrices: row_ptr int32[n+1], col_idx int32[nnzb], vals with a padded block
//    stride: block b starts at vals + b*stride elements, stride = d*d rounded up so that
//    every block starts on a 16-byte boundary; inside a block, row-major d x d.
//  * Vectors: contiguous, unknown (i, k) at i*d + k (block-row major).
//  * Each matrix keeps a host copy of its pattern for the symbolic work (transposes,
//    Galerkin and nested triple products, adaptive FSAI candidate sets).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pum.h"

namespace pum {

// ----------------------------------------------------------------------------- errors

struct Error {
  pum_status st;
  std::string msg;
};

#define PUM_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      cudaGetLastError(); /* a non-sticky error must not resurface in a later check */       \
      throw ::pum::Error{PUM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};  \
    }                                                                                        \
  } while (0)

#define PUM_CHECK(cond, status, text)                                                        \
  do {                                                                                       \
    if (!(cond)) throw ::pum::Error{status, std::string(text)};                              \
  } while (0)

// Device status word: first error wins.
struct DevStatus {
  int code;   // pum_status
  int info;   // e.g. the block row of a failed Cholesky
  int where;  // which kernel family (see kWhere*)
  int pad;
};
enum { kWhereFsai = 1, kWhereCoarse = 2, kWhereAdaptive = 3, kWhereLanczos = 4, kWhereSell = 5, kWhereGg = 6 };

__device__ inline void set_status(DevStatus* s, int code, int info, int where) {
  if (atomicCAS(&s->code, 0, code) == 0) {
    s->info = info;
    s->where = where;
  }
}

// ----------------------------------------------------------------------------- matrices

inline size_t dt_size(int dt) { return dt == PUM_F64 ? 8 : dt == PUM_F32 ? 4 : 2; }
inline int block_stride(int d, int dt) {
  int per16 = 16 / (int)dt_size(dt);
  return (d * d + per16 - 1) / per16 * per16;
}

// Sliced block copy of a BSR matrix used by the smoother's products on large levels:
// block rows in groups of R, group g padded to S_g slots (its longest row); the values of
// (slot, block column c) are contiguous over the group's R*d output unknowns.
struct Sell {
  int R = 0;            // block rows per group (0: not built)
  int n_groups = 0;
  int64_t slots = 0;    // total slots
  int max_slots = 0;    // longest group
  int* goff = nullptr;  // n_groups + 1 slot offsets
  int* cols = nullptr;  // slots * R block columns, -1 for padding
  void* vals = nullptr; // slots * d * R * d values
};

struct Bsr {
  Sell sell;
  int n_brows = 0, n_bcols = 0, d = 0, stride = 0, dt = PUM_F64;
  int max_row_nnzb = 0;  // longest block row
  int64_t nnzb = 0;
  int* row_ptr = nullptr;  // device
  int* col_idx = nullptr;  // device
  void* vals = nullptr;    // device
  std::vector<int> h_row_ptr, h_col_idx;  // host pattern copy
  bool empty() const { return vals == nullptr; }
};

void bsr_free(Bsr& m);
// Block-FSAI application z = G^T (G r) that reads G once (gg.cu): G in the sliced layout with
// groups small enough to stay whole in shared memory, and the partial products G_ji^T t_j
// (d floats per block) stored in the block order of G^T.
struct FusedG {
  Sell S;
  int n = 0, d = 0, dt = PUM_F32;  // block rows, block size, value type of G
  int ctas = 0;   // persistent CTAs of the partial-product kernel
  int parts = 1;  // its consumer partitions of a group's slots
  int* tptr = nullptr;  // n + 1 offsets of the block rows of G^T (blocks (i, j), ascending j)
  int* tpos = nullptr;  // per slot entry of S (slot * R + row in group): position of that block
                        // of G in G^T's block order, -1 for padding
  float* w = nullptr;   // nnzb(G) * d partial products, G^T's block order
};
// Build the fused layout, its group size chosen by timing the candidates on the context's stream.
void gg_build(pum_ctx* ctx, FusedG& F, const Bsr& G);
void gg_free(FusedG& F);
// Sliced layout (sell.cu): build for a FP32/BF16 matrix; product through it (false: not applicable).
void sell_build(Bsr& m, cudaStream_t s, int sm_count);
void sell_free(Sell& s);
bool sell_mv(pum_ctx* ctx, const Bsr& M, int vdt, const void* x, int epi, const struct EpiArgs& e);
// Smoother precision of level l (FP32 only on the first fp32_levels levels of the FP32 form)
// and the precision its FSAI factors are stored in.
int level_vdt(const pum_hier* h, int l);
int level_gdt(const pum_hier* h, int l);
// Sliced layout of an FP64 matrix as FP32 pairs (hi = fl32(a), lo = fl32(a - hi)), and its
// product with a split vector (float2 hi, lo per unknown) in double-float arithmetic: RESID
// into an FP32 y with an FP64 b, or ADD into an FP64 y.
void sell_build_df(Sell& S, const Bsr& M64, cudaStream_t s, int sm_count);
// Largest group size R of a sliced layout for block size d.
int sell_rows_max(int d);
// Sliced layout with a given group size R (FP32 or BF16 values).
void sell_build_rows(Sell& S, const Bsr& M, int R, cudaStream_t s);
void sell_df_mv(pum_ctx* ctx, const Sell& S, int d, int n_brows, const void* xs, int epi, const struct EpiArgs& e,
                int tk = -1);
constexpr int kSellMinRows = 4096;  // levels with at least this many block rows use it (groups of
                                     // 8..32 rows then still give about four CTAs per SM)
// Allocate a device BSR with the given host pattern (values uninitialised).
void bsr_alloc(Bsr& m, int n_brows, int n_bcols, int d, int dt, const std::vector<int>& rp,
               const std::vector<int>& ci);
// Same pattern, other dtype; values converted on the device.
void bsr_convert(Bsr& dst, const Bsr& src, int dt, cudaStream_t s);
// FP64 copy (same pattern) of a matrix stored in any precision.
void bsr_widen(Bsr& dst, const Bsr& src, cudaStream_t s);
// Explicit block transpose (pattern by counting sort on the host, values on the device).
void bsr_transpose(Bsr& dst, const Bsr& src, cudaStream_t s);
// Host copy of FP64 values (unpadded, nnzb*d*d).
std::vector<double> bsr_values_host(const Bsr& m, cudaStream_t s);

// Symbolic product pattern of X (nx rows) times Y: sorted unique columns per row.
void pattern_product(const std::vector<int>& xrp, const std::vector<int>& xci, const std::vector<int>& yrp,
                     const std::vector<int>& yci, int n_rows, std::vector<int>& crp, std::vector<int>& cci);
// Numeric C = X Y on C's (given) pattern, FP64.
void spgemm_numeric(Bsr& C, const Bsr& X, const Bsr& Y, cudaStream_t s);
// C = X Y with pattern computed here (FP64).
void spgemm(Bsr& C, const Bsr& X, const Bsr& Y, cudaStream_t s);

// ----------------------------------------------------------------------------- hierarchy

struct Level {
  int m = 0, n = 0, d = 0;
  int vdt = PUM_F64, gdt = PUM_F64;  // this level's smoother storage/arithmetic and G precision
  Bsr A;                // FP64 operator
  Bsr As;               // smoothing copy (F32) when smooth_dt == F32
  Bsr P, PT;            // FP64 prolongation from level+1 and its transpose
  Bsr Ps, PTs;          // smoothing copies
  Bsr G, GT;            // FSAI factor (non-nested) in g_dt
  Bsr G64;              // FP64 G (kept for export)
  Bsr F0, F0T;          // nested: outer F (in g_dt) and its transpose
  Bsr F064, G164, A1;   // nested FP64 products kept for export
  Bsr G1, G1T;          // nested: inner G
  double beta = 0.0;
  double logdet_S = 0.0;
  double flops_adapt = 0.0, flops_factor = 0.0;  // FP64 flops of this level's set-up kernels
  int learned = 0;      // adaptive = 2: the level kept the learned pattern
  double gate = -1.0;   // adaptive = 2: the gate's shortfall (-1: not scored by the model)
  int nested_inner = 0;  // nested level: 1 inner FSAI of A1, 0 inner block Jacobi
  // work vectors in the smoothing precision
  void *x = nullptr, *b = nullptr, *r = nullptr, *p = nullptr, *t = nullptr, *u = nullptr;
  void *c = nullptr, *e = nullptr;  // correction-form post-smoothing: rhs c = b - A x, iterate e
  double *b64 = nullptr, *z64 = nullptr;  // FP64 right-hand side and iterate of a mixed level
  // Mixed level on the sliced layout: A as FP32 pairs (hi + lo) for the accurate residuals, and
  // the split (hi, lo) shadow of the level's FP64 iterate that those products read.
  Sell Adf;
  void* zs = nullptr;
  Sell Pdf;  // P as FP32 pairs, when the coarser level is a mixed sliced level too
  FusedG gg;  // G (or nested G1) read once per application, on sliced FP32 levels
};

struct Coarse {
  int N = 0;
  double* L = nullptr;  // dense lower Cholesky factor, row-major N x N
};

// The V-cycle of a set-up hierarchy captured once as a CUDA graph and replayed.  When it
// is captured with kernel timing on, the graph holds its own event pairs around every
// finest-level kernel; their times are collected after each replay has completed.
struct TimedEvent {
  int tk;
  cudaEvent_t start, stop;
};
struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;  // kernel launches per replay
  int timed = 0;  // timing mask the graph was captured with
  bool pending = false;  // a timed replay whose events have not been collected
  std::vector<TimedEvent> ev;
  const double* r = nullptr;  // vectors the graph was captured for
  double* z = nullptr;
};
void graph_destroy(GraphCache& g);
// Work blocks and the captured cycle of the multi-right-hand-side path (multi.cu).
struct MultiCache;
void multi_cache_free(MultiCache*& c);

}  // namespace pum

struct pum_hier {
  std::vector<pum::Level> lv;
  pum::Coarse coarse;
  bool setup_done = false;
  bfsai_params fp{};
  smoother_params sp{};
  int smooth_dt = PUM_F64;
  int g_dt = PUM_F64;
  std::vector<double> mu;  // Chebyshev mu_i, i = 1..k
  // FP64 work vectors of the finest level (PCG, conversions)
  double* w64[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // more of them for BiCGStab and the convergence factor, allocated on first use
  double* wb[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  pum::GraphCache vgraph;  // captured V-cycle
  pum::MultiCache* multi = nullptr;  // multi-RHS work blocks and cycle graph (built on first use)
  bool sell = true;        // sliced layouts for the large levels' FP32 products
  bool fused_fsai = true;  // G read once per FSAI application on those levels
};

struct pum_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string last_error;
  pum::DevStatus* status = nullptr;  // device
  double* scal = nullptr;            // device scalars (PCG)
  double* partials = nullptr;        // device reduction partials
  double* h_scal = nullptr;          // pinned host mirror of scal
  int64_t launches = 0;
  int sm_count = 152;
  int timing = 0;  // bitmask of timed kernel classes (1 << PUM_TK_*)
  cudaEvent_t ev_pool[2][PUM_TK_COUNT];
  std::vector<cudaEvent_t> tk_start[PUM_TK_COUNT], tk_stop[PUM_TK_COUNT];
  int64_t tk_launches[PUM_TK_COUNT] = {};  // launches timed since the last reset (collected)
  double tk_ms[PUM_TK_COUNT] = {};         // their summed event time
  int64_t tk_pool_used[PUM_TK_COUNT] = {}; // event pairs of direct launches not yet collected
  std::vector<pum::TimedEvent>* capture_ev = nullptr;  // set while a graph is being captured
  bool graphs = true;                                   // capture the V-cycle when the stream allows it
  bool sell = true;                                     // sliced layouts on large levels
  bool pdl = true;                                      // programmatic dependent launch of the cycle's kernels
  bool fused_fsai = true;                               // G read once per FSAI application on sliced levels
  bool adapt_steps = false;                             // Algorithm 1 step by step (one launch per step)
  pum_mlp* model = nullptr;                             // candidate-scoring network (adaptive = 2)
};

namespace pum {

constexpr int kMaxPartials = 1 << 16;
constexpr int kScalSlots = 32;

// ----------------------------------------------------------------------------- kernels

// Epilogues of the block-row product acc = (M x)_row.
enum Epi { EPI_SET = 0, EPI_RESID = 1, EPI_ADD = 2, EPI_CHEB_FIRST0 = 3, EPI_CHEB_FIRST = 4, EPI_CHEB = 5,
           EPI_DOT = 6 };

struct EpiArgs {
  void* y = nullptr;         // output (SET/RESID/ADD/DOT) or p (CHEB*)
  const void* b = nullptr;   // RESID: right-hand side (same type as the input vector x)
  void* xo = nullptr;        // CHEB*: iterate updated in place (same type as y)
  double mu2 = 0.0;          // CHEB: p <- mu2 p + acc
  double dmu = 0.0;          // CHEB*: x <- x + dmu p
  void* xo2 = nullptr;       // CHEB*: optional second iterate updated the same way (x2 <- x2 + dmu p)
  bool x2_set = false;       // CHEB_FIRST0: x2 <- dmu p instead of x2 += dmu p
  double* partials = nullptr;  // DOT: per-CTA partial sums of acc * x
  int xdt = -1, ydt = -1, x2dt = -1;  // vector dtypes when they differ from the call's vdt
  void* x2s = nullptr;  // CHEB*: float2 (hi, lo) split shadow of the FP64 second iterate, written with it
  void* ys = nullptr;   // ADD into an FP64 y: float2 split shadow of y, written with it
};

// y (by epilogue) = M x for a BSR matrix; vector dtype vdt (F64 or F32).
void bsr_mv(pum_ctx* ctx, const Bsr& M, int vdt, const void* x, int epi, const EpiArgs& e, int tk = -1);
// z (by epilogue) = G^T (G r) through the fused layout (FP32 vectors); timing classes of its two kernels.
void gg_apply(pum_ctx* ctx, const FusedG& F, const void* r, int epi, const EpiArgs& e, int tk_g = -1, int tk_gt = -1);
void convert_vec(pum_ctx* ctx, void* dst, int ddt, const void* src, int sdt, int64_t n);
void zero_vec(pum_ctx* ctx, void* dst, int dt, int64_t n);

// Deterministic dot product: partials then single-CTA reduction into scal[slot].
void dot(pum_ctx* ctx, const double* a, const double* b, int64_t n, int slot);
void dot_to(pum_ctx* ctx, const double* a, const double* b, int64_t n, double* out);
void reduce_partials(pum_ctx* ctx, int n_partials, int slot);

// Assembly, transfers (assemble.cu)
void assemble_finest(pum_ctx* ctx, const pum_problem& pr, Level& L, double* b_dev);
void build_prolongation(pum_ctx* ctx, int m_f, int p, int q, Level& fine);

// FSAI set-up (fsai.cu)
void fsai_setup_level(pum_ctx* ctx, pum_hier* h, int l);
// Learned candidate scoring (learned.cu).  Candidate pools of P0 (ring 1, ring 2) with their
// features, on the device; logits of a model; FP64 per-row log det S_kk of a factor pass.
struct CandidateSet {
  int64_t n = 0;
  std::vector<int> rp, col;    // host: per-row offsets (n_rows + 1) and columns
  int* d_row = nullptr;        // device copies
  int* d_col = nullptr;
  float* d_x = nullptr;        // n x 12 features
};
void candidates_build(pum_ctx* ctx, const Bsr& A, const Bsr& G0, const std::vector<std::vector<int>>& P0, int m,
                      CandidateSet& cs);
void candidates_free(CandidateSet& cs);
void mlp_forward_dev(pum_ctx* ctx, const pum_mlp& m, const float* x, int64_t n, float* logits);
// Algorithm 1's final patterns for every block row, one CTA per row through all steps (adapt.cu);
// false when the block size has no instantiation.
// fp64_flops (may be null) accumulates the kernel's FP64 flops (2 per multiply-add).
// work_rows (may be null): only these rows run Algorithm 1; the others of `rows` keep P0.
// G (and F) not null: the kernel also forms the FSAI factors of the final patterns from its grown
// local factorisations (every row; work_rows must be null) and logdet receives sum log det S_kk.
bool adaptive_patterns_device(pum_ctx* ctx, const Bsr& A, const std::vector<std::vector<int>>& P0, int t_max,
                              double tau, double tie_rel, std::vector<std::vector<int>>& rows, double* fp64_flops,
                              const std::vector<int>* work_rows = nullptr, Bsr* G = nullptr, Bsr* F = nullptr,
                              double* logdet = nullptr);
void lanczos_level(pum_ctx* ctx, pum_hier* h, int l);
void coarse_factor(pum_ctx* ctx, pum_hier* h);

// Smoother / cycle (solve.cu)
void apply_M(pum_ctx* ctx, pum_hier* h, int l, const void* r, void* z, int tk_first);
void cheb4(pum_ctx* ctx, pum_hier* h, int l, const void* rhs, void* x, bool x_zero, void* x_acc, int acc_dt,
           bool acc_set, void* x_acc_split = nullptr, int steps = 0);
void vcycle_level(pum_ctx* ctx, pum_hier* h, int l);
void coarse_solve(pum_ctx* ctx, pum_hier* h, const void* b, void* x, int vdt);

inline void count_launch(pum_ctx* ctx) { ctx->launches++; }

// Raise a kernel's dynamic shared memory limit to the most the device allows it (the opt-in
// limit less its static shared memory).  Always the same value for a kernel, so threads that
// launch it concurrently with different sizes cannot lower the limit under one another.
inline void allow_max_dynamic_smem(const void* kern) {
  int dev = 0, optin = 0;
  PUM_CUDA(cudaGetDevice(&dev));
  PUM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa{};
  PUM_CUDA(cudaFuncGetAttributes(&fa, kern));
  PUM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
}

// Launch a kernel of the V-cycle on the context's stream, with programmatic stream serialization
// when enabled (the kernel must call pdl_wait() before touching dependent memory).
template <typename... KArgs, typename... Args>
void launch_cycle_kernel(pum_ctx* ctx, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = ctx->pdl ? 1 : 0;
  PUM_CUDA(cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...));
}
void timing_begin(pum_ctx* ctx, int tk);
void timing_end(pum_ctx* ctx, int tk);
// Collect the kernel times of the last timed graph replay (waits for it).
void graph_harvest(pum_ctx* ctx, pum_hier* h);

}  // namespace pum
