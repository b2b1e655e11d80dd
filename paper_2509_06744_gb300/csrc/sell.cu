// Sliced block layout for the smoother's products on large levels, streamed through shared
// memory by bulk asynchronous copies.
//
// Layout: block rows are grouped by R; group g stores S_g slots (S_g = its longest block row),
// and slot s of row j holds that row's s-th block (padding: column -1, zero values).  The values
// of one (group, slot) form a contiguous chunk of d x (R d) values ordered (block column c,
// output unknown j d + r), so one cp.async.bulk moves a chunk into shared memory, where the
// thread of output unknown t reads element c (R d) + t: conflict-free.
//
// Kernel: warp 0 is the producer.  Its lane 0 streams the group's chunks into a ring of NS
// shared-memory stages; stage k is guarded by full[k] (completes when the chunk's bytes have
// landed) and empty[k] (one arrival per consumer warp once the chunk has been read).  The other
// warps are consumers: the thread of output unknown j d + r accumulates
// sum_c A_j[r][c] x[col d + c] over the slots, loading the next slot's x segment while the
// current chunk lands.  The bytes in flight per SM are then set by shared memory, not by
// registers.  Every wait is bounded: on expiry the kernel records PUM_ERR_TIMEOUT in the
// context's status word, drains its own copies (bounded) and returns.  The chunks are copied with
// an evict-first L2 policy: each is read once per product, and the vectors the next kernels
// read should stay in L2 instead.  Padding slots read
// column 0 against zero values, which keeps the loop branch-free.  The fused epilogues are those
// of the block-row kernel.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "bulk.cuh"
#include "kernels_common.cuh"

namespace pum {

namespace {

constexpr int kHeader = 128;         // bytes for the full/empty barriers of up to 8 stages
constexpr int kMaxStages = 8;
constexpr int kSellMaxThreads = 32 + 352;  // producer warp + the largest consumer group (d = 21, R = 16)

}  // namespace

// Largest group size R for block size d (bounded by the CTA size and the chunk's shared memory).
int sell_rows_max(int d) { return d <= 3 ? 64 : d <= 10 ? 32 : 16; }

// x[c * D .. c * D + D) of a split vector (float2 per unknown).
template <int D>
__device__ __forceinline__ void load_row_df(const float2* __restrict__ p, float2 (&out)[D]) {
  if constexpr ((D % 2) == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < D / 2; ++i) {
      const float4 v = __ldg(q + i);
      out[2 * i] = make_float2(v.x, v.y);
      out[2 * i + 1] = make_float2(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i) out[i] = __ldg(p + i);
  }
}

// s += a x in double-float: a = (ah, al), x = (xh, xl).  ah xh = p + e exactly (FMA); the
// cross terms and e go to the FP32 tail c; p joins the (sh, sl) pair by Knuth's two-sum.
__device__ __forceinline__ void df_fma(float2 a, float2 x, float& sh, float& sl, float& c) {
  const float p = a.x * x.x;
  const float e = fmaf(a.x, x.x, -p);
  c = fmaf(a.x, x.y, c);
  c = fmaf(a.y, x.x, c);
  c += e;
  const float s = sh + p;
  const float bp = s - sh;
  sl += (sh - (s - bp)) + (p - bp);
  sh = s;
}

template <int D, typename MT, typename XT, typename YT, typename X2T, int EPI>
__global__ void __launch_bounds__(kSellMaxThreads) k_sell_mv(int n_brows, int R, int NS, const int* __restrict__ goff,
                                                             const int* __restrict__ cols, const MT* __restrict__ vals,
                                                             const XT* __restrict__ x, EpiArgs e, DevStatus* st) {
  constexpr bool kDF = std::is_same<MT, float2>::value;  // double-float values and split x
  using AT = typename AccOf<MT>::type;
  using XV = typename std::conditional<kDF, float2, AT>::type;
  extern __shared__ __align__(128) unsigned char smem[];
  const int RD = R * D;
  const int chunk_elems = D * RD;
  const uint32_t chunk = (uint32_t)(chunk_elems * (int)sizeof(MT));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + kMaxStages;
  MT* stage = reinterpret_cast<MT*>(smem + kHeader);
  int* scol = reinterpret_cast<int*>(smem + kHeader + (size_t)NS * chunk);
  const int g = blockIdx.x;
  const int s0 = goff[g], ns = goff[g + 1] - s0;
  const int n_consumer_warps = (int)(blockDim.x >> 5) - 1;
  const MT* src = vals + (int64_t)s0 * chunk_elems;

  if (threadIdx.x == 0) {
    for (int k = 0; k < NS; ++k) {
      mbar_init(full + k, 1);
      mbar_init(empty + k, (uint32_t)n_consumer_warps);
    }
    mbar_fence_init();
    const uint64_t pol = l2_evict_first_policy();
    for (int s = 0; s < min(NS, ns); ++s) {
      mbar_expect_tx(full + s, chunk);
      bulk_g2s_policy(stage + (size_t)s * chunk_elems, src + (int64_t)s * chunk_elems, chunk, full + s, pol);
    }
  }
  for (int i = threadIdx.x; i < ns * R; i += blockDim.x) scol[i] = max(__ldg(cols + (int64_t)s0 * R + i), 0);
  __syncthreads();

  if (threadIdx.x < 32) {  // producer warp
    if (threadIdx.x != 0) return;
    bool ok = true;
    int issued = min(NS, ns);
    const uint64_t pol = l2_evict_first_policy();
    for (int s = NS; s < ns; ++s) {
      const int k = s % NS;
      if (!mbar_wait(empty + k, (uint32_t)((s / NS) - 1) & 1u)) {
        ok = false;
        break;
      }
      mbar_expect_tx(full + k, chunk);
      bulk_g2s_policy(stage + (size_t)k * chunk_elems, src + (int64_t)s * chunk_elems, chunk, full + k, pol);
      issued = s + 1;
    }
    for (int s = max(issued - NS, 0); s < issued; ++s)  // own copies still in flight
      if (!mbar_wait(full + s % NS, (uint32_t)(s / NS) & 1u)) ok = false;
    if (!ok) set_status(st, PUM_ERR_TIMEOUT, g, kWhereSell);
    return;
  }

  const int t = (int)threadIdx.x - 32;
  const bool computes = t < RD;
  const int j = computes ? t / D : 0;
  const int r = t - j * D;
  AT acc = 0;
  float sh = 0.f, sl = 0.f, sc = 0.f;  // double-float accumulator (kDF)
  XV xn[D];
  pdl_wait();  // x and the epilogue's vectors come from the preceding kernel (the matrix does not)
  if constexpr (kEarlyTrigger<D>) pdl_release();  // the next kernel may launch and issue its pre-wait loads
  auto load_x = [&](int c, XV(&out)[D]) {
    if constexpr (kDF)
      load_row_df<D>(reinterpret_cast<const float2*>(x) + (int64_t)c * D, out);
    else
      load_row<D>(x + (int64_t)c * D, out);
  };
  if (computes && ns > 0) load_x(scol[j], xn);
  for (int s = 0; s < ns; ++s) {
    const int k = s % NS;
    XV xv[D];
#pragma unroll
    for (int cc = 0; cc < D; ++cc) xv[cc] = xn[cc];
    if (computes && s + 1 < ns) load_x(scol[(s + 1) * R + j], xn);
    if (!__all_sync(0xffffffffu, mbar_wait(full + k, (uint32_t)(s / NS) & 1u))) {
      if ((threadIdx.x & 31) == 0) set_status(st, PUM_ERR_TIMEOUT, g, kWhereSell);
      return;
    }
    if (computes) {
      const MT* a = stage + (size_t)k * chunk_elems + t;
      if constexpr (kDF) {
#pragma unroll
        for (int cc = 0; cc < D; ++cc) df_fma(a[cc * RD], xv[cc], sh, sl, sc);
      } else {
#pragma unroll
        for (int cc = 0; cc < D; ++cc) acc = fma((AT)to_f(a[cc * RD]), xv[cc], acc);
      }
    }
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(empty + k);
  }
  if constexpr (!kEarlyTrigger<D>) pdl_release();
  const int row = g * R + j;
  if (!(computes && row < n_brows)) return;
  if constexpr (kDF) {
    acc = (double)sh + ((double)sl + (double)sc);
    epilogue<EPI, double, double, YT, double>(e, (int64_t)row * D + r, acc);  // b and y in FP64
  } else {
    epilogue<EPI, AT, XT, YT, X2T>(e, (int64_t)row * D + r, acc);
  }
}

// Ring depth: as many stages as fit in about 40 KB, between 2 and 8 (small chunks of small
// groups need more of them in flight per CTA).
static int sell_stages(size_t chunk) { return (int)std::max<size_t>(2, std::min<size_t>(kMaxStages, 40960 / chunk)); }

static size_t sell_smem(const Sell& S, int d, size_t vsize) {
  const size_t chunk = vsize * (size_t)d * S.R * d;
  return kHeader + (size_t)sell_stages(chunk) * chunk + sizeof(int) * (size_t)S.max_slots * S.R;
}

template <int D, typename MT, typename XT, typename YT, typename X2T>
static void sell_launch(pum_ctx* ctx, const Sell& S, int n_brows, const void* x, int epi, const EpiArgs& e) {
  if (S.n_groups == 0) return;
  const int RD = S.R * D;
  const unsigned threads = 32u + (unsigned)((RD + 31) / 32) * 32u;
  const size_t chunk = sizeof(MT) * (size_t)D * RD;
  const int NS = sell_stages(chunk);
  const size_t smem = sell_smem(S, D, sizeof(MT));
  const MT* v = (const MT*)S.vals;
  const XT* xv = (const XT*)x;
  switch (epi) {
#define PUM_SELL_CASE(E)                                                                                    \
  case E: {                                                                                                 \
    auto kern = k_sell_mv<D, MT, XT, YT, X2T, E>;                                                           \
    if (smem > 48 * 1024)                                                                                   \
      allow_max_dynamic_smem((const void*)kern);                                                           \
    launch_cycle_kernel(ctx, kern, dim3(S.n_groups), dim3(threads), smem, n_brows, S.R, NS, S.goff, S.cols, v, \
                        xv, e, ctx->status);                                                                \
    break;                                                                                                  \
  }
    PUM_SELL_CASE(EPI_SET)
    PUM_SELL_CASE(EPI_RESID)
    PUM_SELL_CASE(EPI_ADD)
    PUM_SELL_CASE(EPI_CHEB_FIRST0)
    PUM_SELL_CASE(EPI_CHEB_FIRST)
    PUM_SELL_CASE(EPI_CHEB)
#undef PUM_SELL_CASE
    default:
      throw Error{PUM_ERR_UNSUPPORTED, "sliced product: unsupported epilogue"};
  }
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
}

template <int D>
static bool sell_mv_d(pum_ctx* ctx, const Bsr& M, int vdt, const void* x, int epi, const EpiArgs& e) {
  const int xdt = e.xdt >= 0 ? e.xdt : vdt;
  const int ydt = e.ydt >= 0 ? e.ydt : vdt;
  const int x2dt = (e.xo2 && e.x2dt >= 0) ? e.x2dt : ydt;
  const int mdt = M.dt;
  const Sell& S = M.sell;
  const int n = M.n_brows;
  if (mdt == PUM_F32 && xdt == PUM_F32 && ydt == PUM_F32 && x2dt == PUM_F32)
    return sell_launch<D, float, float, float, float>(ctx, S, n, x, epi, e), true;
  if (mdt == PUM_F32 && xdt == PUM_F32 && ydt == PUM_F32 && x2dt == PUM_F64)
    return sell_launch<D, float, float, float, double>(ctx, S, n, x, epi, e), true;
  if (mdt == PUM_BF16 && xdt == PUM_F32 && ydt == PUM_F32 && x2dt == PUM_F32)
    return sell_launch<D, __nv_bfloat16, float, float, float>(ctx, S, n, x, epi, e), true;
  if (mdt == PUM_BF16 && xdt == PUM_F32 && ydt == PUM_F32 && x2dt == PUM_F64)
    return sell_launch<D, __nv_bfloat16, float, float, double>(ctx, S, n, x, epi, e), true;
  if (mdt == PUM_F32 && xdt == PUM_F32 && ydt == PUM_F64 && epi == EPI_ADD)
    return sell_launch<D, float, float, double, double>(ctx, S, n, x, epi, e), true;
  return false;  // other precision mixes use the block-row kernel
}

bool sell_mv(pum_ctx* ctx, const Bsr& M, int vdt, const void* x, int epi, const EpiArgs& e) {
  if (!M.sell.R || epi == EPI_DOT) return false;
  switch (M.d) {
    case 3: return sell_mv_d<3>(ctx, M, vdt, x, epi, e);
    case 6: return sell_mv_d<6>(ctx, M, vdt, x, epi, e);
    case 10: return sell_mv_d<10>(ctx, M, vdt, x, epi, e);
    case 15: return sell_mv_d<15>(ctx, M, vdt, x, epi, e);
    case 21: return sell_mv_d<21>(ctx, M, vdt, x, epi, e);
    default: return false;
  }
}

template <int D>
static void sell_df_d(pum_ctx* ctx, const Sell& S, int n_brows, const void* xs, int epi, const EpiArgs& e) {
  if (epi == EPI_RESID) return sell_launch<D, float2, float2, float, double>(ctx, S, n_brows, xs, epi, e);
  if (epi == EPI_ADD) return sell_launch<D, float2, float2, double, double>(ctx, S, n_brows, xs, epi, e);
  throw Error{PUM_ERR_UNSUPPORTED, "double-float product: residual or add only"};
}

void sell_df_mv(pum_ctx* ctx, const Sell& S, int d, int n_brows, const void* xs, int epi, const EpiArgs& e, int tk) {
  PUM_CHECK(S.R > 0, PUM_ERR_UNSUPPORTED, "double-float product: layout not built");
  if (tk >= 0) timing_begin(ctx, tk);
  switch (d) {
    case 3: sell_df_d<3>(ctx, S, n_brows, xs, epi, e); break;
    case 6: sell_df_d<6>(ctx, S, n_brows, xs, epi, e); break;
    case 10: sell_df_d<10>(ctx, S, n_brows, xs, epi, e); break;
    case 15: sell_df_d<15>(ctx, S, n_brows, xs, epi, e); break;
    case 21: sell_df_d<21>(ctx, S, n_brows, xs, epi, e); break;
    default: throw Error{PUM_ERR_UNSUPPORTED, "double-float product: unsupported block size"};
  }
  if (tk >= 0) timing_end(ctx, tk);
}

// ----------------------------------------------------------------------------- build

// Value kinds of a sliced layout: FP32, BF16 (the matrix's own values) or double-float pairs of
// an FP64 matrix.
enum { kKindF32 = 0, kKindBF16 = 1, kKindDF = 2 };

static size_t kind_size(int kind) { return kind == kKindBF16 ? 2 : kind == kKindF32 ? 4 : 8; }

template <typename T, typename S>
__global__ void k_sell_fill(T* __restrict__ dst, const S* __restrict__ src, const int* __restrict__ src_blk, int stride,
                            int d, int R, int64_t slots) {
  const int dd = d * d;
  const int64_t total = slots * R * dd;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sj = i / dd;  // slot * R + j
    const int e = (int)(i - sj * dd);
    const int b = src_blk[sj];
    if (b < 0) continue;
    const int64_t slot = sj / R;
    const int j = (int)(sj - slot * R);
    const int r = e / d, c = e - (e / d) * d;
    const S v = src[(int64_t)b * stride + r * d + c];
    T* at = dst + (slot * d + c) * (int64_t)(R * d) + j * d + r;
    if constexpr (std::is_same<T, float2>::value)
      *at = split_df((double)v);
    else
      *at = v;
  }
}

void sell_free(Sell& s) {
  if (s.goff) cudaFree(s.goff);
  if (s.cols) cudaFree(s.cols);
  if (s.vals) cudaFree(s.vals);
  s = Sell();
}

// Resident CTAs per SM of the kernel that bounds the layout's occupancy for group size R: the
// Chebyshev update for FP32/BF16 values, the residual for double-float values.
template <int D, typename MT>
static int sell_occupancy(int R, int max_slots) {
  Sell S;
  S.R = R;
  S.max_slots = max_slots;
  const int threads = 32 + ((R * D + 31) / 32) * 32;
  const size_t smem = sell_smem(S, D, sizeof(MT));
  const void* kern;
  if constexpr (std::is_same<MT, float2>::value)
    kern = (const void*)k_sell_mv<D, MT, float2, float, double, EPI_RESID>;
  else
    kern = (const void*)k_sell_mv<D, MT, float, float, double, EPI_CHEB>;
  if (smem > 48 * 1024) allow_max_dynamic_smem(kern);
  int nb = 0;
  PUM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem));
  return nb;
}

template <int D>
static int sell_occupancy_d(int kind, int R, int max_slots) {
  if (kind == kKindBF16) return sell_occupancy<D, __nv_bfloat16>(R, max_slots);
  if (kind == kKindDF) return sell_occupancy<D, float2>(R, max_slots);
  return sell_occupancy<D, float>(R, max_slots);
}

static int sell_occupancy_for(int d, int kind, int R, int max_slots) {
  switch (d) {
    case 3: return sell_occupancy_d<3>(kind, R, max_slots);
    case 6: return sell_occupancy_d<6>(kind, R, max_slots);
    case 10: return sell_occupancy_d<10>(kind, R, max_slots);
    case 15: return sell_occupancy_d<15>(kind, R, max_slots);
    case 21: return sell_occupancy_d<21>(kind, R, max_slots);
    default: throw Error{PUM_ERR_UNSUPPORTED, "sliced layout: unsupported block size"};
  }
}

// Group size R: one CTA per group, so the product runs in ceil(groups / (CTAs per SM x SMs))
// waves of equal CTAs.  Among the R in [8, sell_rows_max(d)] whose slot chunk R d^2 values is a
// multiple of 16 bytes, take the one whose last wave is fullest (waves / ceil(waves)), the
// largest R among those within 1% of the best.
static int sell_choose_rows(const Bsr& M, int kind, int sm_count) {
  const int n = M.n_brows, d = M.d;
  const size_t vsize = kind_size(kind);
  int max_row = 0;
  for (int i = 0; i < n; ++i) max_row = std::max(max_row, M.h_row_ptr[i + 1] - M.h_row_ptr[i]);
  int best_r = 0;
  double best = -1.0;
  for (int R = sell_rows_max(d); R >= 8; --R) {
    if ((vsize * (size_t)d * R * d) % 16 != 0) continue;
    const int occ = sell_occupancy_for(d, kind, R, max_row);
    if (occ <= 0) continue;
    const double waves = (double)((n + R - 1) / R) / ((double)occ * sm_count);
    const double eff = waves / std::ceil(waves);
    if (eff > best + 0.01) {
      best = eff;
      best_r = R;
    }
  }
  PUM_CHECK(best_r > 0, PUM_ERR_UNSUPPORTED, "sliced layout: no admissible group size");
  return best_r;
}

// Sliced layout of M with value kind `kind`; group size R_fixed, or (0) chosen for the product kernel.
static void sell_build_kind(Sell& S, const Bsr& M, int kind, cudaStream_t st, int sm_count, int R_fixed = 0) {
  sell_free(S);
  const int d = M.d;
  if (!(d == 3 || d == 6 || d == 10 || d == 15 || d == 21)) return;
  const int n = M.n_brows;
  const int R = R_fixed > 0 ? R_fixed : sell_choose_rows(M, kind, sm_count);
  const int ng = (n + R - 1) / R;
  std::vector<int> goff(ng + 1, 0);
  for (int g = 0; g < ng; ++g) {
    int smax = 0;
    for (int j = 0; j < R && g * R + j < n; ++j) smax = std::max(smax, M.h_row_ptr[g * R + j + 1] - M.h_row_ptr[g * R + j]);
    goff[g + 1] = goff[g] + smax;
  }
  const int64_t slots = goff[ng];
  std::vector<int> cols((size_t)slots * R, -1), src((size_t)slots * R, -1);
  for (int g = 0; g < ng; ++g)
    for (int j = 0; j < R && g * R + j < n; ++j) {
      const int row = g * R + j;
      for (int q = 0; q < M.h_row_ptr[row + 1] - M.h_row_ptr[row]; ++q) {
        const size_t at = (size_t)(goff[g] + q) * R + j;
        cols[at] = M.h_col_idx[M.h_row_ptr[row] + q];
        src[at] = M.h_row_ptr[row] + q;
      }
    }
  S.R = R;
  S.n_groups = ng;
  S.slots = slots;
  S.max_slots = 0;
  for (int g = 0; g < ng; ++g) S.max_slots = std::max(S.max_slots, goff[g + 1] - goff[g]);
  const size_t vsize = kind_size(kind);
  PUM_CHECK((vsize * (size_t)d * R * d) % 16 == 0, PUM_ERR_UNSUPPORTED, "sliced layout: chunk not 16-byte sized");
  PUM_CHECK(sell_smem(S, d, vsize) <= 200 * 1024, PUM_ERR_UNSUPPORTED, "sliced layout: row too long");
  S.R = 0;  // set again once the device arrays exist
  const size_t vbytes = vsize * (size_t)std::max<int64_t>(slots, 1) * R * d * d;
  if (cudaMalloc(&S.goff, sizeof(int) * goff.size()) != cudaSuccess ||
      cudaMalloc(&S.cols, sizeof(int) * std::max<size_t>(cols.size(), 1)) != cudaSuccess ||
      cudaMalloc(&S.vals, vbytes) != cudaSuccess) {
    cudaGetLastError();
    sell_free(S);
    throw Error{PUM_ERR_OOM, "sliced layout: device allocation failed"};
  }
  int* dsrc = nullptr;
  PUM_CUDA(cudaMalloc(&dsrc, sizeof(int) * std::max<size_t>(src.size(), 1)));
  PUM_CUDA(cudaMemcpyAsync(S.goff, goff.data(), sizeof(int) * goff.size(), cudaMemcpyHostToDevice, st));
  if (!cols.empty()) {
    PUM_CUDA(cudaMemcpyAsync(S.cols, cols.data(), sizeof(int) * cols.size(), cudaMemcpyHostToDevice, st));
    PUM_CUDA(cudaMemcpyAsync(dsrc, src.data(), sizeof(int) * src.size(), cudaMemcpyHostToDevice, st));
  }
  PUM_CUDA(cudaMemsetAsync(S.vals, 0, vbytes, st));
  const int64_t total = slots * R * d * d;
  const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
  if (total) {
    if (kind == kKindF32)
      k_sell_fill<<<grid, 256, 0, st>>>((float*)S.vals, (const float*)M.vals, dsrc, M.stride, d, R, slots);
    else if (kind == kKindBF16)
      k_sell_fill<<<grid, 256, 0, st>>>((__nv_bfloat16*)S.vals, (const __nv_bfloat16*)M.vals, dsrc, M.stride, d, R,
                                        slots);
    else
      k_sell_fill<<<grid, 256, 0, st>>>((float2*)S.vals, (const double*)M.vals, dsrc, M.stride, d, R, slots);
    PUM_CUDA(cudaGetLastError());
  }
  PUM_CUDA(cudaStreamSynchronize(st));
  cudaFree(dsrc);
  S.R = R;
}

void sell_build(Bsr& M, cudaStream_t st, int sm_count) {
  if (M.dt == PUM_F64) {
    sell_free(M.sell);
    return;
  }
  sell_build_kind(M.sell, M, M.dt == PUM_BF16 ? kKindBF16 : kKindF32, st, sm_count);
}

void sell_build_rows(Sell& S, const Bsr& M, int R, cudaStream_t st) {
  PUM_CHECK(M.dt == PUM_F32 || M.dt == PUM_BF16, PUM_ERR_UNSUPPORTED, "sliced layout: FP32 or BF16 values");
  PUM_CHECK(R > 0, PUM_ERR_INVALID_ARG, "sliced layout: group size");
  sell_build_kind(S, M, M.dt == PUM_BF16 ? kKindBF16 : kKindF32, st, 0, R);
}

void sell_build_df(Sell& S, const Bsr& M64, cudaStream_t st, int sm_count) {
  PUM_CHECK(M64.dt == PUM_F64, PUM_ERR_UNSUPPORTED, "double-float layout: needs an FP64 matrix");
  sell_build_kind(S, M64, kKindDF, st, sm_count);
}

}  // namespace pum
