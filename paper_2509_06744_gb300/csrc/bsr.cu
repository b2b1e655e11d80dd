// Block-sparse kernels: y = M x with fused epilogues (residual, Chebyshev-4 update of
// Algorithm 3, PCG dot product), precision conversions, explicit block transposes,
// block SpGEMM for Galerkin and nested-FSAI triple products, deterministic dots.
#include <algorithm>
#include <cstring>

#include "kernels_common.cuh"

namespace pum {

// ----------------------------------------------------------------------------- helpers


// ----------------------------------------------------------------------------- y = M x

// G lanes per output unknown (block row `row`, local index r): lane g handles the blocks
// b0 + g, b0 + g + G, ... of the block row and the G partial sums are combined with
// warp shuffles.  The D x G lanes of a block row read the D rows of each d x d block
// (contiguous: a block row's blocks are one contiguous stream) and the D values of x of
// the block column.  G = 1 on fine levels (enough rows to fill the GPU); coarse levels,
// with few rows and up to 25 blocks per row, use G up to 32 so that each lane walks only
// one or two blocks instead of a 25-long chain of dependent loads.
template <int D, typename MT, typename XT, typename YT, typename X2T, int EPI>
__global__ void __launch_bounds__(256) k_bsr_mv(int n_brows, int stride, int lanes, const int* __restrict__ rp,
                                                const int* __restrict__ ci, const MT* __restrict__ vals,
                                                const XT* __restrict__ x, EpiArgs e) {
  using AT = typename AccOf<MT>::type;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tid = gtid / lanes;  // output unknown
  const int g = (int)(gtid - tid * lanes);
  const int row = (int)(tid / D);
  const int r = (int)(tid - (int64_t)row * D);
  const bool active = row < n_brows;
  AT acc = 0;
  if constexpr (kEarlyTrigger<D>) {
    // The matrix does not change while products run (no kernel that writes one triggers its
    // dependents early), so the row's extent and this lane's first block (its column and matrix
    // row) are loaded before waiting for the preceding kernel: on the small coarse levels, where
    // each lane has one or two blocks, that takes two of the three dependent loads off the chain.
    int b = 0, b1 = 0, c = 0;
    AT a[D];
    if (active) {
      b = __ldg(rp + row) + g;
      b1 = __ldg(rp + row + 1);
      if (b < b1) {
        c = __ldg(ci + b);
        load_row<D>(vals + (int64_t)b * stride + r * D, a);
      }
    }
    pdl_wait();
    pdl_release();  // the next kernel may launch and issue its own pre-wait loads
    while (b < b1) {
      AT xv[D];
      load_row<D>(x + (int64_t)c * D, xv);
#pragma unroll
      for (int q = 0; q < D; ++q) acc = fma(a[q], xv[q], acc);
      b += lanes;
      if (b < b1) {
        c = __ldg(ci + b);
        load_row<D>(vals + (int64_t)b * stride + r * D, a);
      }
    }
  } else {
    pdl_wait();
    if (active) {
      const int b1 = rp[row + 1];
      for (int b = rp[row] + g; b < b1; b += lanes) {
        const int c = __ldg(ci + b);
        AT a[D], xv[D];
        load_row<D>(vals + (int64_t)b * stride + r * D, a);
        load_row<D>(x + (int64_t)c * D, xv);
#pragma unroll
        for (int q = 0; q < D; ++q) acc = fma(a[q], xv[q], acc);
      }
    }
    pdl_release();
  }
  for (int o = lanes >> 1; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, lanes);
  const bool leader = active && g == 0;
  if constexpr (EPI == EPI_DOT) {
    __shared__ double red[256 / 32];
    double contrib = 0.0;
    if (leader) {
      ((YT*)e.y)[tid] = (YT)acc;
      contrib = (double)acc * (double)x[tid];
    }
    for (int o = 16; o > 0; o >>= 1) contrib += __shfl_down_sync(0xffffffffu, contrib, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = contrib;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      e.partials[blockIdx.x] = s;
    }
    return;
  }
  if (!leader) return;
  epilogue<EPI, AT, XT, YT, X2T>(e, tid, acc);
}

// Epilogue sets a type combination is instantiated for.
constexpr unsigned kAllEpi = 0x7Fu;
constexpr unsigned kResidOnly = 1u << EPI_RESID;
constexpr unsigned kAddOnly = 1u << EPI_ADD;
constexpr unsigned kSetOnly = 1u << EPI_SET;
constexpr unsigned kChebOnly = (1u << EPI_CHEB_FIRST0) | (1u << EPI_CHEB_FIRST) | (1u << EPI_CHEB);

template <int D, typename MT, typename XT, typename YT, typename X2T, unsigned EPIS>
static void launch_mv_epi(pum_ctx* ctx, const Bsr& M, const void* x, int epi, const EpiArgs& e) {
  // lanes per output: double while the GPU is not filled (about sm_count x 2048 resident
  // threads) and a row still has blocks for the extra lane; the DOT epilogue's per-CTA
  // partials assume one lane per output.
  int lanes = 1;
  if (epi != EPI_DOT)
    while (lanes < 32 && (int64_t)M.n_brows * D * lanes < (int64_t)ctx->sm_count * 2048 && lanes < M.max_row_nnzb)
      lanes *= 2;
  const int64_t nthreads = (int64_t)M.n_brows * D * lanes;
  const int bs = 256;
  const unsigned grid = (unsigned)((nthreads + bs - 1) / bs);
  if (grid == 0) return;
  auto* v = (const MT*)M.vals;
  auto* xv = (const XT*)x;
  cudaStream_t s = ctx->stream;
  PUM_CHECK((EPIS >> epi) & 1u, PUM_ERR_UNSUPPORTED, "bsr_mv: epilogue not available for this precision mix");
#define PUM_MV_CASE(E)                                                                                            \
  case E:                                                                                                         \
    if constexpr ((EPIS >> E) & 1u)                                                                               \
      launch_cycle_kernel(ctx, k_bsr_mv<D, MT, XT, YT, X2T, E>, dim3(grid), dim3(bs), 0, M.n_brows, M.stride, lanes, \
                          M.row_ptr, M.col_idx, v, xv, e);                                                        \
    break;
  switch (epi) {
    PUM_MV_CASE(EPI_SET)
    PUM_MV_CASE(EPI_RESID)
    PUM_MV_CASE(EPI_ADD)
    PUM_MV_CASE(EPI_CHEB_FIRST0)
    PUM_MV_CASE(EPI_CHEB_FIRST)
    PUM_MV_CASE(EPI_CHEB)
    case EPI_DOT:
      if constexpr (std::is_same<MT, double>::value && std::is_same<XT, double>::value &&
                    std::is_same<YT, double>::value && ((EPIS >> EPI_DOT) & 1u)) {
        PUM_CHECK(grid <= (unsigned)(1 << 16), PUM_ERR_UNSUPPORTED, "dot epilogue: too many blocks");
        k_bsr_mv<D, MT, XT, YT, X2T, EPI_DOT><<<grid, bs, 0, s>>>(M.n_brows, M.stride, 1, M.row_ptr, M.col_idx, v,
                                                                 xv, e);
      } else {
        throw Error{PUM_ERR_UNSUPPORTED, "dot epilogue needs float64"};
      }
      break;
    default:
      throw Error{PUM_ERR_INVALID_ARG, "unknown epilogue"};
  }
#undef PUM_MV_CASE
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
}

template <int D>
static void launch_mv_d(pum_ctx* ctx, const Bsr& M, int vdt, const void* x, int epi, const EpiArgs& e) {
  const int xdt = e.xdt >= 0 ? e.xdt : vdt;
  const int ydt = e.ydt >= 0 ? e.ydt : vdt;
  const int x2dt = (e.xo2 && e.x2dt >= 0) ? e.x2dt : ydt;
  const int mdt = M.dt;
  if (mdt == PUM_F64 && xdt == PUM_F64 && ydt == PUM_F64 && x2dt == PUM_F64)
    return launch_mv_epi<D, double, double, double, double, kAllEpi>(ctx, M, x, epi, e);
  if (mdt == PUM_F32 && xdt == PUM_F32 && ydt == PUM_F32 && x2dt == PUM_F32)
    return launch_mv_epi<D, float, float, float, float, kAllEpi & ~(1u << EPI_DOT)>(ctx, M, x, epi, e);
  if (mdt == PUM_BF16 && xdt == PUM_F32 && ydt == PUM_F32 && x2dt == PUM_F32)
    return launch_mv_epi<D, __nv_bfloat16, float, float, float, kAllEpi & ~(1u << EPI_DOT)>(ctx, M, x, epi, e);
  // FP32 smoother accumulating its updates into an FP64 iterate; FP32 restriction with an FP64
  // copy of its result
  if (mdt == PUM_F32 && xdt == PUM_F32 && ydt == PUM_F32 && x2dt == PUM_F64)
    return launch_mv_epi<D, float, float, float, double, kChebOnly | kSetOnly>(ctx, M, x, epi, e);
  if (mdt == PUM_BF16 && xdt == PUM_F32 && ydt == PUM_F32 && x2dt == PUM_F64)
    return launch_mv_epi<D, __nv_bfloat16, float, float, double, kChebOnly>(ctx, M, x, epi, e);
  // residuals with the FP64 operator and FP64 sums, FP32 result
  if (mdt == PUM_F64 && xdt == PUM_F32 && ydt == PUM_F32)
    return launch_mv_epi<D, double, float, float, float, kResidOnly>(ctx, M, x, epi, e);
  if (mdt == PUM_F64 && xdt == PUM_F64 && ydt == PUM_F32)
    return launch_mv_epi<D, double, double, float, float, kResidOnly>(ctx, M, x, epi, e);
  // FP32 prolongation added into an FP64 iterate
  if (mdt == PUM_F32 && xdt == PUM_F32 && ydt == PUM_F64)
    return launch_mv_epi<D, float, float, double, double, kAddOnly>(ctx, M, x, epi, e);
  // FP64 restriction of an FP32 residual to a level that smooths in FP64
  if (mdt == PUM_F64 && xdt == PUM_F32 && ydt == PUM_F64)
    return launch_mv_epi<D, double, float, double, double, kSetOnly>(ctx, M, x, epi, e);
  throw Error{PUM_ERR_UNSUPPORTED, "bsr_mv: unsupported matrix/vector precision mix"};
}

unsigned mv_grid_blocks(const Bsr& M) { return (unsigned)(((int64_t)M.n_brows * M.d + 255) / 256); }

void bsr_mv(pum_ctx* ctx, const Bsr& M, int vdt, const void* x, int epi, const EpiArgs& e, int tk) {
  if (tk >= 0) timing_begin(ctx, tk);
  if (sell_mv(ctx, M, vdt, x, epi, e)) {
    if (tk >= 0) timing_end(ctx, tk);
    return;
  }
  switch (M.d) {
    case 3: launch_mv_d<3>(ctx, M, vdt, x, epi, e); break;
    case 6: launch_mv_d<6>(ctx, M, vdt, x, epi, e); break;
    case 10: launch_mv_d<10>(ctx, M, vdt, x, epi, e); break;
    case 15: launch_mv_d<15>(ctx, M, vdt, x, epi, e); break;
    case 20: launch_mv_d<20>(ctx, M, vdt, x, epi, e); break;
    case 21: launch_mv_d<21>(ctx, M, vdt, x, epi, e); break;
    default: throw Error{PUM_ERR_UNSUPPORTED, "block size must be 3, 6, 10, 15, 21 (square) or 20 (cube)"};
  }
  if (tk >= 0) timing_end(ctx, tk);
}

// ----------------------------------------------------------------------------- vectors

template <typename D_, typename S_>
__global__ void k_convert(D_* __restrict__ d, const S_* __restrict__ s, int64_t n) {
  pdl_wait();
  pdl_release();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = (D_)s[i];
}

static unsigned elem_grid(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16); }

void convert_vec(pum_ctx* ctx, void* dst, int ddt, const void* src, int sdt, int64_t n) {
  if (n == 0) return;
  if (ddt == sdt) {
    PUM_CUDA(cudaMemcpyAsync(dst, src, n * dt_size(ddt), cudaMemcpyDeviceToDevice, ctx->stream));
    return;
  }
  if (ddt == PUM_F32 && sdt == PUM_F64)
    launch_cycle_kernel(ctx, k_convert<float, double>, dim3(elem_grid(n)), dim3(256), 0, (float*)dst,
                        (const double*)src, n);
  else if (ddt == PUM_F64 && sdt == PUM_F32)
    launch_cycle_kernel(ctx, k_convert<double, float>, dim3(elem_grid(n)), dim3(256), 0, (double*)dst,
                        (const float*)src, n);
  else
    throw Error{PUM_ERR_UNSUPPORTED, "convert_vec: dtype pair"};
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
}

void zero_vec(pum_ctx* ctx, void* dst, int dt, int64_t n) {
  if (n) PUM_CUDA(cudaMemsetAsync(dst, 0, n * dt_size(dt), ctx->stream));
}

// Deterministic dot: a fixed grid (function of n only) writes per-CTA partials, then one
// CTA sums them in a fixed order.
__global__ void k_dot_partials(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                               double* __restrict__ partials) {
  __shared__ double red[8];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partials[blockIdx.x] = t;
  }
}

__global__ void k_reduce_partials(const double* __restrict__ partials, int n, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = t;
  }
}

void reduce_partials(pum_ctx* ctx, int n_partials, int slot) {
  k_reduce_partials<<<1, 1024, 0, ctx->stream>>>(ctx->partials, n_partials, ctx->scal + slot);
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
}

void dot_to(pum_ctx* ctx, const double* a, const double* b, int64_t n, double* out) {
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 1024);
  if (grid == 0) {
    PUM_CUDA(cudaMemsetAsync(out, 0, sizeof(double), ctx->stream));
    return;
  }
  k_dot_partials<<<grid, 256, 0, ctx->stream>>>(a, b, n, ctx->partials);
  k_reduce_partials<<<1, 1024, 0, ctx->stream>>>(ctx->partials, grid, out);
  ctx->launches += 2;
  PUM_CUDA(cudaGetLastError());
}

void dot(pum_ctx* ctx, const double* a, const double* b, int64_t n, int slot) { dot_to(ctx, a, b, n, ctx->scal + slot); }

// ----------------------------------------------------------------------------- matrices

void bsr_free(Bsr& m) {
  sell_free(m.sell);
  if (m.row_ptr) cudaFree(m.row_ptr);
  if (m.col_idx) cudaFree(m.col_idx);
  if (m.vals) cudaFree(m.vals);
  m = Bsr();
}

void bsr_alloc(Bsr& m, int n_brows, int n_bcols, int d, int dt, const std::vector<int>& rp,
               const std::vector<int>& ci) {
  bsr_free(m);
  m.n_brows = n_brows;
  m.n_bcols = n_bcols;
  m.d = d;
  m.dt = dt;
  m.stride = block_stride(d, dt);
  m.nnzb = (int64_t)ci.size();
  m.h_row_ptr = rp;
  m.h_col_idx = ci;
  m.max_row_nnzb = 0;
  for (int i = 0; i < n_brows; ++i) m.max_row_nnzb = std::max(m.max_row_nnzb, rp[i + 1] - rp[i]);
  PUM_CHECK((int)rp.size() == n_brows + 1 && rp.back() == (int)ci.size(), PUM_ERR_INVALID_ARG, "bsr pattern");
  if (cudaMalloc(&m.row_ptr, sizeof(int) * rp.size()) != cudaSuccess ||
      cudaMalloc(&m.col_idx, sizeof(int) * std::max<size_t>(ci.size(), 1)) != cudaSuccess ||
      cudaMalloc(&m.vals, dt_size(dt) * (size_t)m.stride * std::max<int64_t>(m.nnzb, 1)) != cudaSuccess) {
    cudaGetLastError();
    bsr_free(m);
    throw Error{PUM_ERR_OOM, "bsr_alloc: device allocation failed"};
  }
  PUM_CUDA(cudaMemcpy(m.row_ptr, rp.data(), sizeof(int) * rp.size(), cudaMemcpyHostToDevice));
  if (!ci.empty()) PUM_CUDA(cudaMemcpy(m.col_idx, ci.data(), sizeof(int) * ci.size(), cudaMemcpyHostToDevice));
  // cudaMemset runs on the legacy stream, which does not order with the non-blocking streams the
  // library works on: wait for it, or a kernel on such a stream could write the values first
  // and be zeroed after (seen with concurrent set-ups)
  PUM_CUDA(cudaMemset(m.vals, 0, dt_size(dt) * (size_t)m.stride * std::max<int64_t>(m.nnzb, 1)));
  PUM_CUDA(cudaStreamSynchronize(0));
}

template <typename DT, typename ST>
__global__ void k_convert_blocks(DT* __restrict__ dst, int dstride, const ST* __restrict__ src, int sstride, int dd,
                                 int64_t nnzb) {
  const int64_t total = nnzb * dd;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / dd;
    const int e = (int)(i - b * dd);
    if constexpr (std::is_same<DT, __nv_bfloat16>::value)
      dst[b * dstride + e] = __double2bfloat16((double)src[b * sstride + e]);
    else
      dst[b * dstride + e] = (DT)src[b * sstride + e];
  }
}

void bsr_convert(Bsr& dst, const Bsr& src, int dt, cudaStream_t s) {
  PUM_CHECK(src.dt == PUM_F64, PUM_ERR_INVALID_ARG, "bsr_convert: source must be float64");
  bsr_alloc(dst, src.n_brows, src.n_bcols, src.d, dt, src.h_row_ptr, src.h_col_idx);
  const int64_t total = src.nnzb * src.d * src.d;
  if (!total) return;
  const unsigned g = elem_grid(total);
  const double* sv = (const double*)src.vals;
  if (dt == PUM_F64)
    k_convert_blocks<<<g, 256, 0, s>>>((double*)dst.vals, dst.stride, sv, src.stride, src.d * src.d, src.nnzb);
  else if (dt == PUM_F32)
    k_convert_blocks<<<g, 256, 0, s>>>((float*)dst.vals, dst.stride, sv, src.stride, src.d * src.d, src.nnzb);
  else
    k_convert_blocks<<<g, 256, 0, s>>>((__nv_bfloat16*)dst.vals, dst.stride, sv, src.stride, src.d * src.d,
                                       src.nnzb);
  PUM_CUDA(cudaGetLastError());
}

template <typename T>
__global__ void k_transpose_blocks(T* __restrict__ dst, const T* __restrict__ src, const int* __restrict__ map,
                                   int stride, int d, int64_t nnzb) {
  const int dd = d * d;
  const int64_t total = nnzb * dd;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / dd;
    const int e = (int)(i - b * dd);
    const int r = e / d, c = e - (e / d) * d;
    dst[b * stride + r * d + c] = src[(int64_t)map[b] * stride + c * d + r];
  }
}

void bsr_transpose(Bsr& dst, const Bsr& src, cudaStream_t s) {
  const int nr = src.n_bcols;
  std::vector<int> cnt(nr + 1, 0);
  for (int c : src.h_col_idx) cnt[c + 1]++;
  for (int i = 0; i < nr; ++i) cnt[i + 1] += cnt[i];
  std::vector<int> rp = cnt, ci(src.nnzb), map(src.nnzb);
  std::vector<int> pos(cnt.begin(), cnt.end() - 1);
  for (int i = 0; i < src.n_brows; ++i)
    for (int b = src.h_row_ptr[i]; b < src.h_row_ptr[i + 1]; ++b) {
      const int c = src.h_col_idx[b];
      const int q = pos[c]++;
      ci[q] = i;  // rows visited in increasing order: columns of the transpose come out sorted
      map[q] = b;
    }
  bsr_alloc(dst, src.n_bcols, src.n_brows, src.d, src.dt, rp, ci);
  if (!src.nnzb) return;
  int* dmap = nullptr;
  PUM_CUDA(cudaMalloc(&dmap, sizeof(int) * map.size()));
  PUM_CUDA(cudaMemcpyAsync(dmap, map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice, s));
  const unsigned g = elem_grid(src.nnzb * src.d * src.d);
  if (src.dt == PUM_F64)
    k_transpose_blocks<<<g, 256, 0, s>>>((double*)dst.vals, (const double*)src.vals, dmap, src.stride, src.d, src.nnzb);
  else if (src.dt == PUM_F32)
    k_transpose_blocks<<<g, 256, 0, s>>>((float*)dst.vals, (const float*)src.vals, dmap, src.stride, src.d, src.nnzb);
  else
    k_transpose_blocks<<<g, 256, 0, s>>>((__nv_bfloat16*)dst.vals, (const __nv_bfloat16*)src.vals, dmap, src.stride,
                                         src.d, src.nnzb);
  PUM_CUDA(cudaGetLastError());
  PUM_CUDA(cudaStreamSynchronize(s));
  cudaFree(dmap);
}

template <typename ST>
__global__ void k_widen_blocks(double* __restrict__ dst, int dstride, const ST* __restrict__ src, int sstride, int dd,
                               int64_t nnzb) {
  const int64_t total = nnzb * dd;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / dd;
    const int e = (int)(i - b * dd);
    dst[b * dstride + e] = (double)to_f(src[b * sstride + e]);
  }
}

void bsr_widen(Bsr& dst, const Bsr& src, cudaStream_t s) {
  bsr_alloc(dst, src.n_brows, src.n_bcols, src.d, PUM_F64, src.h_row_ptr, src.h_col_idx);
  const int64_t total = src.nnzb * src.d * src.d;
  if (!total) return;
  const unsigned g = elem_grid(total);
  if (src.dt == PUM_F64)
    k_widen_blocks<<<g, 256, 0, s>>>((double*)dst.vals, dst.stride, (const double*)src.vals, src.stride, src.d * src.d, src.nnzb);
  else if (src.dt == PUM_F32)
    k_widen_blocks<<<g, 256, 0, s>>>((double*)dst.vals, dst.stride, (const float*)src.vals, src.stride, src.d * src.d, src.nnzb);
  else
    k_widen_blocks<<<g, 256, 0, s>>>((double*)dst.vals, dst.stride, (const __nv_bfloat16*)src.vals, src.stride,
                                     src.d * src.d, src.nnzb);
  PUM_CUDA(cudaGetLastError());
}

std::vector<double> bsr_values_host(const Bsr& m, cudaStream_t s) {
  PUM_CHECK(m.dt == PUM_F64, PUM_ERR_INVALID_ARG, "export needs float64 values");
  const int dd = m.d * m.d;
  std::vector<double> padded((size_t)m.nnzb * m.stride), out((size_t)m.nnzb * dd);
  if (m.nnzb) {
    PUM_CUDA(cudaMemcpyAsync(padded.data(), m.vals, sizeof(double) * padded.size(), cudaMemcpyDeviceToHost, s));
    PUM_CUDA(cudaStreamSynchronize(s));
  }
  for (int64_t b = 0; b < m.nnzb; ++b) std::memcpy(&out[b * dd], &padded[b * m.stride], sizeof(double) * dd);
  return out;
}

// ----------------------------------------------------------------------------- SpGEMM

void pattern_product(const std::vector<int>& xrp, const std::vector<int>& xci, const std::vector<int>& yrp,
                     const std::vector<int>& yci, int n_rows, std::vector<int>& crp, std::vector<int>& cci) {
  int ny_cols = 0;
  for (int c : yci) ny_cols = std::max(ny_cols, c + 1);
  std::vector<int> mark(ny_cols, -1);
  crp.assign(n_rows + 1, 0);
  cci.clear();
  std::vector<int> cols;
  for (int i = 0; i < n_rows; ++i) {
    cols.clear();
    for (int b = xrp[i]; b < xrp[i + 1]; ++b) {
      const int j = xci[b];
      for (int q = yrp[j]; q < yrp[j + 1]; ++q) {
        const int k = yci[q];
        if (mark[k] != i) {
          mark[k] = i;
          cols.push_back(k);
        }
      }
    }
    std::sort(cols.begin(), cols.end());
    cci.insert(cci.end(), cols.begin(), cols.end());
    crp[i + 1] = (int)cci.size();
  }
}

// One CTA per block of C: C_ik = sum_j X_ij Y_jk, j over X's row i (in order), Y_jk
// found by binary search in Y's row j.  Blocks staged in shared memory; FP64.
__global__ void k_spgemm_numeric(const int* __restrict__ c_row_of, const int* __restrict__ c_ci, double* __restrict__ cv,
                                 int cstride, const int* __restrict__ xrp, const int* __restrict__ xci,
                                 const double* __restrict__ xv, int xstride, const int* __restrict__ yrp,
                                 const int* __restrict__ yci, const double* __restrict__ yv, int ystride, int d) {
  extern __shared__ double sm[];
  double* Xs = sm;
  double* Ys = sm + d * d;
  const int64_t cb = blockIdx.x;
  const int i = c_row_of[cb];
  const int k = c_ci[cb];
  const int dd = d * d;
  double acc[4] = {0, 0, 0, 0};  // entries threadIdx.x + 128*t, t < 4 (d <= 21 -> dd <= 441 < 512)
  for (int xb = xrp[i]; xb < xrp[i + 1]; ++xb) {
    const int j = xci[xb];
    int lo = yrp[j], hi = yrp[j + 1] - 1, yb = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int c = yci[mid];
      if (c == k) { yb = mid; break; }
      if (c < k) lo = mid + 1; else hi = mid - 1;
    }
    if (yb < 0) continue;  // uniform across the CTA
    __syncthreads();
    for (int e = threadIdx.x; e < dd; e += blockDim.x) {
      Xs[e] = xv[(int64_t)xb * xstride + e];
      Ys[e] = yv[(int64_t)yb * ystride + e];
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = threadIdx.x + 128 * t;
      if (e < dd) {
        const int r = e / d, c = e - (e / d) * d;
        double s = acc[t];
        for (int q = 0; q < d; ++q) s = fma(Xs[r * d + q], Ys[q * d + c], s);
        acc[t] = s;
      }
    }
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int e = threadIdx.x + 128 * t;
    if (e < dd) cv[cb * cstride + e] = acc[t];
  }
}

void spgemm_numeric(Bsr& C, const Bsr& X, const Bsr& Y, cudaStream_t s) {
  PUM_CHECK(X.dt == PUM_F64 && Y.dt == PUM_F64 && C.dt == PUM_F64, PUM_ERR_INVALID_ARG, "spgemm: float64 only");
  PUM_CHECK(X.d == Y.d && C.d == X.d && X.d <= 21, PUM_ERR_INVALID_ARG, "spgemm: block sizes");
  if (!C.nnzb) return;
  std::vector<int> row_of(C.nnzb);
  for (int i = 0; i < C.n_brows; ++i)
    for (int b = C.h_row_ptr[i]; b < C.h_row_ptr[i + 1]; ++b) row_of[b] = i;
  int* drow = nullptr;
  PUM_CUDA(cudaMalloc(&drow, sizeof(int) * row_of.size()));
  PUM_CUDA(cudaMemcpyAsync(drow, row_of.data(), sizeof(int) * row_of.size(), cudaMemcpyHostToDevice, s));
  const size_t smem = 2 * sizeof(double) * X.d * X.d;
  k_spgemm_numeric<<<(unsigned)C.nnzb, 128, smem, s>>>(drow, C.col_idx, (double*)C.vals, C.stride, X.row_ptr,
                                                      X.col_idx, (const double*)X.vals, X.stride, Y.row_ptr,
                                                      Y.col_idx, (const double*)Y.vals, Y.stride, X.d);
  PUM_CUDA(cudaGetLastError());
  PUM_CUDA(cudaStreamSynchronize(s));
  cudaFree(drow);
}

void spgemm(Bsr& C, const Bsr& X, const Bsr& Y, cudaStream_t s) {
  std::vector<int> rp, ci;
  pattern_product(X.h_row_ptr, X.h_col_idx, Y.h_row_ptr, Y.h_col_idx, X.n_brows, rp, ci);
  bsr_alloc(C, X.n_brows, Y.n_bcols, X.d, PUM_F64, rp, ci);
  spgemm_numeric(C, X, Y, s);
}

}  // namespace pum
