// Sliced block layout for the smoother's products on large levels.
//
// Block rows are grouped by R; group g stores S_g slots, S_g = its longest block row, and
// slot s of row j holds that row's s-th block (padding: column -1, never read).  The
// values of (group, slot, block column index c) are stored contiguously over the group's
// R*d output unknowns, so the R*d threads of a CTA (thread = output unknown) read each
// (slot, c) as one coalesced run: a warp's load is one 128-byte segment (FP32), with no
// reliance on L1 to merge the strided row slices of the block-row-major layout.  Padding
// slots cost memory but no bandwidth.  The fused epilogues are those of the BSR kernel.
#include <algorithm>

#include "kernels_common.cuh"

namespace pum {

template <int D> constexpr int sell_rows() { return D <= 3 ? 64 : D <= 10 ? 32 : 16; }

int sell_rows_for(int d) {
  switch (d) {
    case 3: return sell_rows<3>();
    case 6: return sell_rows<6>();
    case 10: return sell_rows<10>();
    case 15: return sell_rows<15>();
    case 21: return sell_rows<21>();
    default: return 0;
  }
}

// L lanes per output unknown split a group's slots (lane k takes slots s0 + k, s0 + k + L, ...);
// the partial sums meet in shared memory.  L = 2 lets a level with fewer rows fill the GPU.
// The group's column indices are staged in shared memory first, so the loads of a slot do
// not wait on its index, and two slots' loads are issued before their FMAs.  Padding slots
// (column -1) read column 0 against zero values, which keeps the loop branch-free.
template <int D, int R, int L, typename MT, typename XT, typename YT, typename X2T, int EPI>
__global__ void __launch_bounds__(R * D * L) k_sell_mv(int n_brows, const int* __restrict__ goff,
                                                       const int* __restrict__ cols, const MT* __restrict__ vals,
                                                       const XT* __restrict__ x, EpiArgs e) {
  using AT = typename AccOf<MT>::type;
  constexpr int RD = R * D;
  extern __shared__ int scol[];  // (s1 - s0) * R column indices of this group
  __shared__ AT red[L > 1 ? (L - 1) * RD : 1];
  const int g = blockIdx.x;
  const int lane = threadIdx.x / RD;
  const int t = threadIdx.x - lane * RD;  // j * D + r
  const int j = t / D;
  const int row = g * R + j;
  const bool active = row < n_brows;
  const int s0 = goff[g], s1 = goff[g + 1];
  for (int i = threadIdx.x; i < (s1 - s0) * R; i += blockDim.x) scol[i] = max(__ldg(cols + (int64_t)s0 * R + i), 0);
  __syncthreads();
  AT acc = 0;
  if (active) {
    const MT* v = vals + (int64_t)s0 * D * RD + t;
    int s = lane;
    const int ns = s1 - s0;
    for (; s + L < ns; s += 2 * L) {
      const int c0 = scol[s * R + j], c1 = scol[(s + L) * R + j];
      AT a0[D], a1[D], x0[D], x1[D];
#pragma unroll
      for (int cc = 0; cc < D; ++cc) {
        a0[cc] = (AT)to_f(__ldg(v + ((int64_t)s * D + cc) * RD));
        a1[cc] = (AT)to_f(__ldg(v + ((int64_t)(s + L) * D + cc) * RD));
      }
      load_row<D>(x + (int64_t)c0 * D, x0);
      load_row<D>(x + (int64_t)c1 * D, x1);
#pragma unroll
      for (int cc = 0; cc < D; ++cc) acc = fma(a0[cc], x0[cc], acc);
#pragma unroll
      for (int cc = 0; cc < D; ++cc) acc = fma(a1[cc], x1[cc], acc);
    }
    if (s < ns) {
      const int c0 = scol[s * R + j];
      AT xv[D];
      load_row<D>(x + (int64_t)c0 * D, xv);
#pragma unroll
      for (int cc = 0; cc < D; ++cc) acc = fma((AT)to_f(__ldg(v + ((int64_t)s * D + cc) * RD)), xv[cc], acc);
    }
  }
  if constexpr (L > 1) {
    if (lane > 0) red[(lane - 1) * RD + t] = acc;
    __syncthreads();
    if (lane > 0) return;
#pragma unroll
    for (int k = 1; k < L; ++k) acc += red[(k - 1) * RD + t];
  }
  if (!active) return;
  epilogue<EPI, AT, XT, YT, X2T>(e, (int64_t)row * D + (t - j * D), acc);
}

template <int D, int L, typename MT, typename XT, typename YT, typename X2T>
static void sell_launch_l(pum_ctx* ctx, const Bsr& M, const void* x, int epi, const EpiArgs& e) {
  constexpr int R = sell_rows<D>();
  const dim3 grid(M.sell.n_groups), block(R * D * L);
  const size_t smem = sizeof(int) * (size_t)M.sell.max_slots * R;
  const MT* v = (const MT*)M.sell.vals;
  const XT* xv = (const XT*)x;
  cudaStream_t s = ctx->stream;
  switch (epi) {
#define PUM_SELL_CASE(E)                                                                                 \
  case E:                                                                                                \
    k_sell_mv<D, R, L, MT, XT, YT, X2T, E><<<grid, block, smem, s>>>(M.n_brows, M.sell.goff, M.sell.cols, v, \
                                                                 xv, e);                                 \
    break;
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

template <int D, typename MT, typename XT, typename YT, typename X2T>
static void sell_launch(pum_ctx* ctx, const Bsr& M, const void* x, int epi, const EpiArgs& e) {
  // two lanes per output when one would leave the GPU under-filled (about sm_count x 2048 threads)
  if ((int64_t)M.n_brows * D < (int64_t)ctx->sm_count * 1536)
    sell_launch_l<D, 2, MT, XT, YT, X2T>(ctx, M, x, epi, e);
  else
    sell_launch_l<D, 1, MT, XT, YT, X2T>(ctx, M, x, epi, e);
}

template <int D>
static bool sell_mv_d(pum_ctx* ctx, const Bsr& M, int vdt, const void* x, int epi, const EpiArgs& e) {
  const int xdt = e.xdt >= 0 ? e.xdt : vdt;
  const int ydt = e.ydt >= 0 ? e.ydt : vdt;
  const int x2dt = (e.xo2 && e.x2dt >= 0) ? e.x2dt : ydt;
  const int mdt = M.dt;
  if (mdt == PUM_F32 && xdt == PUM_F32 && ydt == PUM_F32 && x2dt == PUM_F32)
    return sell_launch<D, float, float, float, float>(ctx, M, x, epi, e), true;
  if (mdt == PUM_F32 && xdt == PUM_F32 && ydt == PUM_F32 && x2dt == PUM_F64)
    return sell_launch<D, float, float, float, double>(ctx, M, x, epi, e), true;
  if (mdt == PUM_BF16 && xdt == PUM_F32 && ydt == PUM_F32 && x2dt == PUM_F32)
    return sell_launch<D, __nv_bfloat16, float, float, float>(ctx, M, x, epi, e), true;
  if (mdt == PUM_BF16 && xdt == PUM_F32 && ydt == PUM_F32 && x2dt == PUM_F64)
    return sell_launch<D, __nv_bfloat16, float, float, double>(ctx, M, x, epi, e), true;
  if (mdt == PUM_F32 && xdt == PUM_F32 && ydt == PUM_F64 && epi == EPI_ADD)
    return sell_launch<D, float, float, double, double>(ctx, M, x, epi, e), true;
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

// ----------------------------------------------------------------------------- build

template <typename T>
__global__ void k_sell_fill(T* __restrict__ dst, const T* __restrict__ src, const int* __restrict__ src_blk, int stride,
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
    dst[(slot * d + c) * (int64_t)(R * d) + j * d + r] = src[(int64_t)b * stride + r * d + c];
  }
}

void sell_free(Sell& s) {
  if (s.goff) cudaFree(s.goff);
  if (s.cols) cudaFree(s.cols);
  if (s.vals) cudaFree(s.vals);
  s = Sell();
}

void sell_build(Bsr& M, cudaStream_t st) {
  sell_free(M.sell);
  const int R = sell_rows_for(M.d);
  if (!R || M.dt == PUM_F64) return;
  const int n = M.n_brows, d = M.d;
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
  Sell& S = M.sell;
  const size_t vbytes = dt_size(M.dt) * (size_t)std::max<int64_t>(slots, 1) * R * d * d;
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
    if (M.dt == PUM_F32)
      k_sell_fill<<<grid, 256, 0, st>>>((float*)S.vals, (const float*)M.vals, dsrc, M.stride, d, R, slots);
    else
      k_sell_fill<<<grid, 256, 0, st>>>((__nv_bfloat16*)S.vals, (const __nv_bfloat16*)M.vals, dsrc, M.stride, d, R,
                                        slots);
    PUM_CUDA(cudaGetLastError());
  }
  PUM_CUDA(cudaStreamSynchronize(st));
  cudaFree(dsrc);
  S.R = R;
  S.n_groups = ng;
  S.slots = slots;
  S.max_slots = 0;
  for (int g = 0; g < ng; ++g) S.max_slots = std::max(S.max_slots, goff[g + 1] - goff[g]);
  PUM_CHECK((size_t)S.max_slots * R * sizeof(int) <= 32768, PUM_ERR_UNSUPPORTED, "sliced layout: row too long");
}

}  // namespace pum
