// Several right-hand sides of one hierarchy at once: the V(k,k) cycle of Section 5 with the
// Chebyshev-4 smoother of Algorithm 3 applied to a block of K vectors, and PCG run for every
// column in lockstep.  Each product reads a matrix once for all K columns, so per right-hand side
// the operators cost 1/K of their bytes: the batched workload's instances carry 16 right-hand
// sides each.
//
// Block vectors are unknown-major: value (u, c) at u K + c, so the d x K panel X_j of block
// column j is contiguous.  k_bsr_mm: one warp per block row; lane l owns the outputs (r, c) with
// r K + c = l, l + 32, ...; for every block of the row it multiplies the block's row r (read
// through L1, shared by the lanes of one r) with the panel's column c.  The arithmetic intensity
// grows with K (FP32: d^2 K multiply-adds per 4 d^2 bytes of matrix, 4 per byte at K = 16), so at
// K = 16 the FP32 product runs near both the FP32 and the HBM rates; the contraction per block
// (d x d times d x K, different X_j per row) is too small and too irregular to fill tcgen05 tiles,
// and a TF32 product would cost the smoother precision, so it stays on the FP32 pipes.
// The Chebyshev update is the product's epilogue, column by column with the level's scalars (mu
// and beta do not depend on the column).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "pum_internal.cuh"

namespace pum {

namespace {

enum MmEpi { MM_SET = 0, MM_RESID = 1, MM_ADD = 2, MM_CHEB_FIRST0 = 3, MM_CHEB_FIRST = 4, MM_CHEB = 5 };

template <typename T>
__device__ __forceinline__ double ld(const T* p) {
  return (double)p[0];
}
template <>
__device__ __forceinline__ double ld<__nv_bfloat16>(const __nv_bfloat16* p) {
  return (double)__bfloat162float(p[0]);
}

// y (n_rows D x K) by epilogue of acc = M x; MT matrix values, VT vectors (accumulation in VT's
// precision: FP32 for float vectors, FP64 for double).  One warp per block row: the warp loads each
// block and its panel X_j with coalesced loads into registers one block ahead (the column indices
// of the row are read up front, 32 at a time, and passed by shuffles), stages them in its shared
// memory, and every lane then forms its outputs (r, c) from there.
template <int D, int K, typename MT, typename VT>
__global__ void __launch_bounds__(128) k_bsr_mm(int n_rows, const int* __restrict__ rp, const int* __restrict__ ci,
                                                const MT* __restrict__ vals, int stride, const VT* __restrict__ x,
                                                VT* __restrict__ y, const VT* __restrict__ b, VT* __restrict__ xo,
                                                int epi, double mu2, double dmu) {
  static_assert(32 % K == 0, "a lane's column is the same for all its outputs");
  constexpr int kOut = (D * K + 31) / 32;
  constexpr int kM = (D * D + 31) / 32, kX = (D * K + 31) / 32;
  __shared__ VT sM[4][D * D];
  __shared__ VT sX[4][D * K];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 4 + w;
  if (row >= n_rows) return;
  const int c = lane % K;
  VT acc[kOut];
#pragma unroll
  for (int q = 0; q < kOut; ++q) acc[q] = VT(0);
  const int p0 = rp[row], p1 = rp[row + 1];
  VT mv[kM], xv[kX];
  int cols = 0;  // lane i holds the column of block p0 + 32 * chunk + i
  auto fetch = [&](int p) {
    if (((p - p0) & 31) == 0) cols = (p + lane < p1) ? ci[p + lane] : 0;
    const int j = __shfl_sync(0xffffffffu, cols, (p - p0) & 31);
    const MT* M = vals + (int64_t)p * stride;
    const VT* X = x + (int64_t)j * D * K;
#pragma unroll
    for (int i = 0; i < kM; ++i) {
      const int e = lane + 32 * i;
      mv[i] = e < D * D ? (VT)ld(M + e) : VT(0);
    }
#pragma unroll
    for (int i = 0; i < kX; ++i) {
      const int e = lane + 32 * i;
      xv[i] = e < D * K ? X[e] : VT(0);
    }
  };
  if (p0 < p1) fetch(p0);
  for (int p = p0; p < p1; ++p) {
#pragma unroll
    for (int i = 0; i < kM; ++i)
      if (lane + 32 * i < D * D) sM[w][lane + 32 * i] = mv[i];
#pragma unroll
    for (int i = 0; i < kX; ++i)
      if (lane + 32 * i < D * K) sX[w][lane + 32 * i] = xv[i];
    __syncwarp();
    if (p + 1 < p1) fetch(p + 1);  // the next block's loads overlap this block's arithmetic
    VT xc[D];
#pragma unroll
    for (int t = 0; t < D; ++t) xc[t] = sX[w][t * K + c];
#pragma unroll
    for (int q = 0; q < kOut; ++q) {
      const int e = lane + 32 * q;
      if (e < D * K) {
        const int r = e / K;
        VT a = acc[q];
#pragma unroll
        for (int t = 0; t < D; ++t) a = fma(sM[w][r * D + t], xc[t], a);
        acc[q] = a;
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int q = 0; q < kOut; ++q) {
    const int e = lane + 32 * q;
    if (e >= D * K) continue;
    const int64_t u = (int64_t)row * D * K + e;
    const VT v = acc[q];
    switch (epi) {
      case MM_SET: y[u] = v; break;
      case MM_RESID: y[u] = b[u] - v; break;
      case MM_ADD: y[u] += v; break;
      case MM_CHEB_FIRST0: y[u] = v; xo[u] = (VT)dmu * v; break;
      case MM_CHEB_FIRST: y[u] = v; xo[u] += (VT)dmu * v; break;
      default: {
        const VT pn = (VT)mu2 * y[u] + v;
        y[u] = pn;
        xo[u] += (VT)dmu * pn;
      }
    }
  }
}

struct MmArgs {
  const void* x = nullptr;
  void* y = nullptr;
  const void* b = nullptr;
  void* xo = nullptr;
  int epi = MM_SET;
  double mu2 = 0.0, dmu = 0.0;
};

template <int D, int K>
void mm_launch_d(pum_ctx* ctx, const Bsr& M, int vdt, const MmArgs& a) {
  const unsigned grid = (unsigned)((M.n_brows + 3) / 4);
  if (!grid) return;
  if (vdt == PUM_F64) {
    PUM_CHECK(M.dt == PUM_F64, PUM_ERR_UNSUPPORTED, "multi-RHS: FP64 vectors need an FP64 matrix");
    k_bsr_mm<D, K, double, double><<<grid, 128, 0, ctx->stream>>>(
        M.n_brows, M.row_ptr, M.col_idx, (const double*)M.vals, M.stride, (const double*)a.x, (double*)a.y,
        (const double*)a.b, (double*)a.xo, a.epi, a.mu2, a.dmu);
  } else if (M.dt == PUM_BF16) {
    k_bsr_mm<D, K, __nv_bfloat16, float><<<grid, 128, 0, ctx->stream>>>(
        M.n_brows, M.row_ptr, M.col_idx, (const __nv_bfloat16*)M.vals, M.stride, (const float*)a.x, (float*)a.y,
        (const float*)a.b, (float*)a.xo, a.epi, a.mu2, a.dmu);
  } else {
    PUM_CHECK(M.dt == PUM_F32, PUM_ERR_UNSUPPORTED, "multi-RHS: FP32 vectors need an FP32 or BF16 matrix");
    k_bsr_mm<D, K, float, float><<<grid, 128, 0, ctx->stream>>>(
        M.n_brows, M.row_ptr, M.col_idx, (const float*)M.vals, M.stride, (const float*)a.x, (float*)a.y,
        (const float*)a.b, (float*)a.xo, a.epi, a.mu2, a.dmu);
  }
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
}

template <int K>
void mm_launch_k(pum_ctx* ctx, const Bsr& M, int vdt, const MmArgs& a) {
  switch (M.d) {
    case 3: return mm_launch_d<3, K>(ctx, M, vdt, a);
    case 6: return mm_launch_d<6, K>(ctx, M, vdt, a);
    case 10: return mm_launch_d<10, K>(ctx, M, vdt, a);
    case 15: return mm_launch_d<15, K>(ctx, M, vdt, a);
    case 21: return mm_launch_d<21, K>(ctx, M, vdt, a);
    default: throw Error{PUM_ERR_UNSUPPORTED, "multi-RHS: block size"};
  }
}

void mm(pum_ctx* ctx, const Bsr& M, int vdt, int K, const MmArgs& a) {
  switch (K) {
    case 4: return mm_launch_k<4>(ctx, M, vdt, a);
    case 16: return mm_launch_k<16>(ctx, M, vdt, a);
    default: throw Error{PUM_ERR_UNSUPPORTED, "multi-RHS: K must be 4 or 16"};
  }
}

// ---------------------------------------------------------------------------- vector kernels

// Column-major caller block (column c at src + c N) <-> unknown-major block (u K + c); columns
// c >= nrhs of the unknown-major block are zero.
template <typename S, typename T>
__global__ void k_to_umajor(const S* __restrict__ src, T* __restrict__ dst, int64_t N, int K, int nrhs) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N * K; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = i / K;
    const int c = (int)(i - u * K);
    dst[i] = c < nrhs ? (T)src[(int64_t)c * N + u] : T(0);
  }
}

template <typename S, typename T>
__global__ void k_to_cmajor(const S* __restrict__ src, T* __restrict__ dst, int64_t N, int K, int nrhs) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N * nrhs; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / N);
    const int64_t u = i - (int64_t)c * N;
    dst[i] = (T)src[u * K + c];
  }
}

template <typename S, typename T>
__global__ void k_convert(const S* __restrict__ src, T* __restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (T)src[i];
}

// Per-column dot products of two unknown-major FP64 blocks: CTA partials, then a fixed-order sum.
constexpr int kDotThreads = 256;
__global__ void __launch_bounds__(kDotThreads) k_coldot(const double* __restrict__ a, const double* __restrict__ b,
                                                        int64_t N, int K, double* __restrict__ part) {
  __shared__ double s[kDotThreads];
  const int c = threadIdx.x % K, lanes = kDotThreads / K, sub = threadIdx.x / K;
  double acc = 0.0;
  for (int64_t u = (int64_t)blockIdx.x * lanes + sub; u < N; u += (int64_t)gridDim.x * lanes)
    acc += a[u * K + c] * b[u * K + c];
  s[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int q = 0; q < lanes; ++q) t += s[q * K + threadIdx.x];
    part[(int64_t)blockIdx.x * K + threadIdx.x] = t;
  }
}

__global__ void k_coldot_sum(const double* __restrict__ part, int nb, int K, double* __restrict__ out) {
  const int c = threadIdx.x;
  if (c >= K) return;
  double t = 0.0;
  for (int q = 0; q < nb; ++q) t += part[(int64_t)q * K + c];
  out[c] = t;
}

// x += alpha_c p, r -= alpha_c q (alpha_c = rz_c / pq_c, 0 for finished columns)
__global__ void k_pcg_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                         const double* __restrict__ q, const double* __restrict__ rz, const double* __restrict__ pq,
                         const int* __restrict__ live, int64_t N, int K) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N * K; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % K);
    if (!live[c]) continue;
    const double a = rz[c] / pq[c];
    x[i] += a * p[i];
    r[i] -= a * q[i];
  }
}

// p = z + beta_c p with beta_c = (rz_new_c - rzold_c) / rz_c (flexible) or rz_new_c / rz_c
__global__ void k_pcg_p(double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ rz_new,
                        const double* __restrict__ rz_cross, const double* __restrict__ rz, const int* __restrict__ live,
                        int flexible, int64_t N, int K) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N * K; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % K);
    if (!live[c]) continue;
    const double beta = (flexible ? rz_new[c] - rz_cross[c] : rz_new[c]) / rz[c];
    p[i] = z[i] + beta * p[i];
  }
}

template <typename VT>
__global__ void k_coarse_multi(const double* __restrict__ L, int N, int K, const VT* __restrict__ b,
                               VT* __restrict__ x) {
  extern __shared__ double y[];
  const int c = blockIdx.x;
  for (int i = threadIdx.x; i < N; i += blockDim.x) y[i] = (double)b[(int64_t)i * K + c];
  __syncthreads();
  for (int i = 0; i < N; ++i) {  // L y = b
    if (threadIdx.x == 0) y[i] /= L[(int64_t)i * N + i];
    __syncthreads();
    const double yi = y[i];
    for (int j = i + 1 + threadIdx.x; j < N; j += blockDim.x) y[j] -= L[(int64_t)j * N + i] * yi;
    __syncthreads();
  }
  for (int i = N - 1; i >= 0; --i) {  // L^T x = y
    if (threadIdx.x == 0) y[i] /= L[(int64_t)i * N + i];
    __syncthreads();
    const double xi = y[i];
    for (int j = threadIdx.x; j < i; j += blockDim.x) y[j] -= L[(int64_t)i * N + j] * xi;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) x[(int64_t)i * K + c] = (VT)y[i];
}

unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16); }

// ---------------------------------------------------------------------------- the cycle

struct MultiWork {
  int K = 0, vdt = PUM_F64;
  std::vector<void*> x, b, r, p, t;  // per level, N_l K values of the level's type
  std::vector<void*> owned;
  ~MultiWork() {
    for (void* q : owned) cudaFree(q);
  }
  void* alloc(size_t bytes) {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      throw Error{PUM_ERR_OOM, "multi-RHS: device allocation failed"};
    }
    owned.push_back(q);
    return q;
  }
};

const Bsr& smoothA(const pum_hier* h, int l) {
  const Level& L = h->lv[l];
  return L.vdt == PUM_F32 ? L.As : L.A;
}

void cheb4_multi(pum_ctx* ctx, pum_hier* h, MultiWork& w, int l, bool x_zero) {
  Level& L = h->lv[l];
  const int vdt = w.vdt, K = w.K;
  const int k = h->sp.degree_k;
  const bool richardson = h->sp.smoother == PUM_SMOOTHER_RICHARDSON;
  const double dd = 4.0 / L.beta;
  for (int i = 1; i <= k; ++i) {
    const void* src = w.b[l];
    if (!(i == 1 && x_zero)) {
      MmArgs a;
      a.x = w.x[l];
      a.y = w.r[l];
      a.b = w.b[l];
      a.epi = MM_RESID;
      mm(ctx, smoothA(h, l), vdt, K, a);  // r = b - A x
      src = w.r[l];
    }
    MmArgs g;
    g.x = src;
    g.y = w.t[l];
    g.epi = MM_SET;
    mm(ctx, L.G, vdt, K, g);  // t = G r
    MmArgs c;
    c.x = w.t[l];
    c.y = w.p[l];
    c.xo = w.x[l];
    c.dmu = richardson ? 1.0 : dd * h->mu[i - 1];
    if (i == 1) {
      c.epi = x_zero ? MM_CHEB_FIRST0 : MM_CHEB_FIRST;
    } else {
      c.epi = MM_CHEB;
      c.mu2 = richardson ? 0.0 : h->mu[i - 2] * h->mu[i - 2];
    }
    mm(ctx, L.GT, vdt, K, c);  // p (= mu^2 p +) G^T t; x += d mu p
  }
}

void vcycle_multi(pum_ctx* ctx, pum_hier* h, MultiWork& w, int l) {
  const int nl = (int)h->lv.size();
  const int K = w.K, vdt = w.vdt;
  if (l == nl - 1) {
    const int N = h->coarse.N;
    const size_t smem = sizeof(double) * N;
    if (vdt == PUM_F64)
      k_coarse_multi<double><<<K, 256, smem, ctx->stream>>>(h->coarse.L, N, K, (const double*)w.b[l], (double*)w.x[l]);
    else
      k_coarse_multi<float><<<K, 256, smem, ctx->stream>>>(h->coarse.L, N, K, (const float*)w.b[l], (float*)w.x[l]);
    count_launch(ctx);
    PUM_CUDA(cudaGetLastError());
    return;
  }
  Level& L = h->lv[l];
  cheb4_multi(ctx, h, w, l, true);  // pre-smoothing from x = 0
  MmArgs r;
  r.x = w.x[l];
  r.y = w.r[l];
  r.b = w.b[l];
  r.epi = MM_RESID;
  mm(ctx, smoothA(h, l), vdt, K, r);
  MmArgs rc;
  rc.x = w.r[l];
  rc.y = w.b[l + 1];
  rc.epi = MM_SET;
  mm(ctx, vdt == PUM_F32 ? L.PTs : L.PT, vdt, K, rc);  // restriction P^T r
  vcycle_multi(ctx, h, w, l + 1);
  MmArgs pr;
  pr.x = w.x[l + 1];
  pr.y = w.x[l];
  pr.epi = MM_ADD;
  mm(ctx, vdt == PUM_F32 ? L.Ps : L.P, vdt, K, pr);  // x += P e_c
  cheb4_multi(ctx, h, w, l, false);  // post-smoothing
}

void check_multi(pum_hier* h, int nrhs) {
  PUM_CHECK(h && h->setup_done, PUM_ERR_INVALID_ARG, "hierarchy not set up");
  PUM_CHECK(nrhs >= 1 && nrhs <= 16, PUM_ERR_INVALID_ARG, "multi-RHS: 1 to 16 right-hand sides");
  PUM_CHECK(!h->fp.nested, PUM_ERR_UNSUPPORTED, "multi-RHS: nested FSAI is not supported");
  PUM_CHECK(h->sp.cycle == PUM_CYCLE_VKK, PUM_ERR_UNSUPPORTED, "multi-RHS: V(k,k) cycle only");
  const int nl = (int)h->lv.size();
  for (int l = 0; l + 1 < nl; ++l)
    PUM_CHECK(h->lv[l].vdt == h->lv[0].vdt, PUM_ERR_UNSUPPORTED,
              "multi-RHS: every smoothed level in one precision (fp32_levels covering all levels)");
}

void multi_prepare(pum_ctx* ctx, pum_hier* h, MultiWork& w, int nrhs) {
  w.K = nrhs <= 4 ? 4 : 16;
  w.vdt = h->lv[0].vdt;
  const size_t vs = dt_size(w.vdt);
  const int nl = (int)h->lv.size();
  for (int l = 0; l < nl; ++l) {
    const size_t n = (size_t)h->lv[l].n * h->lv[l].d * w.K * vs;
    w.x.push_back(w.alloc(n));
    w.b.push_back(w.alloc(n));
    w.r.push_back(w.alloc(n));
    w.p.push_back(w.alloc(n));
    w.t.push_back(w.alloc(n));
  }
  (void)ctx;
}

// z = B r for an unknown-major FP64 block (K columns) through the cycle's precision.
void cycle_block(pum_ctx* ctx, pum_hier* h, MultiWork& w, const double* r, double* z) {
  const int64_t n = (int64_t)h->lv[0].n * h->lv[0].d * w.K;
  if (w.vdt == PUM_F64) {
    PUM_CUDA(cudaMemcpyAsync(w.b[0], r, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    k_convert<double, float><<<grid_for(n), 256, 0, ctx->stream>>>(r, (float*)w.b[0], n);
    count_launch(ctx);
  }
  vcycle_multi(ctx, h, w, 0);
  if (w.vdt == PUM_F64) {
    PUM_CUDA(cudaMemcpyAsync(z, w.x[0], sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    k_convert<float, double><<<grid_for(n), 256, 0, ctx->stream>>>((const float*)w.x[0], z, n);
    count_launch(ctx);
  }
  PUM_CUDA(cudaGetLastError());
}

bool capturable_stream(pum_ctx* ctx) {
  const uintptr_t st = (uintptr_t)ctx->stream;
  return ctx->graphs && st > 2;  // not the legacy or per-thread default stream
}

template <typename F>
pum_status guarded(pum_ctx* ctx, F&& f) {
  try {
    ctx->last_error.clear();
    PUM_CUDA(cudaSetDevice(ctx->device));
    return f();
  } catch (const Error& e) {
    ctx->last_error = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    ctx->last_error = "host allocation failed";
    return PUM_ERR_OOM;
  }
}

}  // namespace

// Per hierarchy and block width: the cycle's work blocks, the PCG blocks and scalars, and the
// cycle (r -> z on the cached blocks) captured as a CUDA graph on the first call from a
// capturable stream, replayed by every later cycle.
struct MultiCache {
  MultiWork w;
  double *x = nullptr, *r = nullptr, *z = nullptr, *zo = nullptr, *p = nullptr, *q = nullptr;
  double *part = nullptr, *sc = nullptr;
  int* live = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;
};

void multi_cache_free(MultiCache*& c) {
  if (!c) return;
  if (c->exec) cudaGraphExecDestroy(c->exec);
  delete c;
  c = nullptr;
}

namespace {

constexpr int kDotBlocks = 152 * 4;

MultiCache& multi_cache(pum_ctx* ctx, pum_hier* h, int nrhs) {
  const int K = nrhs <= 4 ? 4 : 16;
  if (h->multi && h->multi->w.K == K) return *h->multi;
  multi_cache_free(h->multi);
  auto c = new MultiCache();
  try {
    multi_prepare(ctx, h, c->w, nrhs);
    const int64_t NK = (int64_t)h->lv[0].n * h->lv[0].d * K;
    for (double** v : {&c->x, &c->r, &c->z, &c->zo, &c->p, &c->q}) *v = (double*)c->w.alloc(sizeof(double) * NK);
    c->part = (double*)c->w.alloc(sizeof(double) * kDotBlocks * K);
    c->sc = (double*)c->w.alloc(sizeof(double) * 6 * K);
    c->live = (int*)c->w.alloc(sizeof(int) * K);
  } catch (...) {
    delete c;
    throw;
  }
  h->multi = c;
  return *c;
}

// z = B r on the cache's blocks: replayed from the captured graph where the stream allows it.
void multi_cycle(pum_ctx* ctx, pum_hier* h, MultiCache& c) {
  if (!capturable_stream(ctx)) {
    cycle_block(ctx, h, c.w, c.r, c.z);
    return;
  }
  if (!c.exec) {
    cudaGraph_t graph = nullptr;
    const int64_t l0 = ctx->launches;
    PUM_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    try {
      cycle_block(ctx, h, c.w, c.r, c.z);
    } catch (...) {
      cudaStreamEndCapture(ctx->stream, &graph);
      if (graph) cudaGraphDestroy(graph);
      ctx->launches = l0;
      throw;
    }
    PUM_CUDA(cudaStreamEndCapture(ctx->stream, &graph));
    c.kernels = ctx->launches - l0;
    ctx->launches = l0;
    const cudaError_t e = cudaGraphInstantiate(&c.exec, graph, 0);
    cudaGraphDestroy(graph);
    PUM_CUDA(e);
  }
  PUM_CUDA(cudaGraphLaunch(c.exec, ctx->stream));
  ctx->launches += c.kernels;
}

}  // namespace

}  // namespace pum

using namespace pum;

extern "C" pum_status vcycle_apply_multi(pum_ctx* ctx, pum_hier* h, int32_t nrhs, const double* R, double* Z) {
  if (!ctx || !h || !R || !Z) return PUM_ERR_INVALID_ARG;
  return guarded(ctx, [&]() {
    check_multi(h, nrhs);
    MultiCache& c = multi_cache(ctx, h, nrhs);
    const int K = c.w.K;
    const int64_t N = (int64_t)h->lv[0].n * h->lv[0].d;
    k_to_umajor<double, double><<<grid_for(N * K), 256, 0, ctx->stream>>>(R, c.r, N, K, nrhs);
    count_launch(ctx);
    multi_cycle(ctx, h, c);
    k_to_cmajor<double, double><<<grid_for(N * nrhs), 256, 0, ctx->stream>>>(c.z, Z, N, K, nrhs);
    count_launch(ctx);
    PUM_CUDA(cudaGetLastError());
    PUM_CUDA(cudaStreamSynchronize(ctx->stream));
    return PUM_OK;
  });
}

extern "C" pum_status pcg_solve_multi(pum_ctx* ctx, pum_hier* h, int32_t nrhs, const double* B, double* X,
                                      pcg_report* reps) {
  if (!ctx || !h || !B || !X || !reps) return PUM_ERR_INVALID_ARG;
  return guarded(ctx, [&]() {
    check_multi(h, nrhs);
    const int maxit = reps[0].maxit;
    const double rtol = reps[0].rtol;
    const int flexible = reps[0].flexible;
    PUM_CHECK(maxit >= 1 && rtol > 0.0, PUM_ERR_INVALID_ARG, "multi-RHS: maxit >= 1 and rtol > 0 (from reps[0])");
    MultiCache& c = multi_cache(ctx, h, nrhs);
    const int K = c.w.K;
    cudaStream_t s = ctx->stream;
    const int64_t N = (int64_t)h->lv[0].n * h->lv[0].d, NK = N * K;
    double *x = c.x, *r = c.r, *z = c.z, *zo = c.zo, *p = c.p, *q = c.q, *part = c.part, *sc = c.sc;
    double *rz = sc, *pq = sc + K, *rr = sc + 2 * K, *rzn = sc + 3 * K, *rzc = sc + 4 * K, *bb = sc + 5 * K;
    int* live = c.live;
    auto dots = [&](const double* a, const double* b2, double* out) {
      k_coldot<<<kDotBlocks, kDotThreads, 0, s>>>(a, b2, N, K, part);
      k_coldot_sum<<<1, 32, 0, s>>>(part, kDotBlocks, K, out);
      ctx->launches += 2;
      PUM_CUDA(cudaGetLastError());
    };
    k_to_umajor<double, double><<<grid_for(NK), 256, 0, s>>>(B, r, N, K, nrhs);
    count_launch(ctx);
    PUM_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * NK, s));
    dots(r, r, bb);
    std::vector<double> hbb(K), hrr(K), hpq(K);
    PUM_CUDA(cudaMemcpyAsync(hbb.data(), bb, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
    PUM_CUDA(cudaStreamSynchronize(s));
    std::vector<int> hlive(K, 0);
    for (int cc = 0; cc < nrhs; ++cc) {
      hlive[cc] = hbb[cc] > 0.0;
      reps[cc].iters = 0;
      reps[cc].converged = !hlive[cc];
      reps[cc].final_relres = 0.0;
      if (reps[cc].hist) reps[cc].hist[0] = 1.0;
    }
    PUM_CUDA(cudaMemcpyAsync(live, hlive.data(), sizeof(int) * K, cudaMemcpyHostToDevice, s));
    multi_cycle(ctx, h, c);  // z = B r
    PUM_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * NK, cudaMemcpyDeviceToDevice, s));
    dots(r, z, rz);
    for (int it = 1; it <= maxit; ++it) {
      MmArgs a;
      a.x = p;
      a.y = q;
      a.epi = MM_SET;
      mm(ctx, h->lv[0].A, PUM_F64, K, a);  // q = A p (FP64)
      dots(p, q, pq);
      k_pcg_xr<<<grid_for(NK), 256, 0, s>>>(x, r, p, q, rz, pq, live, N, K);
      count_launch(ctx);
      dots(r, r, rr);
      PUM_CUDA(cudaMemcpyAsync(hrr.data(), rr, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
      PUM_CUDA(cudaMemcpyAsync(hpq.data(), pq, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
      PUM_CUDA(cudaStreamSynchronize(s));
      bool any = false;
      for (int cc = 0; cc < nrhs; ++cc) {
        if (!hlive[cc]) continue;
        PUM_CHECK(hpq[cc] > 0.0 && std::isfinite(hrr[cc]), PUM_ERR_BREAKDOWN,
                  "multi-RHS PCG breakdown in column " + std::to_string(cc) + " (p^T A p not positive)");
        const double rel = std::sqrt(hrr[cc] / hbb[cc]);
        reps[cc].iters = it;
        reps[cc].final_relres = rel;
        if (reps[cc].hist) reps[cc].hist[it] = rel;
        if (rel <= rtol) {
          reps[cc].converged = 1;
          hlive[cc] = 0;
        } else {
          any = true;
        }
      }
      if (!any) break;
      PUM_CUDA(cudaMemcpyAsync(live, hlive.data(), sizeof(int) * K, cudaMemcpyHostToDevice, s));
      if (flexible) PUM_CUDA(cudaMemcpyAsync(zo, z, sizeof(double) * NK, cudaMemcpyDeviceToDevice, s));
      multi_cycle(ctx, h, c);
      dots(r, z, rzn);
      if (flexible) dots(r, zo, rzc);
      k_pcg_p<<<grid_for(NK), 256, 0, s>>>(p, z, rzn, rzc, rz, live, flexible, N, K);
      count_launch(ctx);
      PUM_CUDA(cudaMemcpyAsync(rz, rzn, sizeof(double) * K, cudaMemcpyDeviceToDevice, s));
    }
    k_to_cmajor<double, double><<<grid_for(N * nrhs), 256, 0, s>>>(x, X, N, K, nrhs);
    count_launch(ctx);
    PUM_CUDA(cudaGetLastError());
    PUM_CUDA(cudaStreamSynchronize(s));
    DevStatus st{};
    PUM_CUDA(cudaMemcpy(&st, ctx->status, sizeof(st), cudaMemcpyDeviceToHost));
    PUM_CHECK(st.code == 0, (pum_status)st.code, "multi-RHS: device status");
    for (int cc = 0; cc < nrhs; ++cc)
      if (!reps[cc].converged) return PUM_ERR_NOCONV;
    return PUM_OK;
  });
}
