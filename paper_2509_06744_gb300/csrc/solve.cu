// Hot path: fourth-kind Chebyshev smoothing (Algorithm 3) with the block-FSAI
// preconditioner M = G^T G (nested: F0^T G1^T G1 F0), the V(k,k) cycle with L2
// transfers and a dense coarsest solve (Section 5), and the outer FP64 PCG.
#include <cmath>

#include "kernels_common.cuh"

namespace pum {

// ----------------------------------------------------------------------------- timing

void timing_begin(pum_ctx* ctx, int tk) {
  if (!((ctx->timing >> tk) & 1)) return;
  if (ctx->capture_ev) {  // inside a graph capture: the graph gets its own event pair
    TimedEvent t{tk, nullptr, nullptr};
    PUM_CUDA(cudaEventCreate(&t.start));
    PUM_CUDA(cudaEventCreate(&t.stop));
    ctx->capture_ev->push_back(t);
    PUM_CUDA(cudaEventRecordWithFlags(t.start, ctx->stream, cudaEventRecordExternal));  // a graph node
    return;
  }
  const size_t i = (size_t)ctx->tk_pool_used[tk];
  if (i >= ctx->tk_start[tk].size()) {
    cudaEvent_t a, b;
    PUM_CUDA(cudaEventCreate(&a));
    PUM_CUDA(cudaEventCreate(&b));
    ctx->tk_start[tk].push_back(a);
    ctx->tk_stop[tk].push_back(b);
  }
  PUM_CUDA(cudaEventRecord(ctx->tk_start[tk][i], ctx->stream));
}

void timing_end(pum_ctx* ctx, int tk) {
  if (!((ctx->timing >> tk) & 1)) return;
  if (ctx->capture_ev) {
    PUM_CUDA(cudaEventRecordWithFlags(ctx->capture_ev->back().stop, ctx->stream, cudaEventRecordExternal));
    return;
  }
  const size_t i = (size_t)ctx->tk_pool_used[tk];
  PUM_CUDA(cudaEventRecord(ctx->tk_stop[tk][i], ctx->stream));
  ctx->tk_pool_used[tk]++;
}

// ----------------------------------------------------------------------------- smoother

static const Bsr& smoothA(pum_hier* h, int l) { return h->lv[l].vdt == PUM_F64 ? h->lv[l].A : h->lv[l].As; }

// z = M r with the level's block-FSAI factors; the last product carries the epilogue.
static void fsai_apply_epi(pum_ctx* ctx, pum_hier* h, int l, const void* r, int epi, EpiArgs e) {
  Level& L = h->lv[l];
  const int vdt = L.vdt;
  const bool fin = (l == 0);
  const bool fused = L.gg.S.R > 0;  // G (or G1) read once: partial products, then the gather
  EpiArgs s{};
  if (!h->fp.nested) {
    if (fused) return gg_apply(ctx, L.gg, r, epi, e, fin ? PUM_TK_G : -1, fin ? PUM_TK_GT : -1);
    s.y = L.t;
    bsr_mv(ctx, L.G, vdt, r, EPI_SET, s, fin ? PUM_TK_G : -1);
    bsr_mv(ctx, L.GT, vdt, L.t, epi, e, fin ? PUM_TK_GT : -1);
    return;
  }
  s.y = L.t;
  bsr_mv(ctx, L.F0, vdt, r, EPI_SET, s, fin ? PUM_TK_G : -1);
  if (fused) {  // t <- G1^T G1 t (the gather runs after the partial products have read t)
    gg_apply(ctx, L.gg, L.t, EPI_SET, s, fin ? PUM_TK_G : -1, fin ? PUM_TK_GT : -1);
    bsr_mv(ctx, L.F0T, vdt, L.t, epi, e, fin ? PUM_TK_GT : -1);
    return;
  }
  s.y = L.u;
  bsr_mv(ctx, L.G1, vdt, L.t, EPI_SET, s, fin ? PUM_TK_G : -1);
  s.y = L.t;
  bsr_mv(ctx, L.G1T, vdt, L.u, EPI_SET, s, fin ? PUM_TK_GT : -1);
  bsr_mv(ctx, L.F0T, vdt, L.t, epi, e, fin ? PUM_TK_GT : -1);
}

void apply_M(pum_ctx* ctx, pum_hier* h, int l, const void* r, void* z, int) {
  EpiArgs e{};
  e.y = z;
  fsai_apply_epi(ctx, h, l, r, EPI_SET, e);
}

// Algorithm 3 on level l for A x = rhs with iterate x (in place), `steps` steps (0: degree_k);
// x_zero: x0 = 0.  When x_acc is given, every update of x is also added to x_acc (the correction
// form below).  Richardson smoothing (Section 3.1) is the same loop with p = M r and x = x + p:
// mu^2 = 0 and d mu = 1 in the fused update.
void cheb4(pum_ctx* ctx, pum_hier* h, int l, const void* rhs, void* x, bool x_zero, void* x_acc, int acc_dt,
           bool acc_set, void* x_acc_split, int steps) {
  Level& L = h->lv[l];
  const int vdt = L.vdt;
  const int k = steps > 0 ? steps : h->sp.degree_k;
  const bool richardson = h->sp.smoother == PUM_SMOOTHER_RICHARDSON;
  const double dd = 4.0 / L.beta;  // d = 4 / beta
  const bool fin = (l == 0);
  for (int i = 1; i <= k; ++i) {
    const void* src = rhs;  // r = b when x0 = 0 on the first step
    if (!(i == 1 && x_zero)) {
      EpiArgs e{};
      e.y = L.r;
      e.b = rhs;
      bsr_mv(ctx, smoothA(h, l), vdt, x, EPI_RESID, e, fin ? PUM_TK_RESID : -1);  // r = b - A x
      src = L.r;
    }
    EpiArgs e{};
    e.y = L.p;
    e.xo = x;
    e.xo2 = x_acc;
    e.x2s = x_acc_split;
    e.x2dt = acc_dt;
    e.x2_set = acc_set && x_zero && i == 1;
    e.dmu = richardson ? 1.0 : dd * h->mu[i - 1];
    int epi;
    if (i == 1) {
      epi = x_zero ? EPI_CHEB_FIRST0 : EPI_CHEB_FIRST;  // p = M r; x = x0 + d mu p
    } else {
      epi = EPI_CHEB;  // p = mu^2 p + M r; mu <- 1/(2 - mu); x = x + d mu p
      e.mu2 = richardson ? 0.0 : h->mu[i - 2] * h->mu[i - 2];
    }
    fsai_apply_epi(ctx, h, l, src, epi, e);
  }
}

// ----------------------------------------------------------------------------- coarse solve

template <typename VT>
__global__ void k_coarse_solve(const double* __restrict__ L, int N, const VT* __restrict__ b, VT* __restrict__ x) {
  extern __shared__ double y[];
  pdl_wait();
  pdl_release();
  for (int i = threadIdx.x; i < N; i += blockDim.x) y[i] = (double)b[i];
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
  for (int i = threadIdx.x; i < N; i += blockDim.x) x[i] = (VT)y[i];
}

void coarse_solve(pum_ctx* ctx, pum_hier* h, const void* b, void* x, int vdt) {
  const int N = h->coarse.N;
  const size_t smem = sizeof(double) * N;
  if (vdt == PUM_F64)
    launch_cycle_kernel(ctx, k_coarse_solve<double>, dim3(1), dim3(256), smem, (const double*)h->coarse.L, N,
                        (const double*)b, (double*)x);
  else
    launch_cycle_kernel(ctx, k_coarse_solve<float>, dim3(1), dim3(256), smem, (const double*)h->coarse.L, N,
                        (const float*)b, (float*)x);
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
}

// ----------------------------------------------------------------------------- V-cycle

// One V(k,k) cycle from level l: L.x = B_l L.b.
//
// FP32 form with mixed_levels > 0: Algorithm 3 is a polynomial method, x_k = x0 + q(MA) M (b - A x0),
// so post-smoothing from x0 equals x0 plus post-smoothing of A e = c, c = b - A x0, from e0 = 0.
// After the coarse correction x holds large smooth components, and an FP32 b - A x loses them
// to cancellation (kappa(A) eps_32 >> 1 on the fine levels).  So c is formed once with the FP64
// operator and FP64 sums, the FP32 smoother works on the small correction e, and every update of
// e is also added to x in the same epilogue.  The residual restricted to the coarser level is
// formed the same way.  In exact arithmetic this is the same cycle.
void vcycle_level(pum_ctx* ctx, pum_hier* h, int l) {
  Level& L = h->lv[l];
  const int vdt = L.vdt;
  if (l == (int)h->lv.size() - 1) {
    coarse_solve(ctx, h, L.b, L.x, vdt);
    return;
  }
  Level& C = h->lv[l + 1];
  const Bsr& PT = vdt == PUM_F64 ? L.PT : L.PTs;
  const Bsr& P = vdt == PUM_F64 ? L.P : L.Ps;
  const bool corr = vdt == PUM_F32 && h->sp.mixed_levels > 0;
  const Bsr& Ar = corr ? L.A : smoothA(h, l);  // operator of the two accurate residuals
  const int tk_r = l == 0 ? (corr ? PUM_TK_RESID64 : PUM_TK_RESID) : -1;
  const bool v2k0 = h->sp.cycle == PUM_CYCLE_V2K0;
  // pre-smoothing from x0 = 0: k steps, or 2k for V(2k,0)
  cheb4(ctx, h, l, L.b, L.x, true, nullptr, -1, false, nullptr, v2k0 ? 2 * h->sp.degree_k : 0);
  EpiArgs e{};
  e.y = L.r;
  e.b = L.b;
  bsr_mv(ctx, Ar, vdt, L.x, EPI_RESID, e, tk_r);  // r = b - A x
  EpiArgs rs{};
  rs.y = C.b;
  bsr_mv(ctx, PT, vdt, L.r, EPI_SET, rs);  // b_c = P^T r
  vcycle_level(ctx, h, l + 1);
  EpiArgs pa{};
  pa.y = L.x;
  bsr_mv(ctx, P, vdt, C.x, EPI_ADD, pa);  // x += P x_c
  if (v2k0) return;  // V(2k,0): no post-smoothing
  if (!corr) {
    cheb4(ctx, h, l, L.b, L.x, false, nullptr, -1, false);  // post-smoothing, same polynomial
    return;
  }
  EpiArgs cr{};
  cr.y = L.c;
  cr.b = L.b;
  bsr_mv(ctx, Ar, vdt, L.x, EPI_RESID, cr, tk_r);  // c = b - A x
  cheb4(ctx, h, l, L.c, L.e, true, L.x, -1, false);  // A e = c from e0 = 0; x += each update
}

// ----------------------------------------------------------------------------- PCG

enum { S_RZ = 0, S_PQ = 1, S_RR = 2, S_RZN = 3, S_RZO = 4, S_BB = 5 };

// x += alpha p, r -= alpha q with alpha = scal[RZ] / scal[PQ]; partial sums of r.r
__global__ void k_pcg_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                         const double* __restrict__ q, const double* __restrict__ scal, int64_t n,
                         double* __restrict__ partials) {
  __shared__ double red[8];
  const double alpha = scal[S_RZ] / scal[S_PQ];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    s = fma(ri, ri, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partials[blockIdx.x] = t;
  }
}

// p = z + beta p, beta = (scal[RZN] - flex * scal[RZO]) / scal[RZ]
__global__ void k_pcg_p(double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ scal,
                        int flexible, int64_t n) {
  const double beta = (scal[S_RZN] - (flexible ? scal[S_RZO] : 0.0)) / scal[S_RZ];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

__global__ void k_scal_move(double* scal, int dst, int src) { scal[dst] = scal[src]; }

void graph_destroy(GraphCache& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto& t : g.ev) {
    cudaEventDestroy(t.start);
    cudaEventDestroy(t.stop);
  }
  g = GraphCache();
}

void graph_harvest(pum_ctx* ctx, pum_hier* h) {
  GraphCache& g = h->vgraph;
  if (!g.pending) return;
  g.pending = false;
  for (auto& t : g.ev) {
    PUM_CUDA(cudaEventSynchronize(t.stop));
    float ms = 0.f;
    PUM_CUDA(cudaEventElapsedTime(&ms, t.start, t.stop));
    ctx->tk_ms[t.tk] += ms;
    ctx->tk_launches[t.tk]++;
  }
}

// Streams a graph can be captured on: not the legacy or per-thread default streams.
static bool capturable(pum_ctx* ctx) {
  const uintptr_t s = (uintptr_t)ctx->stream;
  return ctx->graphs && s > 2;
}

// Mixed levels of the FP32 form (l < mixed_levels): the level's iterate z and right-hand
// side r stay in FP64.  The FP32 smoother works on correction vectors (pre-smoothing from
// zero, post-smoothing of A e = c) and its fused epilogue adds every update to z in FP64,
// so z carries no FP32 rounding: A times an FP32 rounding of a smooth z would be
// kappa * eps_32 times larger than a smooth residual.  Both residuals use the FP64
// operator on the FP64 z and r; the coarse correction of a mixed coarser level is
// prolongated with the FP64 P.  In exact arithmetic this is the same V(k,k) cycle.
static bool is_mixed(const pum_hier* h, int l) {
  return h->lv[l].vdt == PUM_F32 && l < h->sp.mixed_levels;
}

// y = b - A z with FP64 b and z, FP32 y, to FP64 accuracy: on the sliced layout in double-float
// arithmetic (A as FP32 pairs, z read through its split shadow, which every writer of z on this
// level keeps current), else with the FP64 operator.
static void accurate_residual(pum_ctx* ctx, Level& L, const double* z, const EpiArgs& e, int tk) {
  if (L.Adf.R) {
    sell_df_mv(ctx, L.Adf, L.d, L.n, L.zs, EPI_RESID, e, tk);
    return;
  }
  bsr_mv(ctx, L.A, PUM_F32, z, EPI_RESID, e, tk);
}

static void vcycle_mixed(pum_ctx* ctx, pum_hier* h, int l, const double* r, double* z) {
  Level& L = h->lv[l];
  const int64_t N = (int64_t)L.n * L.d;
  if (l == (int)h->lv.size() - 1) {
    coarse_solve(ctx, h, r, z, PUM_F64);
    return;
  }
  Level& C = h->lv[l + 1];
  const int tk = l == 0 ? PUM_TK_RESID64 : -1;
  const bool v2k0 = h->sp.cycle == PUM_CYCLE_V2K0;
  // FP32 right-hand side of the smoother; below the finest level the restriction that produced
  // r (an FP64 copy of its FP32 result) has already left exactly these values in L.b
  if (l == 0) convert_vec(ctx, L.b, PUM_F32, r, PUM_F64, N);
  // pre-smoothing: z = e in FP64 (k steps, 2k for V(2k,0))
  cheb4(ctx, h, l, L.b, L.e, true, z, PUM_F64, true, L.zs, v2k0 ? 2 * h->sp.degree_k : 0);
  EpiArgs er{};
  er.y = L.r;
  er.b = r;
  er.xdt = PUM_F64;
  er.ydt = PUM_F32;
  accurate_residual(ctx, L, z, er, tk);  // r_f = r - A z
  EpiArgs rs{};
  rs.y = C.b;
  EpiArgs pa{};
  if (C.vdt == PUM_F64) {  // the coarser levels smooth in FP64: an FP64 cycle from there down
    rs.xdt = PUM_F32;
    bsr_mv(ctx, L.PT, PUM_F64, L.r, EPI_SET, rs);  // b_c = P^T r_f (FP64)
    vcycle_level(ctx, h, l + 1);
    pa.y = z;
    pa.ys = L.zs;
    bsr_mv(ctx, L.P, PUM_F64, C.x, EPI_ADD, pa);  // z += P x_c (FP64)
  } else if (is_mixed(h, l + 1) || l + 1 == (int)h->lv.size() - 1) {
    rs.xo2 = C.b64;  // and its FP64 copy, the coarser level's right-hand side
    rs.x2dt = PUM_F64;
    bsr_mv(ctx, L.PTs, PUM_F32, L.r, EPI_SET, rs);  // b_c = P^T r_f
    vcycle_mixed(ctx, h, l + 1, C.b64, C.z64);
    pa.y = z;
    pa.ys = L.zs;
    if (L.Pdf.R)
      sell_df_mv(ctx, L.Pdf, L.d, L.n, C.zs, EPI_ADD, pa);  // z += P z_c in double-float arithmetic
    else
      bsr_mv(ctx, L.P, PUM_F64, C.z64, EPI_ADD, pa);  // z += P z_c (FP64)
  } else {
    bsr_mv(ctx, L.PTs, PUM_F32, L.r, EPI_SET, rs);  // b_c = P^T r_f
    vcycle_level(ctx, h, l + 1);
    pa.y = z;
    pa.ys = L.zs;
    pa.ydt = PUM_F64;
    bsr_mv(ctx, L.Ps, PUM_F32, C.x, EPI_ADD, pa);  // z += P x_c
  }
  if (v2k0) return;  // V(2k,0): no post-smoothing
  EpiArgs cr{};
  cr.y = L.c;
  cr.b = r;
  cr.xdt = PUM_F64;
  cr.ydt = PUM_F32;
  accurate_residual(ctx, L, z, cr, tk);                 // c = r - A z
  cheb4(ctx, h, l, L.c, L.e, true, z, PUM_F64, false, L.zs);  // A e = c from 0; z += updates
}

static void vcycle_body(pum_ctx* ctx, pum_hier* h, const double* r, double* z) {
  Level& L0 = h->lv[0];
  const int64_t N = (int64_t)L0.n * L0.d;
  if (is_mixed(h, 0) && h->lv.size() > 1) {
    vcycle_mixed(ctx, h, 0, r, z);
    return;
  }
  convert_vec(ctx, L0.b, L0.vdt, r, PUM_F64, N);
  vcycle_level(ctx, h, 0);
  convert_vec(ctx, z, PUM_F64, L0.x, L0.vdt, N);
}

static void build_vcycle_graph(pum_ctx* ctx, pum_hier* h, const double* r, double* z) {
  GraphCache& g = h->vgraph;
  graph_destroy(g);
  cudaGraph_t graph = nullptr;
  const int64_t l0 = ctx->launches;
  PUM_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  ctx->capture_ev = &g.ev;
  try {
    vcycle_body(ctx, h, r, z);
  } catch (...) {
    ctx->capture_ev = nullptr;
    cudaStreamEndCapture(ctx->stream, &graph);
    if (graph) cudaGraphDestroy(graph);
    ctx->launches = l0;
    throw;
  }
  ctx->capture_ev = nullptr;
  PUM_CUDA(cudaStreamEndCapture(ctx->stream, &graph));
  g.kernels = ctx->launches - l0;
  ctx->launches = l0;  // counted per replay
  const cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  PUM_CUDA(e);
  g.timed = ctx->timing;
  g.r = r;
  g.z = z;
}

// z = B r: replayed from a graph captured for these (r, z) on capturable streams.
static void vcycle64(pum_ctx* ctx, pum_hier* h, const double* r, double* z) {
  if (!capturable(ctx)) {
    vcycle_body(ctx, h, r, z);
    return;
  }
  graph_harvest(ctx, h);
  GraphCache& g = h->vgraph;
  if (!g.exec || g.timed != ctx->timing || g.r != r || g.z != z) build_vcycle_graph(ctx, h, r, z);
  PUM_CUDA(cudaGraphLaunch(g.exec, ctx->stream));
  ctx->launches += g.kernels;
  g.pending = g.timed != 0;
}

void vcycle_apply_impl(pum_ctx* ctx, pum_hier* h, const double* r, double* z) {
  vcycle64(ctx, h, r, z);
  if (ctx->timing) graph_harvest(ctx, h);  // timing mode: collect before returning
}

// Device status word after the stream has drained: a kernel that recorded an error (a bounded
// wait that expired) turns into that status.
static void check_device_status(pum_ctx* ctx) {
  DevStatus st{};
  PUM_CUDA(cudaMemcpyAsync(&st, ctx->status, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream));
  PUM_CUDA(cudaStreamSynchronize(ctx->stream));
  if (!st.code) return;
  PUM_CUDA(cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), ctx->stream));
  throw Error{(pum_status)st.code, "device status " + std::to_string(st.code) + " in kernel family " +
                                       std::to_string(st.where) + " at " + std::to_string(st.info)};
}

pum_status pcg_impl(pum_ctx* ctx, pum_hier* h, const double* b, double* x, pcg_report* rep) {
  Level& L0 = h->lv[0];
  const int64_t N = (int64_t)L0.n * L0.d;
  cudaStream_t s = ctx->stream;
  double *r = h->w64[0], *z = h->w64[1], *p = h->w64[2], *q = h->w64[3], *zo = h->w64[4];
  const int grid = (int)std::min<int64_t>((N + 255) / 256, 1024);
  const unsigned mvgrid = (unsigned)((N + 255) / 256);
  PUM_CHECK(mvgrid <= (1u << 16), PUM_ERR_UNSUPPORTED, "PCG: problem too large for the partial buffer");
  PUM_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * N, s));
  PUM_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  dot(ctx, b, b, N, S_BB);
  PUM_CUDA(cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double) * 8, cudaMemcpyDeviceToHost, s));
  PUM_CUDA(cudaStreamSynchronize(s));
  const double nb = std::sqrt(ctx->h_scal[S_BB]);
  rep->iters = 0;
  rep->converged = 0;
  rep->final_relres = 1.0;
  if (rep->hist && rep->maxit >= 0) rep->hist[0] = 1.0;
  if (nb == 0.0) {
    rep->converged = 1;
    rep->final_relres = 0.0;
    return PUM_OK;
  }
  vcycle64(ctx, h, r, z);
  dot(ctx, r, z, N, S_RZ);
  PUM_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  for (int it = 1; it <= rep->maxit; ++it) {
    EpiArgs e{};
    e.y = q;
    e.partials = ctx->partials;
    bsr_mv(ctx, L0.A, PUM_F64, p, EPI_DOT, e, PUM_TK_PCG_AP);  // q = A p, partials of p.q
    reduce_partials(ctx, (int)mvgrid, S_PQ);
    k_pcg_xr<<<grid, 256, 0, s>>>(x, r, p, q, ctx->scal, N, ctx->partials);
    count_launch(ctx);
    reduce_partials(ctx, grid, S_RR);
    PUM_CUDA(cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double) * 8, cudaMemcpyDeviceToHost, s));
    PUM_CUDA(cudaStreamSynchronize(s));
    const double pq = ctx->h_scal[S_PQ], rr = ctx->h_scal[S_RR], rz = ctx->h_scal[S_RZ];
    if (!(pq > 0.0) || !std::isfinite(rr) || !std::isfinite(rz)) {
      rep->iters = it;
      check_device_status(ctx);
      throw Error{PUM_ERR_BREAKDOWN, "PCG breakdown: p^T A p = " + std::to_string(pq) + ", r^T z = " +
                                         std::to_string(rz)};
    }
    const double rel = std::sqrt(rr) / nb;
    if (rep->hist) rep->hist[it] = rel;
    rep->iters = it;
    rep->final_relres = rel;
    if (rel <= rep->rtol) {
      rep->converged = 1;
      graph_harvest(ctx, h);
      check_device_status(ctx);
      return PUM_OK;
    }
    if (rep->flexible) PUM_CUDA(cudaMemcpyAsync(zo, z, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    vcycle64(ctx, h, r, z);
    dot(ctx, r, z, N, S_RZN);
    if (rep->flexible) dot(ctx, r, zo, N, S_RZO);
    k_pcg_p<<<grid, 256, 0, s>>>(p, z, ctx->scal, rep->flexible, N);
    k_scal_move<<<1, 1, 0, s>>>(ctx->scal, S_RZ, S_RZN);
    ctx->launches += 2;
    PUM_CUDA(cudaGetLastError());
  }
  graph_harvest(ctx, h);
  check_device_status(ctx);
  return PUM_ERR_NOCONV;
}


// ----------------------------------------------------------------------------- BiCGStab

// Device scalar slots of BiCGStab and of the convergence factor (after the PCG ones).
enum { B_RHO = 6, B_RHO_OLD = 7, B_ALPHA = 8, B_OMEGA = 9, B_RV = 10, B_TS = 11, B_TT = 12, B_SS = 13, B_RR = 14,
       B_E0 = 15, B_EN = 16 };

__global__ void k_bicg_init(double* scal) {
  scal[B_RHO_OLD] = 1.0;
  scal[B_ALPHA] = 1.0;
  scal[B_OMEGA] = 1.0;
}

// p = r + beta (p - omega v), beta = (rho / rho_old) (alpha / omega)
__global__ void k_bicg_p(double* __restrict__ p, const double* __restrict__ r, const double* __restrict__ v,
                         const double* __restrict__ scal, int64_t n) {
  const double beta = (scal[B_RHO] / scal[B_RHO_OLD]) * (scal[B_ALPHA] / scal[B_OMEGA]);
  const double omega = scal[B_OMEGA];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i] - omega * v[i], r[i]);
}

template <int NT>
__device__ __forceinline__ void block_partial(double sum, double* partials) {
  __shared__ double red[NT / 32];
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += red[w];
    partials[blockIdx.x] = t;
  }
}

// alpha = rho / (r^ . v); s = r - alpha v; partial sums of s . s
__global__ void k_bicg_s(double* __restrict__ s, const double* __restrict__ r, const double* __restrict__ v,
                         double* __restrict__ scal, int64_t n, double* __restrict__ partials) {
  const double alpha = scal[B_RHO] / scal[B_RV];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double si = fma(-alpha, v[i], r[i]);
    s[i] = si;
    acc = fma(si, si, acc);
  }
  block_partial<256>(acc, partials);
  if (blockIdx.x == 0 && threadIdx.x == 0) scal[B_ALPHA] = alpha;
}

// omega = (t . s) / (t . t); x += alpha ph + omega sh; r = s - omega t; partial sums of r . r
__global__ void k_bicg_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ ph,
                          const double* __restrict__ sh, const double* __restrict__ s, const double* __restrict__ t,
                          double* __restrict__ scal, int64_t n, double* __restrict__ partials) {
  const double alpha = scal[B_ALPHA];
  const double omega = scal[B_TS] / scal[B_TT];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(omega, sh[i], fma(alpha, ph[i], x[i]));
    const double ri = fma(-omega, t[i], s[i]);
    r[i] = ri;
    acc = fma(ri, ri, acc);
  }
  block_partial<256>(acc, partials);
  if (blockIdx.x == 0 && threadIdx.x == 0) scal[B_OMEGA] = omega;
}

// x += scal[slot] y (slot < 0: factor 1)
__global__ void k_axpy_slot(double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ scal,
                            int slot, int64_t n) {
  const double a = slot >= 0 ? scal[slot] : 1.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(a, y[i], x[i]);
}

static void ensure_wb(pum_hier* h, int64_t N) {
  for (auto& w : h->wb)
    if (!w && cudaMalloc(&w, sizeof(double) * N) != cudaSuccess) {
      cudaGetLastError();
      w = nullptr;
      throw Error{PUM_ERR_OOM, "Krylov work vectors: device allocation failed"};
    }
}

// z = B r through the fixed pair (vin, vout), so that the captured V-cycle graph is reused.
static void cycle_via(pum_ctx* ctx, pum_hier* h, const double* r, double* z, int64_t N) {
  double *vin = h->w64[0], *vout = h->w64[1];
  PUM_CUDA(cudaMemcpyAsync(vin, r, sizeof(double) * N, cudaMemcpyDeviceToDevice, ctx->stream));
  vcycle64(ctx, h, vin, vout);
  PUM_CUDA(cudaMemcpyAsync(z, vout, sizeof(double) * N, cudaMemcpyDeviceToDevice, ctx->stream));
}

pum_status bicgstab_impl(pum_ctx* ctx, pum_hier* h, const double* b, double* x, pcg_report* rep) {
  Level& L0 = h->lv[0];
  const int64_t N = (int64_t)L0.n * L0.d;
  cudaStream_t st = ctx->stream;
  ensure_wb(h, N);
  double *r = h->wb[0], *rhat = h->wb[1], *p = h->wb[2], *v = h->wb[3], *s = h->wb[4], *t = h->wb[5],
         *ph = h->wb[6], *sh = h->wb[7];
  const int grid = (int)std::min<int64_t>((N + 255) / 256, 1024);
  PUM_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * N, st));
  PUM_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  PUM_CUDA(cudaMemcpyAsync(rhat, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  PUM_CUDA(cudaMemsetAsync(p, 0, sizeof(double) * N, st));
  PUM_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * N, st));
  dot(ctx, b, b, N, S_BB);
  k_bicg_init<<<1, 1, 0, st>>>(ctx->scal);
  count_launch(ctx);
  PUM_CUDA(cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double) * kScalSlots, cudaMemcpyDeviceToHost, st));
  PUM_CUDA(cudaStreamSynchronize(st));
  const double nb = std::sqrt(ctx->h_scal[S_BB]);
  rep->iters = 0;
  rep->converged = 0;
  rep->final_relres = 1.0;
  if (rep->hist && rep->maxit >= 0) rep->hist[0] = 1.0;
  if (nb == 0.0) {
    rep->converged = 1;
    rep->final_relres = 0.0;
    return PUM_OK;
  }
  auto breakdown = [&](int it, const char* what) {
    rep->iters = it;
    check_device_status(ctx);
    return Error{PUM_ERR_BREAKDOWN, std::string("BiCGStab breakdown: ") + what};
  };
  for (int it = 1; it <= rep->maxit; ++it) {
    dot(ctx, rhat, r, N, B_RHO);
    k_bicg_p<<<grid, 256, 0, st>>>(p, r, v, ctx->scal, N);
    count_launch(ctx);
    cycle_via(ctx, h, p, ph, N);  // p^ = B p
    EpiArgs e{};
    e.y = v;
    bsr_mv(ctx, L0.A, PUM_F64, ph, EPI_SET, e);  // v = A p^
    dot(ctx, rhat, v, N, B_RV);
    k_bicg_s<<<grid, 256, 0, st>>>(s, r, v, ctx->scal, N, ctx->partials);
    count_launch(ctx);
    reduce_partials(ctx, grid, B_SS);
    PUM_CUDA(cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double) * kScalSlots, cudaMemcpyDeviceToHost, st));
    PUM_CUDA(cudaStreamSynchronize(st));
    const double rho = ctx->h_scal[B_RHO], rv = ctx->h_scal[B_RV];
    if (!(rho != 0.0 && rv != 0.0 && std::isfinite(rho) && std::isfinite(rv))) throw breakdown(it, "r^.r or r^.v");
    const double srel = std::sqrt(ctx->h_scal[B_SS]) / nb;
    if (srel <= rep->rtol) {  // the half step already converged: x += alpha p^
      k_axpy_slot<<<grid, 256, 0, st>>>(x, ph, ctx->scal, B_ALPHA, N);
      count_launch(ctx);
      if (rep->hist) rep->hist[it] = srel;
      rep->iters = it;
      rep->final_relres = srel;
      rep->converged = 1;
      graph_harvest(ctx, h);
      check_device_status(ctx);
      return PUM_OK;
    }
    cycle_via(ctx, h, s, sh, N);  // s^ = B s
    e.y = t;
    bsr_mv(ctx, L0.A, PUM_F64, sh, EPI_SET, e);  // t = A s^
    dot(ctx, t, s, N, B_TS);
    dot(ctx, t, t, N, B_TT);
    k_bicg_xr<<<grid, 256, 0, st>>>(x, r, ph, sh, s, t, ctx->scal, N, ctx->partials);
    count_launch(ctx);
    reduce_partials(ctx, grid, B_RR);
    k_scal_move<<<1, 1, 0, st>>>(ctx->scal, B_RHO_OLD, B_RHO);
    count_launch(ctx);
    PUM_CUDA(cudaGetLastError());
    PUM_CUDA(cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double) * kScalSlots, cudaMemcpyDeviceToHost, st));
    PUM_CUDA(cudaStreamSynchronize(st));
    const double tt = ctx->h_scal[B_TT], rr = ctx->h_scal[B_RR];
    if (!(tt > 0.0 && std::isfinite(rr))) throw breakdown(it, "t.t");
    const double rel = std::sqrt(rr) / nb;
    if (rep->hist) rep->hist[it] = rel;
    rep->iters = it;
    rep->final_relres = rel;
    if (rel <= rep->rtol) {
      rep->converged = 1;
      graph_harvest(ctx, h);
      check_device_status(ctx);
      return PUM_OK;
    }
  }
  graph_harvest(ctx, h);
  check_device_status(ctx);
  return PUM_ERR_NOCONV;
}

// rho_A of the stationary cycle: e_j = e_{j-1} + B (-A e_{j-1}), the energy ratio over n cycles.
double convergence_factor_impl(pum_ctx* ctx, pum_hier* h, const double* e0, int n_cycles) {
  Level& L0 = h->lv[0];
  const int64_t N = (int64_t)L0.n * L0.d;
  cudaStream_t st = ctx->stream;
  ensure_wb(h, N);
  double *e = h->wb[0], *q = h->wb[1], *zero = h->wb[2], *ar = h->wb[3], *z = h->wb[4];
  const unsigned mvgrid = (unsigned)((N + 255) / 256);
  PUM_CHECK(mvgrid <= (1u << 16), PUM_ERR_UNSUPPORTED, "convergence factor: problem too large for the partials");
  const int grid = (int)std::min<int64_t>((N + 255) / 256, 1024);
  PUM_CUDA(cudaMemcpyAsync(e, e0, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  PUM_CUDA(cudaMemsetAsync(zero, 0, sizeof(double) * N, st));
  auto energy = [&](int slot) {  // e^T A e
    EpiArgs d{};
    d.y = q;
    d.partials = ctx->partials;
    bsr_mv(ctx, L0.A, PUM_F64, e, EPI_DOT, d);
    reduce_partials(ctx, (int)mvgrid, slot);
  };
  energy(B_E0);
  for (int j = 0; j < n_cycles; ++j) {
    EpiArgs rs{};
    rs.y = ar;
    rs.b = zero;
    bsr_mv(ctx, L0.A, PUM_F64, e, EPI_RESID, rs);  // -A e
    cycle_via(ctx, h, ar, z, N);
    k_axpy_slot<<<grid, 256, 0, st>>>(e, z, ctx->scal, -1, N);
    count_launch(ctx);
  }
  energy(B_EN);
  PUM_CUDA(cudaGetLastError());
  PUM_CUDA(cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double) * kScalSlots, cudaMemcpyDeviceToHost, st));
  PUM_CUDA(cudaStreamSynchronize(st));
  graph_harvest(ctx, h);
  check_device_status(ctx);
  const double e0n = ctx->h_scal[B_E0], enn = ctx->h_scal[B_EN];
  PUM_CHECK(e0n > 0.0 && enn >= 0.0 && std::isfinite(enn), PUM_ERR_BREAKDOWN,
            "convergence factor: e^T A e not positive (e0 = 0, or A not SPD)");
  return std::pow(enn / e0n, 1.0 / (2.0 * n_cycles));
}

}  // namespace pum
