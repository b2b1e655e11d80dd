// C-ABI of the library: argument validation, hierarchy construction and set-up,
// persistence, and the exception-to-status boundary.  Every entry point catches all
// library errors and CUDA failures and returns a pum_status.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "pum_internal.cuh"

namespace pum {
void vcycle_apply_impl(pum_ctx* ctx, pum_hier* h, const double* r, double* z);
pum_status pcg_impl(pum_ctx* ctx, pum_hier* h, const double* b, double* x, pcg_report* rep);
pum_status bicgstab_impl(pum_ctx* ctx, pum_hier* h, const double* b, double* x, pcg_report* rep);
double convergence_factor_impl(pum_ctx* ctx, pum_hier* h, const double* e0, int n_cycles);
}  // namespace pum

using namespace pum;

int pum::level_vdt(const pum_hier* h, int l) {
  return (h->smooth_dt == PUM_F32 && l < h->sp.fp32_levels) ? PUM_F32 : PUM_F64;
}

int pum::level_gdt(const pum_hier* h, int l) { return level_vdt(h, l) == PUM_F32 ? h->g_dt : PUM_F64; }

namespace {

template <typename F>
pum_status guard(pum_ctx* ctx, F&& f) {
  try {
    if (ctx) {
      ctx->last_error.clear();
      PUM_CUDA(cudaSetDevice(ctx->device));
    }
    return f();
  } catch (const Error& e) {
    if (ctx) ctx->last_error = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->last_error = "host allocation failed";
    return PUM_ERR_OOM;
  } catch (...) {
    if (ctx) ctx->last_error = "unexpected internal error";
    return PUM_ERR_CUDA;
  }
}

// binom(p+2, 2) for p = 1..5 (the square's local spaces) and 20 = binom(6, 3) (the cube's, p = 3)
bool is_supported_bs(int d) { return d == 3 || d == 6 || d == 10 || d == 15 || d == 20 || d == 21; }

void check_vec(const void* p, const char* name) {
  PUM_CHECK(p != nullptr, PUM_ERR_INVALID_ARG, std::string(name) + " is NULL");
  PUM_CHECK(((uintptr_t)p & 15) == 0, PUM_ERR_INVALID_ARG, std::string(name) + " must be 16-byte aligned");
}

void check_level(const pum_hier* h, int level) {
  PUM_CHECK(h != nullptr, PUM_ERR_INVALID_ARG, "hierarchy is NULL");
  PUM_CHECK(level >= 0 && level < (int)h->lv.size(), PUM_ERR_INVALID_ARG, "level out of range");
}

void check_ready(const pum_hier* h) {
  PUM_CHECK(h != nullptr, PUM_ERR_INVALID_ARG, "hierarchy is NULL");
  PUM_CHECK(h->setup_done, PUM_ERR_INVALID_ARG, "bfsai_setup has not been run on this hierarchy");
}

void free_level(Level& L) {
  for (Bsr* m : {&L.A, &L.As, &L.P, &L.PT, &L.Ps, &L.PTs, &L.G, &L.GT, &L.G64, &L.F0, &L.F0T, &L.F064, &L.G164,
                 &L.A1, &L.G1, &L.G1T})
    bsr_free(*m);
  for (void** v : {&L.x, &L.b, &L.r, &L.p, &L.t, &L.u, &L.c, &L.e, (void**)&L.b64, (void**)&L.z64, &L.zs})
    if (*v) { cudaFree(*v); *v = nullptr; }
  sell_free(L.Adf);
  sell_free(L.Pdf);
  gg_free(L.gg);
}

void free_smoother(pum_hier* h) {
  graph_destroy(h->vgraph);
  multi_cache_free(h->multi);
  for (auto& L : h->lv) {
    for (Bsr* m : {&L.As, &L.PT, &L.Ps, &L.PTs, &L.G, &L.GT, &L.F0, &L.F0T, &L.G1, &L.G1T}) bsr_free(*m);
    for (void** v : {&L.x, &L.b, &L.r, &L.p, &L.t, &L.u, &L.c, &L.e, (void**)&L.b64, (void**)&L.z64, &L.zs})
      if (*v) { cudaFree(*v); *v = nullptr; }
    sell_free(L.Adf);
    sell_free(L.Pdf);
    gg_free(L.gg);
  }
  for (auto& w : h->w64)
    if (w) { cudaFree(w); w = nullptr; }
  for (auto& w : h->wb)
    if (w) { cudaFree(w); w = nullptr; }
  h->setup_done = false;
}

// Copy a caller BSR into the library's padded FP64 layout (validating the pattern).
void import_bsr(Bsr& dst, const pum_bsr_view& v, cudaStream_t s) {
  PUM_CHECK(v.n_brows >= 0 && v.n_bcols >= 0 && v.nnzb >= 0, PUM_ERR_INVALID_ARG, "negative BSR sizes");
  PUM_CHECK(is_supported_bs(v.bs), PUM_ERR_UNSUPPORTED, "block size must be 3, 6, 10, 15 or 21");
  PUM_CHECK(v.row_ptr && (v.nnzb == 0 || (v.col_idx && v.vals)), PUM_ERR_INVALID_ARG, "NULL BSR array");
  std::vector<int> rp(v.n_brows + 1), ci(v.nnzb);
  const cudaMemcpyKind kind = v.on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  PUM_CUDA(cudaMemcpy(rp.data(), v.row_ptr, sizeof(int) * rp.size(), kind));
  if (v.nnzb) PUM_CUDA(cudaMemcpy(ci.data(), v.col_idx, sizeof(int) * ci.size(), kind));
  PUM_CHECK(rp[0] == 0 && rp.back() == (int)v.nnzb, PUM_ERR_INVALID_ARG, "row_ptr must start at 0 and end at nnzb");
  for (int i = 0; i < v.n_brows; ++i) {
    PUM_CHECK(rp[i + 1] >= rp[i], PUM_ERR_INVALID_ARG, "row_ptr must be non-decreasing");
    for (int b = rp[i]; b < rp[i + 1]; ++b) {
      PUM_CHECK(ci[b] >= 0 && ci[b] < v.n_bcols, PUM_ERR_INVALID_ARG, "column index out of range");
      PUM_CHECK(b == rp[i] || ci[b] > ci[b - 1], PUM_ERR_INVALID_ARG, "columns must be sorted and unique per row");
    }
  }
  bsr_alloc(dst, v.n_brows, v.n_bcols, v.bs, PUM_F64, rp, ci);
  const size_t dd = (size_t)v.bs * v.bs;
  if (v.nnzb)
    PUM_CUDA(cudaMemcpy2DAsync(dst.vals, sizeof(double) * dst.stride, v.vals, sizeof(double) * dd, sizeof(double) * dd,
                               (size_t)v.nnzb, v.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  PUM_CUDA(cudaStreamSynchronize(s));
}

void galerkin(pum_ctx* ctx, Level& fine, Level& coarse) {
  Bsr PT, AP;
  bsr_transpose(PT, fine.P, ctx->stream);
  spgemm(AP, fine.A, fine.P, ctx->stream);
  spgemm(coarse.A, PT, AP, ctx->stream);
  bsr_free(PT);
  bsr_free(AP);
}

void* dalloc(size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    throw Error{PUM_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
  }
  return p;
}

// Everything the hot path needs once G (or F0/G1) exist in FP64: precision copies,
// transposes, work vectors, Chebyshev mu sequence.
void finalize_smoother(pum_ctx* ctx, pum_hier* h) {
  cudaStream_t s = ctx->stream;
  const int nl = (int)h->lv.size();
  for (int l = 0; l < nl; ++l) {
    Level& L = h->lv[l];
    L.vdt = level_vdt(h, l);
    L.gdt = level_gdt(h, l);
    const int vdt = L.vdt;
    const size_t vs = dt_size(vdt);
    const size_t N = (size_t)L.n * L.d;
    if (l + 1 < nl) {
      bsr_transpose(L.PT, L.P, s);
      if (vdt == PUM_F32) {
        bsr_convert(L.Ps, L.P, PUM_F32, s);
        bsr_convert(L.PTs, L.PT, PUM_F32, s);
      }
      if (h->fp.nested) {
        bsr_convert(L.F0, L.F064, L.gdt, s);
        bsr_convert(L.G1, L.G164, L.gdt, s);
        bsr_transpose(L.F0T, L.F0, s);
        bsr_transpose(L.G1T, L.G1, s);
      } else {
        bsr_convert(L.G, L.G64, L.gdt, s);
        bsr_transpose(L.GT, L.G, s);
      }
    }
    if (vdt == PUM_F32) bsr_convert(L.As, L.A, PUM_F32, s);
    if (vdt == PUM_F32 && h->sell) {
      // The factor next to the Chebyshev update's input (G, or the inner G1 of the nested chain)
      // is applied through the fused layout when it fits; its two sliced copies are then unused.
      Bsr* fg = h->fp.nested ? &L.G1 : &L.G;
      Bsr* fgt = h->fp.nested ? &L.G1T : &L.GT;
      if (h->fused_fsai && !fg->empty() && fg->n_brows >= kSellMinRows) gg_build(ctx, L.gg, *fg);
      for (Bsr* m : {&L.As, &L.G, &L.GT, &L.F0, &L.F0T, &L.G1, &L.G1T, &L.Ps, &L.PTs})
        if (!m->empty() && m->n_brows >= kSellMinRows && !(L.gg.S.R > 0 && (m == fg || m == fgt)))
          sell_build(*m, s, ctx->sm_count);
    }
    for (void** v : {&L.x, &L.b, &L.r, &L.p, &L.t, &L.u, &L.c, &L.e}) *v = dalloc(vs * N);
    if (h->smooth_dt == PUM_F32 && l > 0 && (l < h->sp.mixed_levels || l == nl - 1)) {
      L.b64 = (double*)dalloc(sizeof(double) * N);
      L.z64 = (double*)dalloc(sizeof(double) * N);
    }
    auto df_level = [&](int m) {  // mixed level on the sliced layout: double-float residuals
      return level_vdt(h, m) == PUM_F32 && h->sell && m < h->sp.mixed_levels && m + 1 < nl &&
             h->lv[m].n >= kSellMinRows;
    };
    if (df_level(l)) {
      sell_build_df(L.Adf, L.A, s, ctx->sm_count);  // accurate residuals in double-float arithmetic
      L.zs = dalloc(sizeof(float) * 2 * N);
      if (df_level(l + 1)) sell_build_df(L.Pdf, L.P, s, ctx->sm_count);  // z += P z_c from the split z_c
    }
    PUM_CUDA(cudaMemsetAsync(L.x, 0, vs * N, s));
  }
  const size_t N0 = (size_t)h->lv[0].n * h->lv[0].d;
  for (auto& w : h->w64) w = (double*)dalloc(sizeof(double) * N0);
  const int steps = h->sp.cycle == PUM_CYCLE_V2K0 ? 2 * h->sp.degree_k : h->sp.degree_k;
  h->mu.assign(steps, 0.0);
  double mu = 1.0 / 3.0;  // Algorithm 3: mu_1 = 1/3, mu_{i+1} = 1 / (2 - mu_i), whatever the degree
  for (int i = 0; i < steps; ++i) {
    h->mu[i] = mu;
    mu = 1.0 / (2.0 - mu);
  }
  PUM_CUDA(cudaStreamSynchronize(s));
  h->setup_done = true;
}

void check_params(const bfsai_params* fp, const smoother_params* sp) {
  PUM_CHECK(fp && sp, PUM_ERR_INVALID_ARG, "NULL parameters");
  PUM_CHECK(fp->p0 == PUM_P0_LOWER || fp->p0 == PUM_P0_DIAG, PUM_ERR_INVALID_ARG, "p0 must be LOWER or DIAG");
  PUM_CHECK(fp->adaptive >= 0 && fp->adaptive <= 2, PUM_ERR_INVALID_ARG, "adaptive must be 0, 1 or 2");
  PUM_CHECK(!fp->adaptive || (fp->t_max >= 1 && fp->tau > 0.0 && fp->tau <= 1.0), PUM_ERR_INVALID_ARG,
            "adaptive FSAI needs t_max >= 1 and tau in (0, 1]");
  PUM_CHECK(!(fp->adaptive == 2 && fp->nested), PUM_ERR_INVALID_ARG, "the learned pattern is not for nested FSAI");
  PUM_CHECK(fp->tie_rel >= 0.0, PUM_ERR_INVALID_ARG, "tie_rel must be >= 0");
  PUM_CHECK(sp->degree_k >= 1 && sp->degree_k <= 64, PUM_ERR_INVALID_ARG, "degree_k must be in 1..64");
  PUM_CHECK(sp->lanczos_its >= 1 && sp->lanczos_safety >= 1.0, PUM_ERR_INVALID_ARG, "Lanczos parameters");
  PUM_CHECK(sp->fp32_levels >= 0, PUM_ERR_INVALID_ARG, "fp32_levels must be >= 0");
  PUM_CHECK(sp->smoother == PUM_SMOOTHER_CHEB4 || sp->smoother == PUM_SMOOTHER_RICHARDSON, PUM_ERR_INVALID_ARG,
            "smoother must be PUM_SMOOTHER_CHEB4 or PUM_SMOOTHER_RICHARDSON");
  PUM_CHECK(sp->cycle == PUM_CYCLE_VKK || sp->cycle == PUM_CYCLE_V2K0, PUM_ERR_INVALID_ARG,
            "cycle must be PUM_CYCLE_VKK or PUM_CYCLE_V2K0");
  PUM_CHECK(sp->mixed_levels >= 0, PUM_ERR_INVALID_ARG, "mixed_levels must be >= 0");
  PUM_CHECK(sp->smooth_dt == PUM_F64 || sp->smooth_dt == PUM_F32, PUM_ERR_INVALID_ARG, "smooth_dt must be F64 or F32");
  PUM_CHECK(sp->g_dt == PUM_F64 || sp->g_dt == PUM_F32 || sp->g_dt == PUM_BF16, PUM_ERR_INVALID_ARG, "g_dt");
  PUM_CHECK(!(sp->smooth_dt == PUM_F64 && sp->g_dt != PUM_F64), PUM_ERR_INVALID_ARG,
            "a float64 smoother needs float64 G");
  PUM_CHECK(!(sp->smooth_dt == PUM_F32 && sp->g_dt == PUM_F64), PUM_ERR_INVALID_ARG,
            "a float32 smoother stores G in float32 or bf16");
}

const Bsr* select_matrix(const pum_hier* h, int level, int which) {
  const Level& L = h->lv[level];
  switch (which) {
    case PUM_MAT_A: return &L.A;
    case PUM_MAT_P: return &L.P;
    case PUM_MAT_G: return &L.G64;
    case PUM_MAT_F0: return &L.F064;
    case PUM_MAT_G1: return &L.G164;
    case PUM_MAT_A1: return &L.A1;
    default: return nullptr;
  }
}

// ---- persistence helpers
const uint32_t kMagic = 0x484D5550u;  // "PUMH"
const uint32_t kVersion = 3;

void wr(FILE* f, const void* p, size_t n) {
  PUM_CHECK(n == 0 || fwrite(p, 1, n, f) == n, PUM_ERR_IO, "write failed");
}
void rd(FILE* f, void* p, size_t n) {
  PUM_CHECK(n == 0 || fread(p, 1, n, f) == n, PUM_ERR_IO, "file truncated or unreadable");
}

void save_bsr(FILE* f, pum_ctx* ctx, const Bsr& m) {
  int32_t hdr[4] = {m.n_brows, m.n_bcols, m.d, m.empty() ? 0 : 1};
  wr(f, hdr, sizeof(hdr));
  if (m.empty()) return;
  int64_t nnzb = m.nnzb;
  wr(f, &nnzb, sizeof(nnzb));
  wr(f, m.h_row_ptr.data(), sizeof(int) * m.h_row_ptr.size());
  wr(f, m.h_col_idx.data(), sizeof(int) * m.h_col_idx.size());
  auto v = bsr_values_host(m, ctx->stream);
  wr(f, v.data(), sizeof(double) * v.size());
}

void load_bsr(FILE* f, pum_ctx* ctx, Bsr& m) {
  int32_t hdr[4];
  rd(f, hdr, sizeof(hdr));
  if (!hdr[3]) return;
  int64_t nnzb;
  rd(f, &nnzb, sizeof(nnzb));
  PUM_CHECK(hdr[0] >= 0 && hdr[1] >= 0 && nnzb >= 0 && is_supported_bs(hdr[2]) && nnzb < (1LL << 31), PUM_ERR_IO,
            "corrupt matrix header");
  std::vector<int> rp(hdr[0] + 1), ci(nnzb);
  rd(f, rp.data(), sizeof(int) * rp.size());
  rd(f, ci.data(), sizeof(int) * ci.size());
  std::vector<double> v((size_t)nnzb * hdr[2] * hdr[2]);
  rd(f, v.data(), sizeof(double) * v.size());
  pum_bsr_view view{hdr[0], hdr[1], hdr[2], nnzb, rp.data(), ci.data(), v.data(), 0};
  import_bsr(m, view, ctx->stream);
}

}  // namespace

// ============================================================================= C-ABI

extern "C" {

pum_status pum_create(pum_ctx** out, int device, void* cuda_stream) {
  if (!out) return PUM_ERR_INVALID_ARG;
  *out = nullptr;
  pum_ctx* ctx = new (std::nothrow) pum_ctx();
  if (!ctx) return PUM_ERR_OOM;
  ctx->device = device;
  const pum_status st = guard(ctx, [&]() {
    int n = 0;
    PUM_CUDA(cudaGetDeviceCount(&n));
    PUM_CHECK(device >= 0 && device < n, PUM_ERR_INVALID_ARG, "no such CUDA device");
    PUM_CUDA(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device));
    if (cuda_stream) {
      ctx->stream = (cudaStream_t)cuda_stream;
    } else {
      PUM_CUDA(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
      ctx->own_stream = true;
    }
    const char* ng = getenv("PUM_NO_GRAPH");
    ctx->graphs = !(ng && ng[0] == '1');
    const char* ns = getenv("PUM_NO_SELL");
    ctx->sell = !(ns && ns[0] == '1');
    const char* np = getenv("PUM_NO_PDL");
    ctx->pdl = !(np && np[0] == '1');
    const char* nf = getenv("PUM_NO_FUSED_FSAI");
    ctx->fused_fsai = !(nf && nf[0] == '1');
    const char* as = getenv("PUM_ADAPT_STEPS");
    ctx->adapt_steps = as && as[0] == '1';
    ctx->status = (DevStatus*)dalloc(sizeof(DevStatus));
    ctx->scal = (double*)dalloc(sizeof(double) * kScalSlots);
    ctx->partials = (double*)dalloc(sizeof(double) * (1 << 16));
    PUM_CUDA(cudaMemset(ctx->status, 0, sizeof(DevStatus)));
    PUM_CUDA(cudaMemset(ctx->scal, 0, sizeof(double) * kScalSlots));
    PUM_CUDA(cudaStreamSynchronize(0));  // legacy-stream memsets, before the context's own stream runs
    PUM_CUDA(cudaMallocHost(&ctx->h_scal, sizeof(double) * kScalSlots));
    return PUM_OK;
  });
  if (st != PUM_OK) {
    pum_destroy(ctx);
    return st;
  }
  *out = ctx;
  return PUM_OK;
}

pum_status pum_destroy(pum_ctx* ctx) {
  if (!ctx) return PUM_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (int k = 0; k < PUM_TK_COUNT; ++k) {
    for (auto e : ctx->tk_start[k]) cudaEventDestroy(e);
    for (auto e : ctx->tk_stop[k]) cudaEventDestroy(e);
  }
  if (ctx->status) cudaFree(ctx->status);
  if (ctx->scal) cudaFree(ctx->scal);
  if (ctx->partials) cudaFree(ctx->partials);
  if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx->model;
  delete ctx;
  return PUM_OK;
}

const char* pum_last_error(const pum_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "NULL context"; }

pum_status pum_sync(pum_ctx* ctx) {
  if (!ctx) return PUM_ERR_INVALID_ARG;
  return guard(ctx, [&]() {
    PUM_CUDA(cudaStreamSynchronize(ctx->stream));
    DevStatus st{};
    PUM_CUDA(cudaMemcpy(&st, ctx->status, sizeof(st), cudaMemcpyDeviceToHost));
    if (st.code) {
      PUM_CUDA(cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), ctx->stream));
      throw Error{(pum_status)st.code, "device status " + std::to_string(st.code) + " at row " + std::to_string(st.info)};
    }
    return PUM_OK;
  });
}

pum_status pum_assemble(pum_ctx* ctx, const pum_problem* pr, pum_hier** out, double* b_dev) {
  if (!ctx || !pr || !out) return PUM_ERR_INVALID_ARG;
  *out = nullptr;
  pum_hier* h = new (std::nothrow) pum_hier();
  if (!h) return PUM_ERR_OOM;
  const pum_status st = guard(ctx, [&]() {
    PUM_CHECK(pr->equation == 4 || pr->equation == 6, PUM_ERR_INVALID_ARG, "equation must be 4 or 6");
    PUM_CHECK(pr->p >= 1 && pr->p <= 5, PUM_ERR_INVALID_ARG, "p must be in 1..5");
    PUM_CHECK(pr->finest_m >= 1 && pr->n_levels >= 1 && pr->n_levels <= 16, PUM_ERR_INVALID_ARG, "sizes");
    PUM_CHECK(pr->finest_m % (1 << (pr->n_levels - 1)) == 0, PUM_ERR_INVALID_ARG,
              "finest_m must be divisible by 2^(n_levels-1)");
    PUM_CHECK(pr->quad_pts >= 0 && pr->quad_pts <= 32, PUM_ERR_INVALID_ARG, "quad_pts must be in 0..32");
    PUM_CHECK(!pr->f_coef || (pr->f_modes >= 1 && pr->f_modes <= 64), PUM_ERR_INVALID_ARG, "f_modes");
    PUM_CHECK((int64_t)pr->finest_m * pr->finest_m * 9 < (1LL << 31), PUM_ERR_UNSUPPORTED, "too many blocks");
    if (b_dev) check_vec(b_dev, "b");
    h->lv.resize(pr->n_levels);
    assemble_finest(ctx, *pr, h->lv[0], b_dev);
    for (int l = 1; l < pr->n_levels; ++l) {
      Level& F = h->lv[l - 1];
      Level& C = h->lv[l];
      build_prolongation(ctx, F.m, pr->p, pr->quad_pts, F);
      C.m = F.m / 2;
      C.n = C.m * C.m;
      C.d = F.d;
      galerkin(ctx, F, C);
    }
    PUM_CUDA(cudaStreamSynchronize(ctx->stream));  // the hierarchy may next be used from another context
    return PUM_OK;
  });
  if (st != PUM_OK) {
    pum_hier_destroy(h);
    return st;
  }
  *out = h;
  return PUM_OK;
}

pum_status pum_hier_from_bsr(pum_ctx* ctx, int n_levels, const pum_bsr_view* A, const pum_bsr_view* P,
                             pum_hier** out) {
  if (!ctx || !A || !out || n_levels < 1 || (n_levels > 1 && !P)) return PUM_ERR_INVALID_ARG;
  *out = nullptr;
  pum_hier* h = new (std::nothrow) pum_hier();
  if (!h) return PUM_ERR_OOM;
  const pum_status st = guard(ctx, [&]() {
    h->lv.resize(n_levels);
    for (int l = 0; l < n_levels; ++l) {
      Level& L = h->lv[l];
      if (l > 0) {
        const pum_bsr_view& pv = P[l - 1];
        PUM_CHECK(pv.n_brows == h->lv[l - 1].n && pv.bs == h->lv[l - 1].d, PUM_ERR_INVALID_ARG,
                  "P[l] must have n_l block rows and the same block size");
        import_bsr(h->lv[l - 1].P, pv, ctx->stream);
        L.n = pv.n_bcols;
        L.d = pv.bs;
      }
      if (l == 0 || A[l].vals) {
        PUM_CHECK(A[l].n_brows == A[l].n_bcols, PUM_ERR_INVALID_ARG, "A must be square");
        PUM_CHECK(l == 0 || (A[l].n_brows == L.n && A[l].bs == L.d), PUM_ERR_INVALID_ARG,
                  "A[l] size does not match P[l-1]");
        import_bsr(L.A, A[l], ctx->stream);
        L.n = A[l].n_brows;
        L.d = A[l].bs;
      } else {
        galerkin(ctx, h->lv[l - 1], L);
      }
      L.m = (int)std::lround(std::sqrt((double)L.n));
      if (L.m * L.m != L.n) L.m = 0;
    }
    PUM_CUDA(cudaStreamSynchronize(ctx->stream));  // the hierarchy may next be used from another context
    return PUM_OK;
  });
  if (st != PUM_OK) {
    pum_hier_destroy(h);
    return st;
  }
  *out = h;
  return PUM_OK;
}

pum_status bfsai_setup(pum_ctx* ctx, pum_hier* h, const bfsai_params* fp, const smoother_params* sp) {
  if (!ctx || !h) return PUM_ERR_INVALID_ARG;
  return guard(ctx, [&]() {
    check_params(fp, sp);
    PUM_CHECK(fp->adaptive != 2 || ctx->model, PUM_ERR_INVALID_ARG,
              "adaptive = 2 needs a pattern model (pum_set_pattern_model)");
    PUM_CUDA(cudaStreamSynchronize(ctx->stream));  // no queued kernel may still use what is freed next
    free_smoother(h);
    for (auto& L : h->lv)
      for (Bsr* m : {&L.G64, &L.F064, &L.G164, &L.A1}) bsr_free(*m);
    h->fp = *fp;
    h->sp = *sp;
    h->smooth_dt = sp->smooth_dt;
    h->g_dt = sp->g_dt;
    h->sell = ctx->sell;
    h->fused_fsai = ctx->fused_fsai;
    const int nl = (int)h->lv.size();
    PUM_CHECK(h->lv.back().n * h->lv.back().d <= 4096, PUM_ERR_UNSUPPORTED, "coarsest level above 4096 unknowns");
    PUM_CHECK(sp->smooth_dt == PUM_F64 || sp->fp32_levels >= nl || sp->fp32_levels <= sp->mixed_levels,
              PUM_ERR_INVALID_ARG, "fp32_levels below the level count needs fp32_levels <= mixed_levels");
    for (int l = 0; l + 1 < nl; ++l) {
      try {
        fsai_setup_level(ctx, h, l);
        lanczos_level(ctx, h, l);
      } catch (const Error& e) {
        throw Error{e.st, "level " + std::to_string(l) + ": " + e.msg};
      }
    }
    coarse_factor(ctx, h);
    finalize_smoother(ctx, h);
    return PUM_OK;
  });
}

pum_status cheb4_smooth(pum_ctx* ctx, pum_hier* h, int level, const double* b, double* x, int x_is_zero) {
  if (!ctx) return PUM_ERR_INVALID_ARG;
  return guard(ctx, [&]() {
    check_ready(h);
    check_level(h, level);
    PUM_CHECK(level + 1 < (int)h->lv.size(), PUM_ERR_INVALID_ARG, "the coarsest level has no smoother");
    check_vec(b, "b");
    check_vec(x, "x");
    Level& L = h->lv[level];
    const int64_t N = (int64_t)L.n * L.d;
    convert_vec(ctx, L.b, L.vdt, b, PUM_F64, N);
    if (!x_is_zero) convert_vec(ctx, L.x, L.vdt, x, PUM_F64, N);
    cheb4(ctx, h, level, L.b, L.x, x_is_zero != 0, nullptr, -1, false);
    convert_vec(ctx, x, PUM_F64, L.x, L.vdt, N);
    return PUM_OK;
  });
}

pum_status vcycle_apply(pum_ctx* ctx, pum_hier* h, const double* r, double* z) {
  if (!ctx) return PUM_ERR_INVALID_ARG;
  return guard(ctx, [&]() {
    check_ready(h);
    check_vec(r, "r");
    check_vec(z, "z");
    vcycle_apply_impl(ctx, h, r, z);
    return PUM_OK;
  });
}

pum_status pcg_solve(pum_ctx* ctx, pum_hier* h, const double* b, double* x, pcg_report* rep) {
  if (!ctx) return PUM_ERR_INVALID_ARG;
  return guard(ctx, [&]() {
    check_ready(h);
    check_vec(b, "b");
    check_vec(x, "x");
    PUM_CHECK(rep && rep->maxit >= 0 && rep->rtol >= 0.0, PUM_ERR_INVALID_ARG, "pcg_report");
    const pum_status st = pcg_impl(ctx, h, b, x, rep);
    PUM_CUDA(cudaStreamSynchronize(ctx->stream));
    if (st == PUM_ERR_NOCONV) ctx->last_error = "PCG reached maxit before rtol";
    return st;
  });
}

pum_status bicgstab_solve(pum_ctx* ctx, pum_hier* h, const double* b, double* x, pcg_report* rep) {
  if (!ctx) return PUM_ERR_INVALID_ARG;
  return guard(ctx, [&]() {
    check_ready(h);
    check_vec(b, "b");
    check_vec(x, "x");
    PUM_CHECK(rep && rep->maxit >= 0 && rep->rtol >= 0.0, PUM_ERR_INVALID_ARG, "pcg_report");
    const pum_status st = bicgstab_impl(ctx, h, b, x, rep);
    PUM_CUDA(cudaStreamSynchronize(ctx->stream));
    if (st == PUM_ERR_NOCONV) ctx->last_error = "BiCGStab reached maxit before rtol";
    return st;
  });
}

pum_status pum_convergence_factor(pum_ctx* ctx, pum_hier* h, const double* e0, int n_cycles, double* rho) {
  if (!ctx) return PUM_ERR_INVALID_ARG;
  return guard(ctx, [&]() {
    check_ready(h);
    check_vec(e0, "e0");
    PUM_CHECK(rho != nullptr && n_cycles >= 1, PUM_ERR_INVALID_ARG, "n_cycles >= 1 and a rho pointer");
    *rho = convergence_factor_impl(ctx, h, e0, n_cycles);
    return PUM_OK;
  });
}

pum_status pum_residual(pum_ctx* ctx, pum_hier* h, int level, const double* b, const double* x, double* r) {
  if (!ctx) return PUM_ERR_INVALID_ARG;
  return guard(ctx, [&]() {
    check_level(h, level);
    check_vec(b, "b");
    check_vec(x, "x");
    check_vec(r, "r");
    EpiArgs e{};
    e.y = r;
    e.b = b;
    bsr_mv(ctx, h->lv[level].A, PUM_F64, x, EPI_RESID, e);
    return PUM_OK;
  });
}

pum_status pum_fsai_apply(pum_ctx* ctx, pum_hier* h, int level, const double* r, double* z) {
  if (!ctx) return PUM_ERR_INVALID_ARG;
  return guard(ctx, [&]() {
    check_ready(h);
    check_level(h, level);
    PUM_CHECK(level + 1 < (int)h->lv.size(), PUM_ERR_INVALID_ARG, "the coarsest level has no FSAI");
    check_vec(r, "r");
    check_vec(z, "z");
    Level& L = h->lv[level];
    const int64_t N = (int64_t)L.n * L.d;
    convert_vec(ctx, L.r, L.vdt, r, PUM_F64, N);
    apply_M(ctx, h, level, L.r, L.p, -1);
    convert_vec(ctx, z, PUM_F64, L.p, L.vdt, N);
    return PUM_OK;
  });
}

pum_status pum_restrict(pum_ctx* ctx, pum_hier* h, int level, const double* r, double* rc) {
  if (!ctx) return PUM_ERR_INVALID_ARG;
  return guard(ctx, [&]() {
    check_level(h, level);
    PUM_CHECK(level + 1 < (int)h->lv.size(), PUM_ERR_INVALID_ARG, "no coarser level");
    check_vec(r, "r");
    check_vec(rc, "rc");
    Level& L = h->lv[level];
    Bsr PT;
    const Bsr* use = &L.PT;
    if (L.PT.empty()) {
      bsr_transpose(PT, L.P, ctx->stream);
      use = &PT;
    }
    EpiArgs e{};
    e.y = rc;
    bsr_mv(ctx, *use, PUM_F64, r, EPI_SET, e);
    if (!PT.empty()) {
      PUM_CUDA(cudaStreamSynchronize(ctx->stream));
      bsr_free(PT);
    }
    return PUM_OK;
  });
}

pum_status pum_prolong_add(pum_ctx* ctx, pum_hier* h, int level, const double* e_, double* x) {
  if (!ctx) return PUM_ERR_INVALID_ARG;
  return guard(ctx, [&]() {
    check_level(h, level);
    PUM_CHECK(level + 1 < (int)h->lv.size(), PUM_ERR_INVALID_ARG, "no coarser level");
    check_vec(e_, "e");
    check_vec(x, "x");
    EpiArgs e{};
    e.y = x;
    bsr_mv(ctx, h->lv[level].P, PUM_F64, e_, EPI_ADD, e);
    return PUM_OK;
  });
}

pum_status pum_coarse_solve(pum_ctx* ctx, pum_hier* h, const double* r, double* z) {
  if (!ctx) return PUM_ERR_INVALID_ARG;
  return guard(ctx, [&]() {
    check_ready(h);
    check_vec(r, "r");
    check_vec(z, "z");
    coarse_solve(ctx, h, r, z, PUM_F64);
    return PUM_OK;
  });
}

pum_status pum_hier_levels(const pum_hier* h, int* n_levels) {
  if (!h || !n_levels) return PUM_ERR_INVALID_ARG;
  *n_levels = (int)h->lv.size();
  return PUM_OK;
}

pum_status pum_level_info_get(const pum_hier* h, int level, pum_level_info* info) {
  if (!h || !info || level < 0 || level >= (int)h->lv.size()) return PUM_ERR_INVALID_ARG;
  const Level& L = h->lv[level];
  std::memset(info, 0, sizeof(*info));
  info->m = L.m;
  info->n = L.n;
  info->d = L.d;
  info->nnzb_A = L.A.nnzb;
  info->nnzb_G = L.G64.nnzb;
  info->nnzb_GT = L.GT.nnzb;
  info->nnzb_P = L.P.nnzb;
  info->nnzb_F0 = L.F064.nnzb;
  info->nnzb_G1 = L.G164.nnzb;
  info->beta = L.beta;
  info->logdet_S = L.logdet_S;
  info->coarsest = level == (int)h->lv.size() - 1;
  info->nested_inner = L.nested_inner;
  info->fused_fsai = L.gg.S.R > 0 ? 1 : 0;
  info->flops_adapt = L.flops_adapt;
  info->flops_factor = L.flops_factor;
  info->learned = L.learned;
  info->gate = L.gate;
  if (L.gg.S.R > 0) {
    info->gg_rows = L.gg.S.R;
    info->gg_parts = L.gg.parts;
    info->gg_ctas = std::min(L.gg.S.n_groups, L.gg.ctas);
  }
  return PUM_OK;
}

pum_status pum_hier_export(pum_ctx* ctx, const pum_hier* h, int level, int which, pum_bsr_host* out) {
  if (!ctx || !out) return PUM_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  return guard(ctx, [&]() {
    check_level(h, level);
    Bsr tmp;
    const Bsr* m = nullptr;
    if (which == PUM_MAT_GT) {
      PUM_CHECK(!h->lv[level].G64.empty(), PUM_ERR_INVALID_ARG, "no G on this level");
      bsr_transpose(tmp, h->lv[level].G64, ctx->stream);
      m = &tmp;
    } else {
      m = select_matrix(h, level, which);
    }
    PUM_CHECK(m && !m->empty(), PUM_ERR_INVALID_ARG, "matrix not present on this level");
    auto v = bsr_values_host(*m, ctx->stream);
    out->n_brows = m->n_brows;
    out->n_bcols = m->n_bcols;
    out->bs = m->d;
    out->nnzb = m->nnzb;
    out->row_ptr = (int32_t*)malloc(sizeof(int32_t) * m->h_row_ptr.size());
    out->col_idx = (int32_t*)malloc(sizeof(int32_t) * std::max<size_t>(m->h_col_idx.size(), 1));
    out->vals = (double*)malloc(sizeof(double) * std::max<size_t>(v.size(), 1));
    if (!out->row_ptr || !out->col_idx || !out->vals) {
      pum_bsr_free(out);
      throw Error{PUM_ERR_OOM, "export: host allocation failed"};
    }
    std::memcpy(out->row_ptr, m->h_row_ptr.data(), sizeof(int32_t) * m->h_row_ptr.size());
    std::memcpy(out->col_idx, m->h_col_idx.data(), sizeof(int32_t) * m->h_col_idx.size());
    std::memcpy(out->vals, v.data(), sizeof(double) * v.size());
    bsr_free(tmp);
    return PUM_OK;
  });
}

void pum_bsr_free(pum_bsr_host* m) {
  if (!m) return;
  free(m->row_ptr);
  free(m->col_idx);
  free(m->vals);
  std::memset(m, 0, sizeof(*m));
}

pum_status pum_hier_save(pum_ctx* ctx, const pum_hier* h, const char* path) {
  if (!ctx || !h || !path) return PUM_ERR_INVALID_ARG;
  return guard(ctx, [&]() {
    check_ready(h);
    FILE* f = fopen(path, "wb");
    PUM_CHECK(f, PUM_ERR_IO, std::string("cannot open ") + path);
    try {
      const uint32_t head[2] = {kMagic, kVersion};
      wr(f, head, sizeof(head));
      wr(f, &h->fp, sizeof(h->fp));
      wr(f, &h->sp, sizeof(h->sp));
      const int32_t nl = (int32_t)h->lv.size();
      wr(f, &nl, sizeof(nl));
      for (const auto& L : h->lv) {
        const int32_t dims[3] = {L.m, L.n, L.d};
        wr(f, dims, sizeof(dims));
        wr(f, &L.beta, sizeof(double));
        wr(f, &L.logdet_S, sizeof(double));
        for (const Bsr* m : {&L.A, &L.P, &L.G64, &L.F064, &L.G164, &L.A1}) save_bsr(f, ctx, *m);
      }
      const int32_t N = h->coarse.N;
      wr(f, &N, sizeof(N));
      std::vector<double> Lc((size_t)N * N);
      PUM_CUDA(cudaMemcpy(Lc.data(), h->coarse.L, sizeof(double) * Lc.size(), cudaMemcpyDeviceToHost));
      wr(f, Lc.data(), sizeof(double) * Lc.size());
    } catch (...) {
      fclose(f);
      throw;
    }
    PUM_CHECK(fclose(f) == 0, PUM_ERR_IO, "close failed");
    return PUM_OK;
  });
}

pum_status pum_hier_load(pum_ctx* ctx, const char* path, pum_hier** out) {
  if (!ctx || !path || !out) return PUM_ERR_INVALID_ARG;
  *out = nullptr;
  pum_hier* h = new (std::nothrow) pum_hier();
  if (!h) return PUM_ERR_OOM;
  const pum_status st = guard(ctx, [&]() {
    FILE* f = fopen(path, "rb");
    PUM_CHECK(f, PUM_ERR_IO, std::string("cannot open ") + path);
    try {
      uint32_t head[2];
      rd(f, head, sizeof(head));
      PUM_CHECK(head[0] == kMagic, PUM_ERR_IO, "not a hierarchy file");
      PUM_CHECK(head[1] == kVersion, PUM_ERR_IO, "unsupported hierarchy file version");
      rd(f, &h->fp, sizeof(h->fp));
      rd(f, &h->sp, sizeof(h->sp));
      check_params(&h->fp, &h->sp);
      h->smooth_dt = h->sp.smooth_dt;
      h->g_dt = h->sp.g_dt;
      h->sell = ctx->sell;
      h->fused_fsai = ctx->fused_fsai;
      int32_t nl;
      rd(f, &nl, sizeof(nl));
      PUM_CHECK(nl >= 1 && nl <= 16, PUM_ERR_IO, "corrupt level count");
      h->lv.resize(nl);
      for (auto& L : h->lv) {
        int32_t dims[3];
        rd(f, dims, sizeof(dims));
        L.m = dims[0];
        L.n = dims[1];
        L.d = dims[2];
        rd(f, &L.beta, sizeof(double));
        rd(f, &L.logdet_S, sizeof(double));
        for (Bsr* m : {&L.A, &L.P, &L.G64, &L.F064, &L.G164, &L.A1}) load_bsr(f, ctx, *m);
      }
      int32_t N;
      rd(f, &N, sizeof(N));
      PUM_CHECK(N == h->lv.back().n * h->lv.back().d, PUM_ERR_IO, "corrupt coarse factor size");
      std::vector<double> Lc((size_t)N * N);
      rd(f, Lc.data(), sizeof(double) * Lc.size());
      h->coarse.N = N;
      h->coarse.L = (double*)dalloc(sizeof(double) * Lc.size());
      PUM_CUDA(cudaMemcpy(h->coarse.L, Lc.data(), sizeof(double) * Lc.size(), cudaMemcpyHostToDevice));
    } catch (...) {
      fclose(f);
      throw;
    }
    fclose(f);
    finalize_smoother(ctx, h);
    return PUM_OK;
  });
  if (st != PUM_OK) {
    pum_hier_destroy(h);
    return st;
  }
  *out = h;
  return PUM_OK;
}

pum_status pum_hier_destroy(pum_hier* h) {
  if (!h) return PUM_ERR_INVALID_ARG;
  cudaDeviceSynchronize();  // kernels queued on any stream may still read the hierarchy
  graph_destroy(h->vgraph);
  multi_cache_free(h->multi);
  for (auto& L : h->lv) free_level(L);
  for (auto& w : h->w64)
    if (w) cudaFree(w);
  for (auto& w : h->wb)
    if (w) cudaFree(w);
  if (h->coarse.L) cudaFree(h->coarse.L);
  delete h;
  return PUM_OK;
}

pum_status pum_timing_enable(pum_ctx* ctx, int mask) {
  if (!ctx || mask < 0 || mask >= (1 << PUM_TK_COUNT)) return PUM_ERR_INVALID_ARG;
  ctx->timing = mask;
  return PUM_OK;
}

pum_status pum_timing_reset(pum_ctx* ctx) {
  if (!ctx) return PUM_ERR_INVALID_ARG;
  return guard(ctx, [&]() {
    PUM_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < PUM_TK_COUNT; ++k) {
      ctx->tk_launches[k] = 0;
      ctx->tk_ms[k] = 0.0;
      ctx->tk_pool_used[k] = 0;
    }
    return PUM_OK;
  });
}

pum_status pum_timing_read(pum_ctx* ctx, int64_t* launches, double* ms) {
  if (!ctx || !launches || !ms) return PUM_ERR_INVALID_ARG;
  return guard(ctx, [&]() {
    PUM_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < PUM_TK_COUNT; ++k) {
      // collect the direct launches' event pairs (graph replays are collected as they finish)
      for (int64_t i = 0; i < ctx->tk_pool_used[k]; ++i) {
        float t = 0.f;
        PUM_CUDA(cudaEventElapsedTime(&t, ctx->tk_start[k][i], ctx->tk_stop[k][i]));
        ctx->tk_ms[k] += t;
        ctx->tk_launches[k]++;
      }
      ctx->tk_pool_used[k] = 0;
      launches[k] = ctx->tk_launches[k];
      ms[k] = ctx->tk_ms[k];
    }
    return PUM_OK;
  });
}

int64_t pum_launch_count(const pum_ctx* ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"
