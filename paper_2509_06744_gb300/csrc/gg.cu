// Block-FSAI application z = G^T (G r) that reads the factor once (Definition 2.2: M = G^T G).
//
// The two-product form streams G for t = G r and then its explicit transpose for z = G^T t, so
// the factor's values cross HBM twice per application: more bytes than the operator A itself.
// Here G crosses once.  The partial-product kernel is persistent: each CTA walks groups of R
// block rows of G in the sliced layout, and each group's slots stay resident in shared memory
// until the group is done (one cp.async.bulk per slot, each completing on its own mbarrier,
// evict-first in L2).  Two group buffers per CTA: warp 0 (producer) fills the next buffer while
// the other warps (consumers) work on the current one.  For a group, the producer
//   - issues the slot copies (lane 0),
//   - copies the group's block columns and the G^T positions of its blocks into shared memory,
//     then gathers the r segments of every slot there with per-lane cp.async copies that
//     arrive on the buffer's meta barrier when they land (all lanes);
// the consumers
//   1. form t_j = sum_s G_js r_col(j,s) for the group's rows (thread of unknown j d + r, reading
//      the slot chunks conflict-free, as in the sliced product),
//   2. form the partial products w_js = G_js^T t_j from the same resident slots (thread of
//      component c of row j, rows fastest across the warp: conflict-free for the block sizes
//      used), staged in shared memory over the consumed r segments,
//   3. store each block's d values contiguously at that block's position in G^T's block order,
//      and release the buffer (empty barrier).
// A second, light kernel then streams the partial products: z_i = sum_j w_ji over the blocks
// (i, j) of G^T in ascending j, a fixed order, so the result is deterministic, and applies the
// product's epilogue (the Chebyshev-4 update of Algorithm 3).  The partial products are d floats
// per block of G: a tenth of G's FP32 bytes for d = 10, written once and read once.
//
// Every wait is bounded: on expiry the kernel records PUM_ERR_TIMEOUT in the context's status
// word; the producer still waits (bounded) for its own copies before its warp leaves, and the
// consumer warps leave together after a barrier they all reach.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "bulk.cuh"
#include "kernels_common.cuh"

namespace pum {

namespace {

constexpr int kGgMaxThreads = 1024;
constexpr int kGgBuffers = 2;
constexpr int kGgMaxParts = 4;  // consumer partitions of a group's slots
constexpr int kGgPre = 4;       // slot entries per producer lane held in registers (32 x 4 per group)

// Shared memory: barriers (full per buffer and slot, meta and empty per buffer), then per buffer
// the group's slots, its r segments (reused for the staged partial products), its block columns
// and G^T positions; then t of the group's rows.
struct GgSmem {
  int hdr;          // bytes of the barrier header
  size_t buf;       // bytes of one group buffer
  size_t chunk;     // bytes of one slot chunk
  size_t total;
};

__host__ __device__ inline GgSmem gg_layout(int d, int R, int ns_max, int vsize) {
  GgSmem L;
  L.hdr = ((kGgBuffers * ns_max + 2 * kGgBuffers) * 8 + 127) / 128 * 128;
  L.chunk = (size_t)vsize * d * R * d;
  const size_t raw = (size_t)ns_max * L.chunk + sizeof(float) * (size_t)ns_max * R * d + 2 * sizeof(int) * (size_t)ns_max * R;
  L.buf = (raw + 127) / 128 * 128;
  L.total = (size_t)L.hdr + kGgBuffers * L.buf + sizeof(float) * (size_t)R * d * (1 + kGgMaxParts);
  return L;
}

// Producer warp + P consumer partitions of R d threads rounded up to whole warps.
unsigned gg_threads(int d, int R, int P) { return 32u + (unsigned)P * (unsigned)((R * d + 31) / 32) * 32u; }

template <int D, typename MT>
__device__ __forceinline__ void load_smem_row(const MT* p, float (&out)[D]) {
  if constexpr (sizeof(MT) == 4 && (D % 2) == 0) {
    const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
    for (int i = 0; i < D / 2; ++i) {
      const float2 v = q[i];
      out[2 * i] = v.x;
      out[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i) out[i] = to_f(p[i]);
  }
}

template <int D, typename MT>
__global__ void __launch_bounds__(kGgMaxThreads) k_gg_partial(int n_groups, int R, int ns_max,
                                                              const int* __restrict__ goff, const int* __restrict__ cols,
                                                              const int* __restrict__ tpos, const MT* __restrict__ vals,
                                                              const float* __restrict__ x, float* __restrict__ w,
                                                              DevStatus* st) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int timed_out;
  __shared__ int ginfo[kGgBuffers][2];  // (first slot, slot count) of the group in each buffer
  const int RD = R * D;
  const int chunk_elems = D * RD;
  const GgSmem lay = gg_layout(D, R, ns_max, (int)sizeof(MT));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);  // [buffer][slot]
  uint64_t* meta = full + kGgBuffers * ns_max;
  uint64_t* empty = meta + kGgBuffers;
  auto stage = [&](int b) { return reinterpret_cast<MT*>(smem + lay.hdr + b * lay.buf); };
  auto xsb = [&](int b) { return reinterpret_cast<float*>(smem + lay.hdr + b * lay.buf + ns_max * lay.chunk); };
  auto scolb = [&](int b) { return reinterpret_cast<int*>(xsb(b) + (size_t)ns_max * RD); };
  auto sposb = [&](int b) { return scolb(b) + ns_max * R; };
  float* ts = reinterpret_cast<float*>(smem + lay.hdr + kGgBuffers * lay.buf);
  float* tpart = ts + RD;  // P * RD partial sums of t
  const int n_consumer_warps = (int)(blockDim.x >> 5) - 1;

  if (threadIdx.x == 0) {
    timed_out = 0;
    for (int i = 0; i < kGgBuffers * ns_max; ++i) mbar_init(full + i, 1);
    for (int b = 0; b < kGgBuffers; ++b) {
      mbar_init(meta + b, 64);  // per producer lane: one arrival, one when its gathers land
      mbar_init(empty + b, (uint32_t)n_consumer_warps);
    }
    mbar_fence_init();
  }
  __syncthreads();

  if (threadIdx.x < 32) {  // producer warp
    const int lane = (int)threadIdx.x;
    bool ok = true, waited = false;
    int k = 0;
    for (int g = blockIdx.x; g < n_groups; g += gridDim.x, ++k) {
      const int b = k & 1;
      const uint32_t ph = (uint32_t)(k >> 1) & 1u;
      // The group's extent, block columns and G^T positions (constant data) are loaded into
      // registers first, so that their latency overlaps the wait for the buffer.
      const int s0 = __ldg(goff + g), ns = __ldg(goff + g + 1) - s0;
      const int m = ns * R;
      int pc[kGgPre], pp[kGgPre];
#pragma unroll
      for (int u = 0; u < kGgPre; ++u) {
        const int i = lane + 32 * u;
        pc[u] = i < m ? __ldg(cols + (int64_t)s0 * R + i) : 0;
        pp[u] = i < m ? __ldg(tpos + (int64_t)s0 * R + i) : -1;
      }
      if (k >= kGgBuffers && !__all_sync(0xffffffffu, mbar_wait(empty + b, ph ^ 1u))) {  // use k - 2 released
        ok = false;
        break;
      }
      if (lane == 0) {
        ginfo[b][0] = s0;
        ginfo[b][1] = ns;
        const uint64_t pol = l2_evict_first_policy();
        const MT* src = vals + (int64_t)s0 * chunk_elems;
        for (int s = 0; s < ns; ++s) {
          mbar_expect_tx(full + b * ns_max + s, (uint32_t)lay.chunk);
          bulk_g2s_policy(stage(b) + (size_t)s * chunk_elems, src + (int64_t)s * chunk_elems, (uint32_t)lay.chunk,
                          full + b * ns_max + s, pol);
        }
        // slots this group does not have: complete their phase too, so that every slot barrier of
        // a buffer completes once per use and its parity stays that of the use
        for (int s = ns; s < ns_max; ++s) mbar_arrive(full + b * ns_max + s);
      }
      int* scol = scolb(b);
      int* spos = sposb(b);
#pragma unroll
      for (int u = 0; u < kGgPre; ++u) {
        const int i = lane + 32 * u;
        if (i < m) {
          scol[i] = pc[u];
          spos[i] = pp[u];
        }
      }
      for (int i = lane + 32 * kGgPre; i < m; i += 32) {  // entries beyond the registers' share
        cp_async4(scol + i, cols + (int64_t)s0 * R + i);
        cp_async4(spos + i, tpos + (int64_t)s0 * R + i);
      }
      cp_async_wait_all();
      __syncwarp();
      if (!waited) {
        pdl_wait();  // r comes from the preceding kernel (the matrix and the index arrays do not)
        waited = true;
      }
      mbar_arrive(meta + b);  // releases the columns and positions
      // the r segment of every slot (column 0 for padding, against zero values), landing on the
      // meta barrier without holding registers
      float* xs = xsb(b);
      auto gather = [&](int sj, int col) {
        const float* src = x + (int64_t)max(col, 0) * D;
        float* dst = xs + sj * D;
        if constexpr ((D % 2) == 0) {
#pragma unroll
          for (int c = 0; c < D; c += 2) cp_async8(dst + c, src + c);
        } else {
#pragma unroll
          for (int c = 0; c < D; ++c) cp_async4(dst + c, src + c);
        }
      };
#pragma unroll
      for (int u = 0; u < kGgPre; ++u)
        if (lane + 32 * u < m) gather(lane + 32 * u, pc[u]);
      for (int sj = lane + 32 * kGgPre; sj < m; sj += 32) gather(sj, scol[sj]);
      cp_async_mbar_arrive_noinc(meta + b);
    }
    // own copies still in flight (normally all consumed already)
    const int kk = k;
    for (int u = max(kk - kGgBuffers, 0); u < kk && lane == 0; ++u) {
      const int b = u & 1;
      for (int s = 0; s < ginfo[b][1]; ++s)
        if (!mbar_wait(full + b * ns_max + s, (uint32_t)(u >> 1) & 1u)) ok = false;
    }
    cp_async_wait_all();  // the gathers of a group no consumer waited for
    if (!ok && lane == 0) set_status(st, PUM_ERR_TIMEOUT, blockIdx.x, kWhereGg);
    return;
  }

  // Consumers: P partitions of RDp threads (RD rounded up to whole warps); partition p takes the
  // slots s = p, p + P, ... of the group.
  if constexpr (kEarlyTrigger<D>) pdl_release();  // the gather may launch; it waits for this kernel
  const int nct = (int)blockDim.x - 32;
  const int RDp = (RD + 31) / 32 * 32;
  const int P = nct / RDp;
  const int t = (int)threadIdx.x - 32;
  const int p = t / RDp, tl = t - p * RDp;
  const bool computes = tl < RD;
  const int j = computes ? tl / D : 0;
  const int bpt = nct / D, c3 = t % D;  // step 3: blocks per pass, this thread's component
  int k = 0;
  for (int g = blockIdx.x; g < n_groups; g += gridDim.x, ++k) {
    const int b = k & 1;
    const uint32_t ph = (uint32_t)(k >> 1) & 1u;
    const MT* stg = stage(b);
    float* xs = xsb(b);
    const int* spos = sposb(b);
    float acc0 = 0.f, acc1 = 0.f;
    int ns = 0;
    if (!__all_sync(0xffffffffu, mbar_wait(meta + b, ph))) {
      if ((threadIdx.x & 31) == 0) {
        timed_out = 1;
        set_status(st, PUM_ERR_TIMEOUT, blockIdx.x, kWhereGg);
      }
    } else {
      ns = ginfo[b][1];
      // 1. this partition's part of t_j = sum over the slots of G_js r_col (thread of unknown
      //    j D + r; two accumulators, even and odd columns)
      for (int s = p; s < ns; s += P) {
        if (!__all_sync(0xffffffffu, mbar_wait(full + b * ns_max + s, ph))) {
          if ((threadIdx.x & 31) == 0) {
            timed_out = 1;
            set_status(st, PUM_ERR_TIMEOUT, blockIdx.x, kWhereGg);
          }
          break;
        }
        if (computes) {
          const MT* a = stg + (size_t)s * chunk_elems + tl;
          float xr[D];
          load_smem_row<D, float>(xs + (s * R + j) * D, xr);
#pragma unroll
          for (int cc = 0; cc < D; ++cc) {
            if (cc & 1)
              acc1 = fmaf(to_f(a[cc * RD]), xr[cc], acc1);
            else
              acc0 = fmaf(to_f(a[cc * RD]), xr[cc], acc0);
          }
        }
      }
    }
    if (computes) tpart[p * RD + tl] = acc0 + acc1;
    named_barrier(1, nct);
    if (timed_out) break;  // read after the barrier: the same decision in every consumer warp
    if (p == 0 && computes) {  // the partitions' sums in partition order
      float v = tpart[tl];
      for (int q = 1; q < P; ++q) v += tpart[q * RD + tl];
      ts[tl] = v;
    }
    named_barrier(1, nct);

    // 2. w_js = G_js^T t_j (thread of component c of row jj, rows fastest; partition p takes the
    //    same slots as in 1), staged over xs
    if (computes) {
      const int jj = tl % R, c = tl / R;
      float tv[D];
#pragma unroll
      for (int q = 0; q < D; ++q) tv[q] = ts[jj * D + q];
      for (int s = p; s < ns; s += P) {  // padding blocks are zero; step 3 does not store them
        float a[D];
        load_smem_row<D, MT>(stg + (size_t)s * chunk_elems + c * RD + jj * D, a);
        float v0 = 0.f, v1 = 0.f;
#pragma unroll
        for (int q = 0; q < D; ++q) {
          if (q & 1)
            v1 = fmaf(a[q], tv[q], v1);
          else
            v0 = fmaf(a[q], tv[q], v0);
        }
        xs[(s * R + jj) * D + c] = v0 + v1;
      }
    }
    named_barrier(1, nct);

    // 3. each block's d partial products, contiguous, at its position in G^T's block order
    //    (thread of component c3 of every bpt-th block)
    if (t < bpt * D)
      for (int sj = t / D; sj < ns * R; sj += bpt) {
        const int pos = spos[sj];
        if (pos >= 0) w[(int64_t)pos * D + c3] = xs[sj * D + c3];
      }
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(empty + b);  // this warp is done with buffer b
  }
  if constexpr (!kEarlyTrigger<D>) pdl_release();
}

template <int D, typename YT, typename X2T, int EPI>
__global__ void __launch_bounds__(256) k_gg_gather(int n_brows, const int* __restrict__ tptr,
                                                   const float* __restrict__ w, EpiArgs e) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = u < (int64_t)n_brows * D;
  const int i = live ? (int)(u / D) : 0;
  const int c = (int)(u - (int64_t)i * D);
  int q0 = 0, q1 = 0;
  if (live) {
    q0 = __ldg(tptr + i);
    q1 = __ldg(tptr + i + 1);
  }
  pdl_wait();  // w, and the epilogue's vectors, come from the preceding kernels
  if constexpr (kEarlyTrigger<D>) pdl_release();  // the next kernel may launch and issue its pre-wait loads
  const float* wc = w + c;
  float acc = 0.f;
  // sixteen independent loads in flight (one round for the rows of G^T of the workloads' factors,
  // 11 blocks on average), summed in block order
  for (int q = q0; q < q1; q += 16) {
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) v[u] = q + u < q1 ? wc[(int64_t)(q + u) * D] : 0.f;
#pragma unroll
    for (int u = 0; u < 16; ++u)
      if (q + u < q1) acc += v[u];
  }
  if constexpr (!kEarlyTrigger<D>) pdl_release();
  if (live) epilogue<EPI, float, float, YT, X2T>(e, u, acc);
}

template <int D, typename MT>
int gg_occupancy(int R, int P, int ns_max) {
  const void* kern = (const void*)k_gg_partial<D, MT>;
  allow_max_dynamic_smem(kern);
  int nb = 0;
  PUM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, (int)gg_threads(D, R, P),
                                                         gg_layout(D, R, ns_max, (int)sizeof(MT)).total));
  return nb;
}

template <int D>
int gg_occupancy_d(int dt, int R, int P, int ns_max) {
  return dt == PUM_BF16 ? gg_occupancy<D, __nv_bfloat16>(R, P, ns_max) : gg_occupancy<D, float>(R, P, ns_max);
}

int gg_occupancy_for(int d, int dt, int R, int P, int ns_max) {
  switch (d) {
    case 3: return gg_occupancy_d<3>(dt, R, P, ns_max);
    case 6: return gg_occupancy_d<6>(dt, R, P, ns_max);
    case 10: return gg_occupancy_d<10>(dt, R, P, ns_max);
    case 15: return gg_occupancy_d<15>(dt, R, P, ns_max);
    default: return gg_occupancy_d<21>(dt, R, P, ns_max);
  }
}

// Group size R and consumer partitions P: two buffers of the largest group must stay resident,
// so R is bounded by shared memory; P (at most kGgMaxParts and the longest row, within 1024
// threads) multiplies the consumer warps.  Take the R with the most block rows resident per SM
// (CTAs per SM x R), then the most consumer warps per SM, the largest R on ties.  Returns 0 when
// no group fits.
struct GgConfig {
  int R = 0, P = 0, occ = 0;
};

// Candidate group sizes R with their consumer partitions P and CTAs per SM: for every number of
// resident CTAs per SM, the largest R that reaches it (two buffers of the largest group must stay
// resident, so R is bounded by shared memory; P is at most kGgMaxParts and the longest row, within
// 1024 threads).  The first entry is the one with the most block rows resident per SM (CTAs per
// SM x R), then the most consumer warps, the largest R on ties.
std::vector<GgConfig> gg_candidates(const Bsr& G) {
  const int n = G.n_brows, d = G.d;
  const int vsize = (int)dt_size(G.dt);
  int max_row = 0;
  for (int i = 0; i < n; ++i) max_row = std::max(max_row, G.h_row_ptr[i + 1] - G.h_row_ptr[i]);
  int optin = 0, dev = 0;
  PUM_CUDA(cudaGetDevice(&dev));
  PUM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  GgConfig best;
  int best_rows = 0, best_warps = 0;
  std::vector<GgConfig> by_occ(64);
  for (int R = sell_rows_max(d); R >= 2; --R) {
    if (((size_t)vsize * d * R * d) % 16 != 0) continue;
    if (gg_layout(d, R, max_row, vsize).total + 1024 > (size_t)optin) continue;
    const int rdp = (R * d + 31) / 32 * 32;
    const int P = std::max(1, std::min({kGgMaxParts, max_row, (1024 - 32) / rdp}));
    const int occ = gg_occupancy_for(d, G.dt, R, P, max_row);
    if (occ <= 0) continue;
    const int rows = occ * R, warps = occ * P * rdp / 32;
    if (rows > best_rows || (rows == best_rows && warps > best_warps)) {
      best_rows = rows;
      best_warps = warps;
      best = GgConfig{R, P, occ};
    }
    if (occ < 64 && by_occ[occ].R == 0) by_occ[occ] = GgConfig{R, P, occ};  // R descends: the largest
  }
  std::vector<GgConfig> out;
  if (best.R) out.push_back(best);
  for (const auto& c : by_occ)
    if (c.R && c.R != best.R) out.push_back(c);
  return out;
}

template <int D, typename MT, typename YT, typename X2T>
void gg_launch(pum_ctx* ctx, const FusedG& F, const void* r, int epi, const EpiArgs& e, int tk_g, int tk_gt) {
  const Sell& S = F.S;
  const unsigned threads = gg_threads(D, S.R, F.parts);
  const size_t smem = gg_layout(D, S.R, S.max_slots, (int)sizeof(MT)).total;
  if (tk_g >= 0) timing_begin(ctx, tk_g);
  {
    auto kern = k_gg_partial<D, MT>;
    allow_max_dynamic_smem((const void*)kern);
    const unsigned grid = (unsigned)std::min(S.n_groups, F.ctas);
    launch_cycle_kernel(ctx, kern, dim3(grid), dim3(threads), smem, S.n_groups, S.R, S.max_slots, S.goff, S.cols,
                        (const int*)F.tpos, (const MT*)S.vals, (const float*)r, F.w, ctx->status);
    count_launch(ctx);
    PUM_CUDA(cudaGetLastError());
  }
  if (tk_g >= 0) timing_end(ctx, tk_g);
  if (tk_gt >= 0) timing_begin(ctx, tk_gt);
  const int64_t N = (int64_t)F.n * D;
  const dim3 grid((unsigned)((N + 255) / 256));
  switch (epi) {
#define PUM_GG_CASE(E)                                                                                       \
  case E:                                                                                                    \
    launch_cycle_kernel(ctx, k_gg_gather<D, YT, X2T, E>, grid, dim3(256), 0, F.n, (const int*)F.tptr,        \
                        (const float*)F.w, e);                                                               \
    break;
    PUM_GG_CASE(EPI_SET)
    PUM_GG_CASE(EPI_CHEB_FIRST0)
    PUM_GG_CASE(EPI_CHEB_FIRST)
    PUM_GG_CASE(EPI_CHEB)
#undef PUM_GG_CASE
    default:
      throw Error{PUM_ERR_UNSUPPORTED, "fused FSAI application: unsupported epilogue"};
  }
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
  if (tk_gt >= 0) timing_end(ctx, tk_gt);
}

template <int D>
void gg_apply_d(pum_ctx* ctx, const FusedG& F, int gdt, const void* r, int epi, const EpiArgs& e, int tk_g,
                int tk_gt) {
  const int ydt = e.ydt >= 0 ? e.ydt : PUM_F32;
  const int x2dt = (e.xo2 && e.x2dt >= 0) ? e.x2dt : ydt;
  PUM_CHECK(ydt == PUM_F32 && (x2dt == PUM_F32 || x2dt == PUM_F64), PUM_ERR_UNSUPPORTED,
            "fused FSAI application: FP32 vectors only");
  if (gdt == PUM_BF16) {
    if (x2dt == PUM_F64) return gg_launch<D, __nv_bfloat16, float, double>(ctx, F, r, epi, e, tk_g, tk_gt);
    return gg_launch<D, __nv_bfloat16, float, float>(ctx, F, r, epi, e, tk_g, tk_gt);
  }
  if (x2dt == PUM_F64) return gg_launch<D, float, float, double>(ctx, F, r, epi, e, tk_g, tk_gt);
  return gg_launch<D, float, float, float>(ctx, F, r, epi, e, tk_g, tk_gt);
}

}  // namespace

void gg_free(FusedG& F) {
  sell_free(F.S);
  for (void** p : {(void**)&F.tptr, (void**)&F.tpos, (void**)&F.w})
    if (*p) {
      cudaFree(*p);
      *p = nullptr;
    }
  F.n = F.d = 0;
  F.dt = PUM_F32;
}

namespace {

// The fused layout of G for one group size.
void gg_build_config(FusedG& F, const Bsr& G, cudaStream_t st, int sm_count, const GgConfig& cfg) {
  gg_free(F);
  const int d = G.d, n = G.n_brows;
  const int R = cfg.R;
  std::vector<int> goff;
  sell_build_rows(F.S, G, R, st);
  const int ng = F.S.n_groups;
  goff.assign(ng + 1, 0);
  PUM_CUDA(cudaMemcpy(goff.data(), F.S.goff, sizeof(int) * goff.size(), cudaMemcpyDeviceToHost));
  // G^T's block rows: block (j, i) of G is block (i, j) of G^T; rows of G in ascending j.
  std::vector<int> tptr(n + 1, 0), tpos((size_t)std::max<int64_t>(F.S.slots, 1) * R, -1);
  for (int64_t b = 0; b < G.nnzb; ++b) tptr[G.h_col_idx[b] + 1]++;
  for (int i = 0; i < n; ++i) tptr[i + 1] += tptr[i];
  std::vector<int> fill(tptr.begin(), tptr.end() - 1);
  for (int jr = 0; jr < n; ++jr) {
    const int grp = jr / R, jj = jr - grp * R;
    for (int q = 0; q < G.h_row_ptr[jr + 1] - G.h_row_ptr[jr]; ++q) {
      const int i = G.h_col_idx[G.h_row_ptr[jr] + q];
      tpos[(size_t)(goff[grp] + q) * R + jj] = fill[i]++;
    }
  }
  const size_t wbytes = sizeof(float) * (size_t)std::max<int64_t>(G.nnzb, 1) * d;
  if (cudaMalloc(&F.tptr, sizeof(int) * tptr.size()) != cudaSuccess ||
      cudaMalloc(&F.tpos, sizeof(int) * tpos.size()) != cudaSuccess || cudaMalloc(&F.w, wbytes) != cudaSuccess) {
    cudaGetLastError();
    gg_free(F);
    throw Error{PUM_ERR_OOM, "fused FSAI layout: device allocation failed"};
  }
  PUM_CUDA(cudaMemcpyAsync(F.tptr, tptr.data(), sizeof(int) * tptr.size(), cudaMemcpyHostToDevice, st));
  PUM_CUDA(cudaMemcpyAsync(F.tpos, tpos.data(), sizeof(int) * tpos.size(), cudaMemcpyHostToDevice, st));
  PUM_CUDA(cudaStreamSynchronize(st));
  F.n = n;
  F.d = d;
  F.dt = G.dt;
  F.ctas = cfg.occ * sm_count;
  F.parts = cfg.P;
}

template <int D, typename MT>
void gg_partial_launch(pum_ctx* ctx, const FusedG& F, const float* x) {
  auto kern = k_gg_partial<D, MT>;
  allow_max_dynamic_smem((const void*)kern);
  launch_cycle_kernel(ctx, kern, dim3((unsigned)std::min(F.S.n_groups, F.ctas)), dim3(gg_threads(D, F.S.R, F.parts)),
                      gg_layout(D, F.S.R, F.S.max_slots, (int)sizeof(MT)).total, F.S.n_groups, F.S.R, F.S.max_slots,
                      F.S.goff, F.S.cols, (const int*)F.tpos, (const MT*)F.S.vals, x, F.w, ctx->status);
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
}

template <int D>
void gg_partial_launch_dt(pum_ctx* ctx, const FusedG& F, const float* x) {
  if (F.dt == PUM_BF16) gg_partial_launch<D, __nv_bfloat16>(ctx, F, x);
  else gg_partial_launch<D, float>(ctx, F, x);
}

// Mean time of the partial-product kernel of layout F over `reps` launches (after one warm-up).
float gg_time_partial(pum_ctx* ctx, const FusedG& F, const float* x, int reps) {
  auto run = [&]() {
    switch (F.d) {
      case 3: gg_partial_launch_dt<3>(ctx, F, x); break;
      case 6: gg_partial_launch_dt<6>(ctx, F, x); break;
      case 10: gg_partial_launch_dt<10>(ctx, F, x); break;
      case 15: gg_partial_launch_dt<15>(ctx, F, x); break;
      default: gg_partial_launch_dt<21>(ctx, F, x); break;
    }
  };
  cudaEvent_t a, b;
  PUM_CUDA(cudaEventCreate(&a));
  PUM_CUDA(cudaEventCreate(&b));
  run();
  PUM_CUDA(cudaEventRecord(a, ctx->stream));
  for (int i = 0; i < reps; ++i) run();
  PUM_CUDA(cudaEventRecord(b, ctx->stream));
  PUM_CUDA(cudaEventSynchronize(b));
  float ms = 0.f;
  PUM_CUDA(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / (float)reps;
}

}  // namespace

// Fused layout of G with its group size chosen by measurement: every candidate configuration
// (gg_candidates: the heuristic's choice and the largest R for each number of CTAs per SM) is
// built and its partial-product kernel timed on the context's stream; a candidate more than 5%
// faster than the current choice replaces it.
void gg_build(pum_ctx* ctx, FusedG& F, const Bsr& G) {
  gg_free(F);
  const int d = G.d, n = G.n_brows;
  if (!(d == 3 || d == 6 || d == 10 || d == 15 || d == 21)) return;
  if (!(G.dt == PUM_F32 || G.dt == PUM_BF16) || G.n_bcols != n || n == 0) return;
  const std::vector<GgConfig> cands = gg_candidates(G);
  if (cands.empty()) return;  // rows too long to keep two groups resident: the two-product form stays
  GgConfig best = cands[0];
  if (cands.size() > 1) {
    float* x = nullptr;
    PUM_CUDA(cudaMalloc(&x, sizeof(float) * (size_t)n * d));
    PUM_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * (size_t)n * d, ctx->stream));
    float best_ms = 0.f;
    try {
      for (size_t i = 0; i < cands.size(); ++i) {
        gg_build_config(F, G, ctx->stream, ctx->sm_count, cands[i]);
        const float ms = gg_time_partial(ctx, F, x, 5);
        // another configuration replaces the current choice only when clearly faster, so that
        // timing noise does not flip the choice (and the partition order of the sums) between runs
        if (i == 0 || ms < 0.95f * best_ms) {
          best_ms = ms;
          best = cands[i];
        }
      }
    } catch (...) {
      cudaFree(x);
      throw;
    }
    PUM_CUDA(cudaStreamSynchronize(ctx->stream));
    cudaFree(x);
    if (F.S.R == best.R && F.parts == best.P) return;
  }
  gg_build_config(F, G, ctx->stream, ctx->sm_count, best);
}

void gg_apply(pum_ctx* ctx, const FusedG& F, const void* r, int epi, const EpiArgs& e, int tk_g, int tk_gt) {
  PUM_CHECK(F.S.R > 0, PUM_ERR_UNSUPPORTED, "fused FSAI application: layout not built");
  const int gdt = F.dt;
  switch (F.d) {
    case 3: gg_apply_d<3>(ctx, F, gdt, r, epi, e, tk_g, tk_gt); break;
    case 6: gg_apply_d<6>(ctx, F, gdt, r, epi, e, tk_g, tk_gt); break;
    case 10: gg_apply_d<10>(ctx, F, gdt, r, epi, e, tk_g, tk_gt); break;
    case 15: gg_apply_d<15>(ctx, F, gdt, r, epi, e, tk_g, tk_gt); break;
    case 21: gg_apply_d<21>(ctx, F, gdt, r, epi, e, tk_g, tk_gt); break;
    default: throw Error{PUM_ERR_UNSUPPORTED, "fused FSAI application: unsupported block size"};
  }
}

}  // namespace pum
