// Learned candidate scoring for the adaptive block-FSAI pattern -- an addition to the paper's
// method (Algorithm 1, Section 2.1, stays its fallback and judge).
//
// Features.  For block row k with initial pattern P0_k, ring 1 is Algorithm 1's admissible set
// of P0 and ring 2 the further columns c < k reachable through ring 1's A-rows.  Per candidate
// c the first-order gain g_c = |L_c^{-1} (G0 A)_kc^T|_F^2 (G0 the static FSAI on P0, A_cc =
// L_c L_c^T) is Lemma 2.8's 1 - rho_c to first order; it and the other features come from A and
// G0 only, so one launch scores every row of a level without Algorithm 1's steps:
//   k_diag_info   (warp per block row)  |A_ii|_F and chol(A_ii)
//   k_cand_gain   (warp per candidate)  g_c and the direct coupling |A_kc| / sqrt(|A_kk||A_cc|)
//   k_cand_feat   (warp per block row)  the 12 float features of the row's candidates
// The network 12 -> 64 -> 64 -> 1 (ReLU) multiplies with BF16-rounded weights and accumulates in
// FP32: k_mlp_forward (thread per sample, weights in shared memory); training: k_mlp_backward
// (tiles of 128 samples, per-CTA gradient partials from shared-memory tiles), k_mlp_reduce
// (fixed-order sum of the partials), k_adam.  The contractions are 64 wide and cost well under a
// millisecond for a million samples, so they run on the FP32 pipes.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "pum_internal.cuh"
#include "small_dense.cuh"

namespace pum {

namespace {

constexpr int kF = PUM_MLP_FEATURES;
constexpr int kH = PUM_MLP_HIDDEN;
constexpr int kOffB1 = kH * kF;
constexpr int kOffW2 = kOffB1 + kH;
constexpr int kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH;
constexpr int kOffB3 = kOffW3 + kH;
constexpr int kParams = kOffB3 + 1;
static_assert(sizeof(pum_mlp) == sizeof(float) * kParams, "pum_mlp is the flat parameter vector");

constexpr int kWarps = 4;  // warps per CTA of the feature kernels

// ---------------------------------------------------------------------------- features

template <int D>
__global__ void __launch_bounds__(kWarps * 32) k_diag_info(const int* arp, const int* aci, const double* av, int astride,
                                                          int n, double* nrm, double* Ld, double* invd,
                                                          DevStatus* status) {
  const int w = blockIdx.x * kWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  __shared__ double scratch[kWarps][D * D];
  if (w >= n) return;
  const int b = find_blk(arp, aci, w, w);
  const double* Ab = av + (int64_t)b * astride;
  double s = 0.0;
  for (int e = lane; e < D * D; e += 32) s += Ab[e] * Ab[e];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) nrm[w] = sqrt(s);
  for (int e = lane; e < D * D; e += 32) scratch[threadIdx.x >> 5][e] = Ab[e];
  __syncwarp();
  double m;
  int ex;
  if (!warp_chol<D>(scratch[threadIdx.x >> 5], Ld + (int64_t)w * D * D, invd + (int64_t)w * D, m, ex) && lane == 0)
    set_status(status, PUM_ERR_NOT_SPD, w, kWhereFsai);
}

template <int D>
__global__ void __launch_bounds__(kWarps * 32) k_cand_gain(const int* arp, const int* aci, const double* av,
                                                          int astride, const int* grp, const int* gci,
                                                          const double* gv, int gstride, const int* crow,
                                                          const int* ccol, int64_t n_cand, const double* nrm,
                                                          const double* Ld, const double* invd, double* gain,
                                                          double* akc) {
  const int64_t w = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  __shared__ double R[kWarps][D * D];
  if (w >= n_cand) return;
  double* r = R[threadIdx.x >> 5];
  const int k = crow[w], c = ccol[w];
  // (G0 A)_kc = sum over the blocks G0_kj of row k of G0_kj A_jc, stored transposed in r
  double acc[(D * D + 31) / 32];
#pragma unroll
  for (int q = 0; q < (D * D + 31) / 32; ++q) acc[q] = 0.0;
  for (int b = grp[k]; b < grp[k + 1]; ++b) {
    const int j = gci[b];
    int ab = 0;
    if (lane == 0) ab = find_blk(arp, aci, j, c);
    ab = __shfl_sync(0xffffffffu, ab, 0);
    if (ab < 0) continue;
    const double* G = gv + (int64_t)b * gstride;
    const double* Aj = av + (int64_t)ab * astride;
#pragma unroll
    for (int q = 0; q < (D * D + 31) / 32; ++q) {
      const int e = lane + 32 * q;
      if (e < D * D) {
        const int rr = e / D, cc = e - (e / D) * D;
        double v = acc[q];
#pragma unroll
        for (int t = 0; t < D; ++t) v += G[rr * D + t] * Aj[t * D + cc];
        acc[q] = v;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < (D * D + 31) / 32; ++q) {
    const int e = lane + 32 * q;
    if (e < D * D) {
      const int rr = e / D, cc = e - (e / D) * D;
      r[cc * D + rr] = acc[q];
    }
  }
  __syncwarp();
  warp_lsolve<D>(Ld + (int64_t)c * D * D, invd + (int64_t)c * D, r);  // L_c^{-1} (G0 A)_kc^T
  double s = 0.0;
  for (int e = lane; e < D * D; e += 32) s += r[e] * r[e];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  int kb = 0;
  if (lane == 0) kb = find_blk(arp, aci, k, c);
  kb = __shfl_sync(0xffffffffu, kb, 0);
  double f = 0.0;
  if (kb >= 0)
    for (int e = lane; e < D * D; e += 32) f += av[(int64_t)kb * astride + e] * av[(int64_t)kb * astride + e];
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  if (lane == 0) {
    gain[w] = s;
    akc[w] = kb >= 0 ? sqrt(f) / sqrt(nrm[k] * nrm[c]) : 0.0;
  }
}

// Normalised coupling |A_ij|_F / sqrt(|A_ii| |A_jj|) by one thread (0 when not stored).
__device__ double coupling(const int* arp, const int* aci, const double* av, int astride, int dd, const double* nrm,
                           int i, int j) {
  const int b = find_blk(arp, aci, i, j);
  if (b < 0) return 0.0;
  double f = 0.0;
  for (int e = 0; e < dd; ++e) f += av[(int64_t)b * astride + e] * av[(int64_t)b * astride + e];
  return sqrt(f) / sqrt(nrm[i] * nrm[j]);
}

// One warp per block row: the 12 features of its candidates (ring 1 first, then ring 2).
__global__ void __launch_bounds__(kWarps * 32) k_cand_feat(const int* arp, const int* aci, const double* av,
                                                          int astride, int d, int n, int m, int max_row,
                                                          const int* prp, const int* pci, const int* cptr,
                                                          const int* ccol, const int* n1s, const double* gain,
                                                          const double* akc, const double* nrm, float* x) {
  const int k = blockIdx.x * kWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k >= n) return;
  const int c0 = cptr[k], c1 = cptr[k + 1], n1 = n1s[k];
  double gmax = 0.0;
  for (int q = c0 + lane; q < c0 + n1; q += 32) gmax = fmax(gmax, gain[q]);
  for (int o = 16; o > 0; o >>= 1) gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  const int np0 = prp[k + 1] - prp[k];
  const int kx = m ? k % m : 0, ky = m ? k / m : 0;
  for (int q = c0 + lane; q < c1; q += 32) {
    const int c = ccol[q];
    const bool r1 = q < c0 + n1;
    const double g = gain[q];
    int rank = 0;
    double via = 0.0;
    for (int q2 = c0; q2 < c0 + n1; ++q2) {
      if (r1 && gain[q2] > g * (1.0 + 1e-9)) ++rank;  // ties within the band share a rank
      if (q2 != q) {
        const double a = coupling(arp, aci, av, astride, d * d, nrm, ccol[q2], c);
        if (a > 0.0) via = fmax(via, gain[q2] * a * a);
      }
    }
    int linked = 0;
    for (int b = prp[k]; b < prp[k + 1]; ++b) linked += find_blk(arp, aci, pci[b], c) >= 0;
    const int cx = m ? c % m : 0, cy = m ? c / m : 0;
    float* f = x + (int64_t)q * kF;
    f[0] = r1 ? 1.0f : 0.0f;
    f[1] = (float)log10(1e-30 + akc[q]);
    f[2] = (float)log10(1e-30 + g);
    f[3] = (float)log10(1e-30 + via);
    f[4] = r1 ? (float)(rank / 10.0) : 1.0f;
    f[5] = gmax > 0.0 ? (float)(g / gmax) : 0.0f;
    f[6] = (float)((double)linked / np0);
    f[7] = (float)(np0 / 16.0);
    f[8] = (float)((cx - kx) / 4.0);
    f[9] = (float)((cy - ky) / 4.0);
    f[10] = (float)((double)(arp[k + 1] - arp[k]) / max_row);
    f[11] = (float)(n1 / 32.0);
  }
}

template <int D>
void gain_launch(pum_ctx* ctx, const Bsr& A, const Bsr& G0, const CandidateSet& cs, const double* nrm,
                 const double* Ld, const double* invd, double* gain, double* akc) {
  if (!cs.n) return;
  k_cand_gain<D><<<(unsigned)((cs.n + kWarps - 1) / kWarps), kWarps * 32, 0, ctx->stream>>>(
      A.row_ptr, A.col_idx, (const double*)A.vals, A.stride, G0.row_ptr, G0.col_idx, (const double*)G0.vals,
      G0.stride, cs.d_row, cs.d_col, cs.n, nrm, Ld, invd, gain, akc);
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
}

template <int D>
void diag_launch(pum_ctx* ctx, const Bsr& A, double* nrm, double* Ld, double* invd) {
  k_diag_info<D><<<(unsigned)((A.n_brows + kWarps - 1) / kWarps), kWarps * 32, 0, ctx->stream>>>(
      A.row_ptr, A.col_idx, (const double*)A.vals, A.stride, A.n_brows, nrm, Ld, invd, ctx->status);
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------- the network

__device__ __forceinline__ float to_bf16(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }

// Weights into shared memory: W1, W2, w3 rounded to BF16, biases as they are.
__device__ void load_params(const float* __restrict__ P, float* S) {
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) {
    const bool bias = (i >= kOffB1 && i < kOffW2) || (i >= kOffB2 && i < kOffW3) || i == kOffB3;
    S[i] = bias ? P[i] : to_bf16(P[i]);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) k_mlp_forward(const float* __restrict__ P, const float* __restrict__ X,
                                                    int64_t n, float* __restrict__ out) {
  __shared__ float S[kParams];
  load_params(P, S);
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    float x[kF], h1[kH];
#pragma unroll
    for (int f = 0; f < kF; ++f) x[f] = X[s * kF + f];
#pragma unroll
    for (int o = 0; o < kH; ++o) {
      float a = S[kOffB1 + o];
#pragma unroll
      for (int f = 0; f < kF; ++f) a = fmaf(S[o * kF + f], x[f], a);
      h1[o] = fmaxf(a, 0.0f);
    }
    float logit = S[kOffB3];
    for (int o = 0; o < kH; ++o) {
      float a = S[kOffB2 + o];
#pragma unroll
      for (int i = 0; i < kH; ++i) a = fmaf(S[kOffW2 + o * kH + i], h1[i], a);
      logit = fmaf(S[kOffW3 + o], fmaxf(a, 0.0f), logit);
    }
    out[s] = logit;
  }
}

constexpr int kTile = 128;       // samples per tile = threads per CTA of the backward kernel
constexpr int kPad = kH + 1;     // row stride of the per-sample tiles (no bank conflicts)
constexpr int kPerThread = (kParams + kTile - 1) / kTile;

size_t backward_smem() { return sizeof(float) * ((size_t)kParams + kTile * kF + 4 * (size_t)kTile * kPad + kTile); }

// Gradient partials of the mean loss over samples idx[0..count) (idx NULL: 0..count), scaled by
// inv_n; CTA b writes its kParams partial sums to part + b * kParams and its loss to lpart[b].
__global__ void __launch_bounds__(kTile) k_mlp_backward(const float* __restrict__ P, const float* __restrict__ X,
                                                       const float* __restrict__ Y, const int* __restrict__ idx,
                                                       int64_t count, float inv_n, float* __restrict__ part,
                                                       double* __restrict__ lpart) {
  extern __shared__ float sm[];
  float* S = sm;
  float* Xs = S + kParams;
  float* H1 = Xs + kTile * kF;
  float* Z2 = H1 + kTile * kPad;
  float* DZ2 = Z2 + kTile * kPad;
  float* DZ1 = DZ2 + kTile * kPad;
  float* DL = DZ1 + kTile * kPad;
  __shared__ double red[kTile / 32];
  load_params(P, S);
  const int t = threadIdx.x;
  float acc[kPerThread];
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) acc[j] = 0.0f;
  double loss = 0.0;
  const int64_t tiles = (count + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t s = tile * kTile + t;
    const bool valid = s < count;
    const int64_t row = valid ? (idx ? (int64_t)idx[s] : s) : 0;
    float x[kF];
#pragma unroll
    for (int f = 0; f < kF; ++f) {
      x[f] = valid ? X[row * kF + f] : 0.0f;
      Xs[t * kF + f] = x[f];
    }
    for (int o = 0; o < kH; ++o) {
      float a = S[kOffB1 + o];
#pragma unroll
      for (int f = 0; f < kF; ++f) a = fmaf(S[o * kF + f], x[f], a);
      H1[t * kPad + o] = fmaxf(a, 0.0f);
    }
    float logit = S[kOffB3];
    for (int o = 0; o < kH; ++o) {
      float a = S[kOffB2 + o];
      for (int i = 0; i < kH; ++i) a = fmaf(S[kOffW2 + o * kH + i], H1[t * kPad + i], a);
      Z2[t * kPad + o] = a;
      logit = fmaf(S[kOffW3 + o], fmaxf(a, 0.0f), logit);
    }
    const float y = valid ? Y[row] : 0.0f;
    const float p = 1.0f / (1.0f + expf(-logit));
    const float dl = valid ? (p - y) * inv_n : 0.0f;
    if (valid) loss += (double)fmaxf(logit, 0.0f) + log1p(exp(-fabs((double)logit))) - (double)y * logit;
    DL[t] = dl;
    for (int o = 0; o < kH; ++o) DZ2[t * kPad + o] = Z2[t * kPad + o] > 0.0f ? dl * S[kOffW3 + o] : 0.0f;
    for (int i = 0; i < kH; ++i) {
      float a = 0.0f;
      for (int o = 0; o < kH; ++o) a = fmaf(DZ2[t * kPad + o], S[kOffW2 + o * kH + i], a);
      DZ1[t * kPad + i] = H1[t * kPad + i] > 0.0f ? a : 0.0f;
    }
    __syncthreads();
#pragma unroll 1
    for (int j = 0; j < kPerThread; ++j) {
      const int q = t + j * kTile;
      if (q >= kParams) break;
      float a = 0.0f;
      if (q < kOffB1) {
        const int o = q / kF, f = q - (q / kF) * kF;
        for (int u = 0; u < kTile; ++u) a = fmaf(DZ1[u * kPad + o], Xs[u * kF + f], a);
      } else if (q < kOffW2) {
        const int o = q - kOffB1;
        for (int u = 0; u < kTile; ++u) a += DZ1[u * kPad + o];
      } else if (q < kOffB2) {
        const int o = (q - kOffW2) / kH, i = (q - kOffW2) - ((q - kOffW2) / kH) * kH;
        for (int u = 0; u < kTile; ++u) a = fmaf(DZ2[u * kPad + o], H1[u * kPad + i], a);
      } else if (q < kOffW3) {
        const int o = q - kOffB2;
        for (int u = 0; u < kTile; ++u) a += DZ2[u * kPad + o];
      } else if (q < kOffB3) {
        const int o = q - kOffW3;
        for (int u = 0; u < kTile; ++u) a = fmaf(DL[u], fmaxf(Z2[u * kPad + o], 0.0f), a);
      } else {
        for (int u = 0; u < kTile; ++u) a += DL[u];
      }
      acc[j] += a;
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) {
    const int q = t + j * kTile;
    if (q < kParams) part[(int64_t)blockIdx.x * kParams + q] = acc[j];
  }
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
  if ((t & 31) == 0) red[t >> 5] = loss;
  __syncthreads();
  if (t == 0) {
    double l = 0.0;
    for (int w = 0; w < kTile / 32; ++w) l += red[w];
    lpart[blockIdx.x] = l;
  }
}

// grad[q] = sum over the CTAs of part[b][q], in CTA order; lsum = sum of the loss partials.
__global__ void k_mlp_reduce(const float* __restrict__ part, const double* __restrict__ lpart, int nb,
                             float* __restrict__ grad, double* __restrict__ lsum) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < kParams) {
    double a = 0.0;
    for (int b = 0; b < nb; ++b) a += part[(int64_t)b * kParams + q];
    grad[q] = (float)a;
  }
  if (q == 0 && lsum) {
    double l = 0.0;
    for (int b = 0; b < nb; ++b) l += lpart[b];
    *lsum = l;
  }
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, float lr, float c1, float c2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= kParams) return;
  const float gq = g[q];
  const float a = 0.9f * m1[q] + 0.1f * gq;
  const float b = 0.999f * m2[q] + 0.001f * gq * gq;
  m1[q] = a;
  m2[q] = b;
  P[q] -= lr * (a / c1) / (sqrtf(b / c2) + 1e-8f);
}

struct MlpWork {
  float *P = nullptr, *part = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
  double *lpart = nullptr, *lsum = nullptr;
  int nb = 0;
  ~MlpWork() {
    for (void* p : {(void*)P, (void*)part, (void*)grad, (void*)m1, (void*)m2, (void*)lpart, (void*)lsum})
      if (p) cudaFree(p);
  }
};

void mlp_work_alloc(pum_ctx* ctx, MlpWork& w, const pum_mlp& m, int nb) {
  w.nb = nb;
  PUM_CUDA(cudaMalloc(&w.P, sizeof(float) * kParams));
  PUM_CUDA(cudaMalloc(&w.part, sizeof(float) * kParams * (size_t)nb));
  PUM_CUDA(cudaMalloc(&w.grad, sizeof(float) * kParams));
  PUM_CUDA(cudaMalloc(&w.lpart, sizeof(double) * nb));
  PUM_CUDA(cudaMalloc(&w.lsum, sizeof(double)));
  PUM_CUDA(cudaMemcpyAsync(w.P, &m, sizeof(float) * kParams, cudaMemcpyHostToDevice, ctx->stream));
}

void backward_launch(pum_ctx* ctx, MlpWork& w, const float* x, const float* y, const int* idx, int64_t count,
                     float inv_n) {
  const size_t smem = backward_smem();
  allow_max_dynamic_smem((const void*)k_mlp_backward);
  k_mlp_backward<<<w.nb, kTile, smem, ctx->stream>>>(w.P, x, y, idx, count, inv_n, w.part, w.lpart);
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
  k_mlp_reduce<<<(kParams + 255) / 256, 256, 0, ctx->stream>>>(w.part, w.lpart, w.nb, w.grad, w.lsum);
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
}

uint64_t splitmix64(uint64_t& s) {  // Steele, Lea & Flood (2014)
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
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

// ---------------------------------------------------------------------------- library side

void candidates_free(CandidateSet& cs) {
  for (void* p : {(void*)cs.d_row, (void*)cs.d_col, (void*)cs.d_x})
    if (p) cudaFree(p);
  cs = CandidateSet{};
}

void candidates_build(pum_ctx* ctx, const Bsr& A, const Bsr& G0, const std::vector<std::vector<int>>& P0, int m,
                      CandidateSet& cs) {
  const int n = A.n_brows, d = A.d;
  PUM_CHECK(d == 3 || d == 6 || d == 10 || d == 15 || d == 21, PUM_ERR_UNSUPPORTED, "block size");
  cudaStream_t s = ctx->stream;
  // ring 1 and ring 2 of every row (host; the pattern of A is on the host)
  std::vector<int> mark(n, -1), n1(n), row;
  cs.rp.assign(n + 1, 0);
  cs.col.clear();
  for (int k = 0; k < n; ++k) {
    for (int j : P0[k]) mark[j] = 3 * k;
    const size_t start = cs.col.size();
    for (int j : P0[k])
      for (int b = A.h_row_ptr[j]; b < A.h_row_ptr[j + 1]; ++b) {
        const int c = A.h_col_idx[b];
        if (c < k && mark[c] < 3 * k) {
          mark[c] = 3 * k + 1;
          cs.col.push_back(c);
        }
      }
    std::sort(cs.col.begin() + start, cs.col.end());
    const size_t mid = cs.col.size();
    for (size_t q = start; q < mid; ++q)
      for (int b = A.h_row_ptr[cs.col[q]]; b < A.h_row_ptr[cs.col[q] + 1]; ++b) {
        const int c = A.h_col_idx[b];
        if (c < k && mark[c] < 3 * k) {
          mark[c] = 3 * k + 2;
          cs.col.push_back(c);
        }
      }
    std::sort(cs.col.begin() + mid, cs.col.end());
    n1[k] = (int)(mid - start);
    cs.rp[k + 1] = (int)cs.col.size();
    row.insert(row.end(), cs.col.size() - start, k);
  }
  cs.n = (int64_t)cs.col.size();
  std::vector<int> prp(n + 1, 0), pci;
  for (int k = 0; k < n; ++k) {
    pci.insert(pci.end(), P0[k].begin(), P0[k].end());
    prp[k + 1] = (int)pci.size();
  }
  auto up = [&](const std::vector<int>& v) {
    int* p = nullptr;
    PUM_CUDA(cudaMalloc(&p, sizeof(int) * std::max<size_t>(v.size(), 1)));
    if (!v.empty()) PUM_CUDA(cudaMemcpyAsync(p, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, s));
    return p;
  };
  cs.d_row = up(row);
  cs.d_col = up(cs.col);
  int* d_cptr = up(cs.rp);
  int* d_n1 = up(n1);
  int* d_prp = up(prp);
  int* d_pci = up(pci);
  PUM_CUDA(cudaMalloc(&cs.d_x, sizeof(float) * kF * std::max<int64_t>(cs.n, 1)));
  double *nrm = nullptr, *Ld = nullptr, *invd = nullptr, *gain = nullptr, *akc = nullptr;
  PUM_CUDA(cudaMalloc(&nrm, sizeof(double) * n));
  PUM_CUDA(cudaMalloc(&Ld, sizeof(double) * (size_t)n * d * d));
  PUM_CUDA(cudaMalloc(&invd, sizeof(double) * (size_t)n * d));
  PUM_CUDA(cudaMalloc(&gain, sizeof(double) * std::max<int64_t>(cs.n, 1)));
  PUM_CUDA(cudaMalloc(&akc, sizeof(double) * std::max<int64_t>(cs.n, 1)));
  switch (d) {
    case 3: diag_launch<3>(ctx, A, nrm, Ld, invd); gain_launch<3>(ctx, A, G0, cs, nrm, Ld, invd, gain, akc); break;
    case 6: diag_launch<6>(ctx, A, nrm, Ld, invd); gain_launch<6>(ctx, A, G0, cs, nrm, Ld, invd, gain, akc); break;
    case 10: diag_launch<10>(ctx, A, nrm, Ld, invd); gain_launch<10>(ctx, A, G0, cs, nrm, Ld, invd, gain, akc); break;
    case 15: diag_launch<15>(ctx, A, nrm, Ld, invd); gain_launch<15>(ctx, A, G0, cs, nrm, Ld, invd, gain, akc); break;
    case 21: diag_launch<21>(ctx, A, nrm, Ld, invd); gain_launch<21>(ctx, A, G0, cs, nrm, Ld, invd, gain, akc); break;
    default: throw Error{PUM_ERR_UNSUPPORTED, "learned candidates: unsupported block size"};
  }
  k_cand_feat<<<(unsigned)((n + kWarps - 1) / kWarps), kWarps * 32, 0, s>>>(
      A.row_ptr, A.col_idx, (const double*)A.vals, A.stride, d, n, m, std::max(A.max_row_nnzb, 1), d_prp, d_pci,
      d_cptr, cs.d_col, d_n1, gain, akc, nrm, cs.d_x);
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
  PUM_CUDA(cudaStreamSynchronize(s));
  for (void* p : {(void*)d_cptr, (void*)d_n1, (void*)d_prp, (void*)d_pci, (void*)nrm, (void*)Ld, (void*)invd,
                  (void*)gain, (void*)akc})
    cudaFree(p);
  DevStatus st{};
  PUM_CUDA(cudaMemcpy(&st, ctx->status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st.code) {
    PUM_CUDA(cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), s));
    throw Error{(pum_status)st.code, "candidate features: diagonal block " + std::to_string(st.info) +
                                         " of A is not SPD"};
  }
}

void mlp_forward_dev(pum_ctx* ctx, const pum_mlp& m, const float* x, int64_t n, float* logits) {
  if (n <= 0) return;
  float* P = nullptr;
  PUM_CUDA(cudaMalloc(&P, sizeof(float) * kParams));
  PUM_CUDA(cudaMemcpyAsync(P, &m, sizeof(float) * kParams, cudaMemcpyHostToDevice, ctx->stream));
  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)ctx->sm_count * 8);
  k_mlp_forward<<<grid, 256, 0, ctx->stream>>>(P, x, n, logits);
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
  PUM_CUDA(cudaStreamSynchronize(ctx->stream));
  cudaFree(P);
}

}  // namespace pum

using namespace pum;

extern "C" pum_status pum_mlp_forward(pum_ctx* ctx, const pum_mlp* m, const float* x, int64_t n, float* logits) {
  if (!ctx || !m || (n > 0 && (!x || !logits)) || n < 0) return PUM_ERR_INVALID_ARG;
  return guarded(ctx, [&]() {
    mlp_forward_dev(ctx, *m, x, n, logits);
    return PUM_OK;
  });
}

extern "C" pum_status pum_mlp_grad(pum_ctx* ctx, const pum_mlp* m, const float* x, const float* y, int64_t n,
                                   double* loss, pum_mlp* grad) {
  if (!ctx || !m || !x || !y || n <= 0 || !grad) return PUM_ERR_INVALID_ARG;
  return guarded(ctx, [&]() {
    MlpWork w;
    const int tiles = (int)std::min<int64_t>((n + kTile - 1) / kTile, (int64_t)ctx->sm_count);
    mlp_work_alloc(ctx, w, *m, tiles);
    backward_launch(ctx, w, x, y, nullptr, n, (float)(1.0 / (double)n));
    PUM_CUDA(cudaMemcpyAsync(grad, w.grad, sizeof(float) * kParams, cudaMemcpyDeviceToHost, ctx->stream));
    double l = 0.0;
    PUM_CUDA(cudaMemcpyAsync(&l, w.lsum, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    PUM_CUDA(cudaStreamSynchronize(ctx->stream));
    if (loss) *loss = l / (double)n;
    return PUM_OK;
  });
}

extern "C" pum_status pum_mlp_train(pum_ctx* ctx, pum_mlp* m, const float* x, const float* y, int64_t n,
                                    int32_t epochs, int32_t batch, double lr, uint64_t seed, double* loss) {
  if (!ctx || !m || !x || !y || n <= 0 || epochs < 0 || batch <= 0 || !(lr > 0.0)) return PUM_ERR_INVALID_ARG;
  return guarded(ctx, [&]() {
    MlpWork w;
    const int tiles = (int)std::min<int64_t>(((int64_t)batch + kTile - 1) / kTile, (int64_t)ctx->sm_count);
    mlp_work_alloc(ctx, w, *m, std::max(tiles, (int)std::min<int64_t>((n + kTile - 1) / kTile, ctx->sm_count)));
    PUM_CUDA(cudaMalloc(&w.m1, sizeof(float) * kParams));
    PUM_CUDA(cudaMalloc(&w.m2, sizeof(float) * kParams));
    PUM_CUDA(cudaMemsetAsync(w.m1, 0, sizeof(float) * kParams, ctx->stream));
    PUM_CUDA(cudaMemsetAsync(w.m2, 0, sizeof(float) * kParams, ctx->stream));
    std::vector<int> perm(n);
    int* dperm = nullptr;
    PUM_CUDA(cudaMalloc(&dperm, sizeof(int) * n));
    uint64_t state = seed;
    int64_t step = 0;
    const int nb_all = w.nb;
    for (int e = 0; e < epochs; ++e) {
      for (int64_t i = 0; i < n; ++i) perm[i] = (int)i;
      for (int64_t i = n - 1; i > 0; --i) std::swap(perm[i], perm[splitmix64(state) % (uint64_t)(i + 1)]);
      PUM_CUDA(cudaStreamSynchronize(ctx->stream));  // the previous epoch's batches have read dperm
      PUM_CUDA(cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
      for (int64_t b0 = 0; b0 < n; b0 += batch) {
        const int64_t cnt = std::min<int64_t>(batch, n - b0);
        w.nb = tiles;
        backward_launch(ctx, w, x, y, dperm + b0, cnt, (float)(1.0 / (double)cnt));
        ++step;
        const float c1 = (float)(1.0 - std::pow(0.9, (double)step)), c2 = (float)(1.0 - std::pow(0.999, (double)step));
        k_adam<<<(kParams + 255) / 256, 256, 0, ctx->stream>>>(w.P, w.grad, w.m1, w.m2, (float)lr, c1, c2);
        count_launch(ctx);
        PUM_CUDA(cudaGetLastError());
      }
    }
    PUM_CUDA(cudaStreamSynchronize(ctx->stream));
    cudaFree(dperm);
    PUM_CUDA(cudaMemcpy(m, w.P, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
    if (loss) {
      w.nb = nb_all;
      backward_launch(ctx, w, x, y, nullptr, n, (float)(1.0 / (double)n));
      double l = 0.0;
      PUM_CUDA(cudaMemcpyAsync(&l, w.lsum, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      PUM_CUDA(cudaStreamSynchronize(ctx->stream));
      *loss = l / (double)n;
    }
    return PUM_OK;
  });
}

extern "C" pum_status pum_set_pattern_model(pum_ctx* ctx, const pum_mlp* m) {
  if (!ctx) return PUM_ERR_INVALID_ARG;
  delete ctx->model;
  ctx->model = m ? new pum_mlp(*m) : nullptr;
  return PUM_OK;
}

extern "C" void pum_candidates_free(pum_candidates* c) {
  if (!c) return;
  for (void* p : {(void*)c->row, (void*)c->col, (void*)c->x, (void*)c->y})
    if (p) cudaFree(p);
  *c = pum_candidates{};
}

extern "C" pum_status pum_candidates_copy(pum_ctx* ctx, const pum_candidates* c, int32_t* row, int32_t* col, float* x,
                                          float* y) {
  if (!ctx || !c) return PUM_ERR_INVALID_ARG;
  return guarded(ctx, [&]() {
    if (c->n > 0) {
      auto cp = [&](void* dst, const void* src, size_t bytes) {
        if (dst) PUM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
      };
      cp(row, c->row, sizeof(int32_t) * c->n);
      cp(col, c->col, sizeof(int32_t) * c->n);
      cp(x, c->x, sizeof(float) * kF * c->n);
      cp(y, c->y, sizeof(float) * c->n);
    }
    return PUM_OK;
  });
}
