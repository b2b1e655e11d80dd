// Block-FSAI set-up on the device (Definition 2.2, Lemma 2.8, Algorithm 1, Section 2.2),
// the Lanczos estimate of lambda_max(M A) (Section 5) and the coarsest-level Cholesky.
//
// Block row k of the FSAI is an independent dense SPD problem of size s = |P~_k| d, so
// the set-up is a batch of small FP64 factorisations: one CTA per block row gathers
// A[P~_k, P~_k] (packed lower triangle) and A[P~_k, k] into shared memory, factors
// A[P~_k, P~_k] = L L^T, forms Z_k = L^{-1} A[P~_k, k], S_kk = A_kk - Z_k^T Z_k,
// S_kk = L_S L_S^T, F[k, P~_k] = -(L^{-T} Z_k)^T and G row k = L_S^{-1} F row k.
// Algorithm 1's candidate scores reuse L:  Z_c = L^{-1} A[P~_k, c],
// W_c = A_cc - Z_c^T Z_c, H_kc = A_kc - Z_k^T Z_c (= (F A)_kc),
// rho_c = det(W_c - H_kc^T S_kk^{-1} H_kc) / det(W_c) by Cholesky log-determinants.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>

#include "pum_internal.cuh"

namespace pum {

constexpr int kFsaiThreads = 256;
constexpr int kMaxPt = 32;   // max |P~_k| (blocks) per row
constexpr int kMaxD = 21;

struct FsaiArgs {
  // A (FP64)
  const int* arp; const int* aci; const double* av; int astride; int d;
  // pattern P (lower, sorted, diagonal last) per block row
  const int* prp; const int* pci;
  // work list
  const int* rows; int n_rows;
  // adaptive candidates per work item
  const int* crp; const int* cci; int group;  // candidates solved together
  double tie_rel, tau;
  int* chosen;      // per work item: c* or -1 (retire)
  int max_cand;     // max candidates of a work item (rho list length)
  // outputs of the factorisation (may be null)
  double* gv; int gstride;  // G values on pattern P
  double* fv; int fstride;  // F values on pattern P
  double* logdetS;          // per block row
  DevStatus* status;
  int where;
};

__device__ __forceinline__ int find_block(const int* rp, const int* ci, int row, int col) {
  int lo = rp[row], hi = rp[row + 1] - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int c = ci[mid];
    if (c == col) return mid;
    if (c < col) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

__device__ __forceinline__ int pidx(int i, int j) { return i * (i + 1) / 2 + j; }  // packed lower, j <= i

// Cholesky of a small d x d matrix held in shared memory (row-major), by one thread.
// Returns log det (sum of 2 log L_ii) or NaN when not positive definite.
__device__ double chol_small(double* M, int d) {
  double ld = 0.0;
  for (int j = 0; j < d; ++j) {
    double v = M[j * d + j];
    for (int q = 0; q < j; ++q) v -= M[j * d + q] * M[j * d + q];
    if (!(v > 0.0)) return __longlong_as_double(0x7ff8000000000000LL);
    const double ljj = sqrt(v);
    M[j * d + j] = ljj;
    ld += 2.0 * log(ljj);
    for (int i = j + 1; i < d; ++i) {
      double t = M[i * d + j];
      for (int q = 0; q < j; ++q) t -= M[i * d + q] * M[j * d + q];
      M[i * d + j] = t / ljj;
    }
    for (int q = j + 1; q < d; ++q) M[j * d + q] = 0.0;
  }
  return ld;
}

// Forward solve L Y = Y in place for `ncol` right-hand-side columns (row-major s x ld).
__device__ void fwd_solve(const double* Lp, double* Y, int s, int ncol, int ld) {
  for (int i = 0; i < s; ++i) {
    const double lii = Lp[pidx(i, i)];
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) Y[i * ld + c] /= lii;
    __syncthreads();
    const int rest = (s - i - 1) * ncol;
    for (int t = threadIdx.x; t < rest; t += blockDim.x) {
      const int l = i + 1 + t / ncol, c = t - (t / ncol) * ncol;
      Y[l * ld + c] -= Lp[pidx(l, i)] * Y[i * ld + c];
    }
    __syncthreads();
  }
}

// Backward solve L^T Y = Y in place.
__device__ void bwd_solve(const double* Lp, double* Y, int s, int ncol, int ld) {
  for (int i = s - 1; i >= 0; --i) {
    const double lii = Lp[pidx(i, i)];
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) Y[i * ld + c] /= lii;
    __syncthreads();
    const int rest = i * ncol;
    for (int t = threadIdx.x; t < rest; t += blockDim.x) {
      const int l = t / ncol, c = t - (t / ncol) * ncol;
      Y[l * ld + c] -= Lp[pidx(i, l)] * Y[i * ld + c];
    }
    __syncthreads();
  }
}

// Shared-memory layout: doubles Lp[s(s+1)/2] | Zk[s*d] | S[d*d] | J[d*d] | Zc[group*max(s,d)*d] |
// Wc[group*d*d] | Xc[group*d*d] | rho[ncand], then ints pt[kMaxPt+1] | blk[np*np].
__global__ void __launch_bounds__(kFsaiThreads) k_fsai_rows(FsaiArgs a) {
  extern __shared__ double smem[];
  __shared__ int s_fail;
  __shared__ double s_ld;
  const int w = blockIdx.x;
  if (w >= a.n_rows) return;
  const int k = a.rows[w];
  const int d = a.d, dd = d * d;
  const int p0 = a.prp[k], p1 = a.prp[k + 1];
  const int np = p1 - p0 - 1;  // |P~_k| (diagonal is last)
  const int s = np * d;
  const int group = max(a.group, 1);
  const int c0 = a.crp ? a.crp[w] : 0, c1 = a.crp ? a.crp[w + 1] : 0;
  double* Lp = smem;
  double* Zk = Lp + s * (s + 1) / 2;
  double* S = Zk + s * d;
  double* J = S + dd;
  double* Zc = J + dd;
  double* Wc = Zc + (size_t)group * max(s, d) * d;  // Zc also holds X = W - U^T U (group d x d)
  double* Xc = Wc + (size_t)group * dd;
  double* rl = Xc + (size_t)group * dd;
  int* pt = reinterpret_cast<int*>(rl + (a.crp ? a.max_cand : 0));
  int* blk = pt + kMaxPt + 1;
  if (threadIdx.x == 0) s_fail = 0;
  for (int t = threadIdx.x; t < np; t += blockDim.x) pt[t] = a.pci[p0 + t];
  __syncthreads();
  // block indices of A[P~, P~] (lower part) and gather
  for (int t = threadIdx.x; t < np * np; t += blockDim.x) {
    const int u = t / np, v = t - (t / np) * np;
    blk[t] = (v <= u) ? find_block(a.arp, a.aci, pt[u], pt[v]) : -1;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < s * (s + 1) / 2; t += blockDim.x) {
    // decode packed (i, j), j <= i
    int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (pidx(i, 0) > t) --i;
    while (pidx(i + 1, 0) <= t) ++i;
    const int j = t - pidx(i, 0);
    const int bi = i / d, bj = j / d;
    const int b = blk[bi * np + bj];
    Lp[t] = b >= 0 ? a.av[(int64_t)b * a.astride + (i - bi * d) * d + (j - bj * d)] : 0.0;
  }
  for (int t = threadIdx.x; t < s * d; t += blockDim.x) {
    const int i = t / d, c = t - (t / d) * d;
    const int bi = i / d;
    const int b = find_block(a.arp, a.aci, pt[bi], k);
    Zk[t] = b >= 0 ? a.av[(int64_t)b * a.astride + (i - bi * d) * d + c] : 0.0;
  }
  {
    const int bkk = find_block(a.arp, a.aci, k, k);
    for (int t = threadIdx.x; t < dd; t += blockDim.x) S[t] = bkk >= 0 ? a.av[(int64_t)bkk * a.astride + t] : 0.0;
  }
  __syncthreads();
  // Cholesky of A[P~, P~] (right-looking, packed)
  for (int j = 0; j < s; ++j) {
    if (threadIdx.x == 0) {
      const double v = Lp[pidx(j, j)];
      if (!(v > 0.0)) s_fail = 1;
      Lp[pidx(j, j)] = sqrt(fmax(v, 0.0));
    }
    __syncthreads();
    if (s_fail) break;
    const double ljj = Lp[pidx(j, j)];
    for (int i = j + 1 + threadIdx.x; i < s; i += blockDim.x) Lp[pidx(i, j)] /= ljj;
    __syncthreads();
    const int rem = s - j - 1;
    const int cnt = rem * (rem + 1) / 2;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      int ii = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
      while (pidx(ii, 0) > t) --ii;
      while (pidx(ii + 1, 0) <= t) ++ii;
      const int jj = t - pidx(ii, 0);
      const int i = j + 1 + ii, l = j + 1 + jj;
      Lp[pidx(i, l)] -= Lp[pidx(i, j)] * Lp[pidx(l, j)];
    }
    __syncthreads();
  }
  if (s_fail) {
    if (threadIdx.x == 0) set_status(a.status, PUM_ERR_NOT_SPD, k, a.where);
    return;
  }
  // Z_k = L^{-1} A[P~, k]
  fwd_solve(Lp, Zk, s, d, d);
  // S_kk = A_kk - Z_k^T Z_k
  for (int t = threadIdx.x; t < dd; t += blockDim.x) {
    const int r = t / d, c = t - (t / d) * d;
    double v = S[t];
    for (int i = 0; i < s; ++i) v -= Zk[i * d + r] * Zk[i * d + c];
    S[t] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double ld = chol_small(S, d);  // S <- L_S
    s_ld = ld;
    if (!(ld == ld)) s_fail = 1;
  }
  __syncthreads();
  if (s_fail) {
    if (threadIdx.x == 0) set_status(a.status, PUM_ERR_NOT_SPD, k, a.where);
    return;
  }
  // J = L_S^{-1} (column c by thread c)
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    for (int i = 0; i < d; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int q = c; q < i; ++q) v -= S[i * d + q] * J[q * d + c];
      J[i * d + c] = (i >= c) ? v / S[i * d + i] : 0.0;
    }
  }
  __syncthreads();
  if (a.logdetS && threadIdx.x == 0) a.logdetS[k] = s_ld;

  if (a.crp) {
    // ---------------- Algorithm 1: rho_c for every admissible c, groups of `group` columns
    for (int g0 = c0; g0 < c1; g0 += group) {
      const int ng = min(group, c1 - g0);
      const int ld = ng * d;
      // A[P~, c] for the group (row-major s x ld)
      for (int t = threadIdx.x; t < s * ld; t += blockDim.x) {
        const int i = t / ld, col = t - (t / ld) * ld;
        const int g = col / d, cc = col - g * d;
        const int bi = i / d;
        const int b = find_block(a.arp, a.aci, pt[bi], a.cci[g0 + g]);
        Zc[t] = b >= 0 ? a.av[(int64_t)b * a.astride + (i - bi * d) * d + cc] : 0.0;
      }
      __syncthreads();
      fwd_solve(Lp, Zc, s, ld, ld);  // Z_c = L^{-1} A[P~, c]
      // W_c = A_cc - Z_c^T Z_c,  H_kc = A_kc - Z_k^T Z_c
      for (int t = threadIdx.x; t < ng * dd; t += blockDim.x) {
        const int g = t / dd, e = t - g * dd;
        const int r = e / d, c = e - (e / d) * d;
        const int cand = a.cci[g0 + g];
        const int bcc = find_block(a.arp, a.aci, cand, cand);
        const int bkc = find_block(a.arp, a.aci, k, cand);
        double wv = bcc >= 0 ? a.av[(int64_t)bcc * a.astride + e] : 0.0;
        double hv = bkc >= 0 ? a.av[(int64_t)bkc * a.astride + e] : 0.0;
        for (int i = 0; i < s; ++i) {
          wv -= Zc[i * ld + g * d + r] * Zc[i * ld + g * d + c];
          hv -= Zk[i * d + r] * Zc[i * ld + g * d + c];
        }
        Wc[g * dd + e] = wv;
        Xc[g * dd + e] = hv;
      }
      __syncthreads();
      // U = L_S^{-1} H_kc in place (each thread owns one column of one candidate)
      for (int t = threadIdx.x; t < ng * d; t += blockDim.x) {
        const int g = t / d, c = t - (t / d) * d;
        double u[kMaxD];
        for (int r = 0; r < d; ++r) {
          double v = 0.0;
          for (int q = 0; q <= r; ++q) v += J[r * d + q] * Xc[g * dd + q * d + c];
          u[r] = v;
        }
        for (int r = 0; r < d; ++r) Xc[g * dd + r * d + c] = u[r];
      }
      __syncthreads();
      // X = W_c - U^T U  (= W_c - H_kc^T S_kk^{-1} H_kc), into the dead Zc area
      double* Xm = Zc;
      for (int t = threadIdx.x; t < ng * dd; t += blockDim.x) {
        const int g = t / dd, e = t - g * dd;
        const int r = e / d, c = e - (e / d) * d;
        double v = Wc[g * dd + e];
        for (int q = 0; q < d; ++q) v -= Xc[g * dd + q * d + r] * Xc[g * dd + q * d + c];
        Xm[g * dd + e] = v;
      }
      __syncthreads();
      // A candidate whose W_c or Schur complement X is not numerically positive definite has
      // no computable rho_c in FP64 (it is linearly dependent on the current pattern to working
      // precision); it is marked -1 and not chosen.
      for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const double lx = chol_small(Xm + g * dd, d);
        const double lw = chol_small(Wc + g * dd, d);
        rl[g0 - c0 + g] = (lx == lx && lw == lw) ? exp(lx - lw) : -1.0;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      // argmin with the tie band: smallest column among rho_c <= rho_min (1 + tie_rel), over
      // the candidates with a computable rho_c
      double rmin = -1.0;
      for (int q = c0; q < c1; ++q) {
        const double r = rl[q - c0];
        if (r >= 0.0 && (rmin < 0.0 || r < rmin)) rmin = r;
      }
      int choice = -1;
      if (rmin >= 0.0) {
        const double thr = rmin * (1.0 + a.tie_rel);
        int cstar = -1;
        double rstar = 0.0;
        for (int q = c0; q < c1; ++q) {
          const double r = rl[q - c0];
          if (r >= 0.0 && r <= thr && (cstar < 0 || a.cci[q] < cstar)) { cstar = a.cci[q]; rstar = r; }
        }
        // stop test with the tie band (a gain 1 - rho below tie_rel of tau is rounding)
        choice = (rstar < a.tau * (1.0 - a.tie_rel)) ? cstar : -1;
      }
      a.chosen[w] = choice;
    }
    return;
  }

  // ---------------- F and G rows: Y = L^{-T} Z_k, F[k, P~] = -Y^T, G = J F
  bwd_solve(Lp, Zk, s, d, d);
  const int g0 = p0;  // position of row k's blocks in the pattern arrays (= G/F block index)
  for (int t = threadIdx.x; t < np * dd; t += blockDim.x) {
    const int b = t / dd, e = t - b * dd;
    const int r = e / d, c = e - (e / d) * d;
    const double f = -Zk[(b * d + c) * d + r];
    if (a.fv) a.fv[(int64_t)(g0 + b) * a.fstride + e] = f;
    if (a.gv) {
      double v = 0.0;
      for (int q = 0; q <= r; ++q) v -= J[r * d + q] * Zk[(b * d + c) * d + q];
      a.gv[(int64_t)(g0 + b) * a.gstride + e] = v;
    }
  }
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    if (a.fv) a.fv[(int64_t)(g0 + np) * a.fstride + e] = (e / d == e % d) ? 1.0 : 0.0;
    if (a.gv) a.gv[(int64_t)(g0 + np) * a.gstride + e] = J[e];
  }
}

// ----------------------------------------------------------------------------- host side

namespace {

size_t fsai_smem_bytes(int s, int d, int group, int np, int ncand) {
  const size_t dbl = (size_t)s * (s + 1) / 2 + (size_t)s * d + 2 * (size_t)d * d + (size_t)group * std::max(s, d) * d +
                     2 * (size_t)group * d * d + (size_t)ncand;
  const size_t ints = kMaxPt + 1 + (size_t)np * np;
  return dbl * 8 + ints * 4;
}

int max_smem_optin(int dev) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

struct Pattern {
  std::vector<std::vector<int>> rows;
  void to_csr(std::vector<int>& rp, std::vector<int>& ci) const {
    rp.assign(rows.size() + 1, 0);
    ci.clear();
    for (size_t i = 0; i < rows.size(); ++i) {
      ci.insert(ci.end(), rows[i].begin(), rows[i].end());
      rp[i + 1] = (int)ci.size();
    }
  }
};

Pattern initial_pattern(const Bsr& A, int p0) {
  Pattern P;
  P.rows.resize(A.n_brows);
  for (int i = 0; i < A.n_brows; ++i) {
    if (p0 == PUM_P0_DIAG) {
      P.rows[i] = {i};
    } else {
      for (int b = A.h_row_ptr[i]; b < A.h_row_ptr[i + 1]; ++b)
        if (A.h_col_idx[b] <= i) P.rows[i].push_back(A.h_col_idx[b]);
    }
  }
  return P;
}

template <typename T> T* dev_upload(const std::vector<T>& v, cudaStream_t s) {
  T* d = nullptr;
  PUM_CUDA(cudaMalloc(&d, sizeof(T) * std::max<size_t>(v.size(), 1)));
  if (!v.empty()) PUM_CUDA(cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s));
  return d;
}

void check_status(pum_ctx* ctx, const char* what) {
  DevStatus st{};
  PUM_CUDA(cudaMemcpy(&st, ctx->status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st.code != 0) {
    PUM_CUDA(cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), ctx->stream));
    const char* stage = st.where == kWhereFsai ? "Cholesky of A[P~,P~] or S_kk" :
                        st.where == kWhereAdaptive ? "candidate Schur complement" : "dense Cholesky";
    throw Error{(pum_status)st.code, std::string(what) + ": factorisation failed (non-positive pivot, " + stage +
                                         ") at block row " + std::to_string(st.info)};
  }
}

// Run the row kernel: either factor rows into G/F (cand == nullptr) or score candidates.
void run_rows(pum_ctx* ctx, const Bsr& A, const Pattern& P, const std::vector<int>& rows,
              const std::vector<int>* crp, const std::vector<int>* cci, double tie_rel, double tau,
              std::vector<int>* chosen, Bsr* G, Bsr* F, double* logdetS) {
  if (rows.empty()) return;
  cudaStream_t s = ctx->stream;
  const int d = A.d;
  std::vector<int> prp, pci;
  P.to_csr(prp, pci);
  int max_np = 0, max_cand = 0;
  for (int k : rows) max_np = std::max(max_np, (int)P.rows[k].size() - 1);
  if (crp)
    for (size_t w = 0; w < rows.size(); ++w) max_cand = std::max(max_cand, (*crp)[w + 1] - (*crp)[w]);
  PUM_CHECK(max_np <= kMaxPt, PUM_ERR_UNSUPPORTED, "FSAI row pattern longer than 32 blocks");
  PUM_CHECK(d <= kMaxD, PUM_ERR_UNSUPPORTED, "FSAI block size above 21");
  PUM_CHECK(max_cand <= 64 * 64, PUM_ERR_UNSUPPORTED, "too many FSAI candidates");
  const int s_max = max_np * d;
  cudaFuncAttributes fa{};
  PUM_CUDA(cudaFuncGetAttributes(&fa, (const void*)k_fsai_rows));
  const int limit = max_smem_optin(ctx->device) - (int)fa.sharedSizeBytes;  // dynamic part
  int group = 1;  // the kernel lays shared memory out with at least one candidate group
  if (crp) {
    group = std::min(std::max(max_cand, 1), 64);
    while (group > 1 && fsai_smem_bytes(s_max, d, group, max_np, max_cand) > (size_t)limit) --group;
  }
  const size_t smem = fsai_smem_bytes(s_max, d, group, max_np, max_cand);
  PUM_CHECK(smem <= (size_t)limit, PUM_ERR_UNSUPPORTED,
            "FSAI row too large for shared memory (s = " + std::to_string(s_max) + ")");
  // the largest limit, not this launch's size: concurrent set-ups (batches) share the function
  // attribute, and a smaller value set by another thread would fail this launch
  allow_max_dynamic_smem((const void*)k_fsai_rows);
  int* dprp = dev_upload(prp, s);
  int* dpci = dev_upload(pci, s);
  int* drows = dev_upload(rows, s);
  int *dcrp = nullptr, *dcci = nullptr, *dchosen = nullptr;
  FsaiArgs a{};
  a.arp = A.row_ptr; a.aci = A.col_idx; a.av = (const double*)A.vals; a.astride = A.stride; a.d = d;
  a.prp = dprp; a.pci = dpci; a.rows = drows; a.n_rows = (int)rows.size();
  a.tie_rel = tie_rel; a.tau = tau; a.status = ctx->status; a.where = kWhereFsai; a.logdetS = logdetS;
  a.group = group;
  if (crp) {
    dcrp = dev_upload(*crp, s);
    dcci = dev_upload(*cci, s);
    PUM_CUDA(cudaMalloc(&dchosen, sizeof(int) * rows.size()));
    a.crp = dcrp; a.cci = dcci; a.group = group; a.chosen = dchosen; a.max_cand = max_cand;
  } else {
    if (G) { a.gv = (double*)G->vals; a.gstride = G->stride; }
    if (F) { a.fv = (double*)F->vals; a.fstride = F->stride; }
  }
  k_fsai_rows<<<(unsigned)rows.size(), kFsaiThreads, smem, s>>>(a);
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
  PUM_CUDA(cudaStreamSynchronize(s));
  check_status(ctx, crp ? "adaptive FSAI" : "block-FSAI");
  if (crp) {
    chosen->resize(rows.size());
    PUM_CUDA(cudaMemcpy(chosen->data(), dchosen, sizeof(int) * rows.size(), cudaMemcpyDeviceToHost));
  }
  for (void* p : {(void*)dprp, (void*)dpci, (void*)drows, (void*)dcrp, (void*)dcci, (void*)dchosen})
    if (p) cudaFree(p);
}

// Algorithm 1 (or the static pattern when !adaptive); returns the final pattern.
Pattern fsai_pattern(pum_ctx* ctx, const Bsr& A, const Pattern& P0, const bfsai_params& fp, double* flops) {
  Pattern P = P0;
  if (!fp.adaptive) return P;
  if (!ctx->adapt_steps && adaptive_patterns_device(ctx, A, P0.rows, fp.t_max, fp.tau, fp.tie_rel, P.rows, flops))
    return P;
  const int n = A.n_brows;
  std::vector<char> inR(n, 1);
  std::vector<int> mark(n, -1);
  for (int t = 0; t < fp.t_max; ++t) {
    std::vector<int> rows, crp{0}, cci;
    for (int k = 0; k < n; ++k) {
      if (!inR[k]) continue;
      // structural admissible set: c < k in the union of A's pattern rows j in P_k, c not in P_k
      std::vector<int> cand;
      for (int j : P.rows[k]) mark[j] = k;  // mark P_k
      std::vector<int> seen;
      for (int j : P.rows[k])
        for (int b = A.h_row_ptr[j]; b < A.h_row_ptr[j + 1]; ++b) {
          const int c = A.h_col_idx[b];
          if (c < k && mark[c] != k && mark[c] != -2 - k) {
            mark[c] = -2 - k;
            cand.push_back(c);
          }
        }
      if (cand.empty()) {
        inR[k] = 0;
        continue;
      }
      std::sort(cand.begin(), cand.end());
      rows.push_back(k);
      cci.insert(cci.end(), cand.begin(), cand.end());
      crp.push_back((int)cci.size());
    }
    if (rows.empty()) break;
    std::vector<int> chosen;
    run_rows(ctx, A, P, rows, &crp, &cci, fp.tie_rel, fp.tau, &chosen, nullptr, nullptr, nullptr);
    for (size_t w = 0; w < rows.size(); ++w) {
      const int k = rows[w];
      if (chosen[w] < 0) {
        inR[k] = 0;
      } else {
        auto& r = P.rows[k];
        r.insert(std::lower_bound(r.begin(), r.end(), chosen[w]), chosen[w]);
      }
    }
  }
  return P;
}

// G (and optionally F) of A on pattern P, FP64; returns sum_k log det S_kk.
double fsai_factor(pum_ctx* ctx, const Bsr& A, const Pattern& P, Bsr& G, Bsr* F, double* flops,
                   std::vector<double>* ld_rows = nullptr) {
  std::vector<int> rp, ci;
  P.to_csr(rp, ci);
  bsr_alloc(G, A.n_brows, A.n_bcols, A.d, PUM_F64, rp, ci);
  if (F) bsr_alloc(*F, A.n_brows, A.n_bcols, A.d, PUM_F64, rp, ci);
  std::vector<int> rows(A.n_brows);
  for (int i = 0; i < A.n_brows; ++i) rows[i] = i;
  if (flops) {
    // FP64 multiply-adds per row (s = |P~_k| d): Cholesky s^3/6, Z_k = L^-1 A[P~,k] and the
    // backward solve s^2 d / 2 each, S_kk s d^2, chol(S_kk) d^3/6, J = L_S^-1 d^3/6, G = J F d^2 (s + d) / 2
    const double d = A.d;
    double fma = 0.0;
    for (const auto& r : P.rows) {
      const double s = (double)(r.size() - 1) * d;
      fma += s * s * s / 6.0 + s * s * d + s * d * d + d * d * d / 3.0 + d * d * (s + d) / 2.0;
    }
    *flops += 2.0 * fma;
  }
  double* dld = nullptr;
  PUM_CUDA(cudaMalloc(&dld, sizeof(double) * A.n_brows));
  timing_begin(ctx, PUM_TK_FACTOR);
  run_rows(ctx, A, P, rows, nullptr, nullptr, 0, 0, nullptr, &G, F, dld);
  timing_end(ctx, PUM_TK_FACTOR);
  std::vector<double> ld(A.n_brows);
  PUM_CUDA(cudaMemcpy(ld.data(), dld, sizeof(double) * A.n_brows, cudaMemcpyDeviceToHost));
  cudaFree(dld);
  double sum = 0.0;
  for (double v : ld) sum += v;
  if (ld_rows) *ld_rows = std::move(ld);
  return sum;
}

// log det S_kk (Definition 2.2) of the given rows for pattern P (the rest of P is not factored).
std::vector<double> logdet_rows(pum_ctx* ctx, const Bsr& A, const Pattern& P, const std::vector<int>& rows,
                                double* flops) {
  std::vector<int> rp, ci;
  P.to_csr(rp, ci);
  Bsr G;
  bsr_alloc(G, A.n_brows, A.n_bcols, A.d, PUM_F64, rp, ci);
  double* dld = nullptr;
  PUM_CUDA(cudaMalloc(&dld, sizeof(double) * A.n_brows));
  run_rows(ctx, A, P, rows, nullptr, nullptr, 0, 0, nullptr, &G, nullptr, dld);
  std::vector<double> all(A.n_brows), out;
  PUM_CUDA(cudaMemcpy(all.data(), dld, sizeof(double) * A.n_brows, cudaMemcpyDeviceToHost));
  cudaFree(dld);
  bsr_free(G);
  const double d = A.d;
  for (int k : rows) {
    out.push_back(all[k]);
    const double s = (double)(P.rows[k].size() - 1) * d;
    if (flops) *flops += 2.0 * (s * s * s / 6.0 + s * s * d + s * d * d + d * d * d / 3.0 + d * d * (s + d) / 2.0);
  }
  return out;
}

// Algorithm 1's pattern (or P0 when not adaptive) and the FSAI factors on it: in one device launch
// that also forms G (and F) from its grown local factorisations when available, else the pattern
// search followed by the factor kernel.  Returns sum_k log det S_kk.
double pattern_and_factor(pum_ctx* ctx, const Bsr& A, const Pattern& P0, const bfsai_params& fp, Pattern& P, Bsr& G,
                          Bsr* F, Level& L) {
  if (fp.adaptive && !ctx->adapt_steps) {
    P = P0;
    double ld = 0.0;
    timing_begin(ctx, PUM_TK_ADAPT);
    const bool done = adaptive_patterns_device(ctx, A, P0.rows, fp.t_max, fp.tau, fp.tie_rel, P.rows, &L.flops_adapt,
                                               nullptr, &G, F, &ld);
    timing_end(ctx, PUM_TK_ADAPT);
    if (done) return ld;
  }
  P = fsai_pattern(ctx, A, P0, fp, &L.flops_adapt);
  return fsai_factor(ctx, A, P, G, F, &L.flops_factor);
}

constexpr int kLearnedMinRows = 1024;  // smaller levels run Algorithm 1 (cheap there)
constexpr int kGateStride = 16;        // the gate runs Algorithm 1 on every 16th block row
constexpr double kGateShortfall = 0.05;

// The learned pattern of a level: the static FSAI G0 on P0 (its per-row log det S_kk into ld0),
// candidate features, the model's logits, and each row's t_max best-scoring candidates
// (ties: smaller column).
Pattern learned_pattern(pum_ctx* ctx, Level& L, const Pattern& P0, const bfsai_params& fp, std::vector<double>& ld0) {
  Bsr G0;
  fsai_factor(ctx, L.A, P0, G0, nullptr, &L.flops_factor, &ld0);
  CandidateSet cs;
  try {
    candidates_build(ctx, L.A, G0, P0.rows, L.m, cs);
  } catch (...) {
    bsr_free(G0);
    throw;
  }
  bsr_free(G0);
  std::vector<float> logit(cs.n);
  float* dl = nullptr;
  PUM_CUDA(cudaMalloc(&dl, sizeof(float) * std::max<int64_t>(cs.n, 1)));
  mlp_forward_dev(ctx, *ctx->model, cs.d_x, cs.n, dl);
  if (cs.n) PUM_CUDA(cudaMemcpy(logit.data(), dl, sizeof(float) * cs.n, cudaMemcpyDeviceToHost));
  cudaFree(dl);
  Pattern P = P0;
  std::vector<std::pair<float, int>> order;
  for (int k = 0; k < L.n; ++k) {
    order.clear();
    for (int q = cs.rp[k]; q < cs.rp[k + 1]; ++q) order.push_back({-logit[q], cs.col[q]});
    std::sort(order.begin(), order.end());
    auto& r = P.rows[k];
    for (int i = 0; i < (int)order.size() && i < fp.t_max; ++i) r.push_back(order[i].second);
    std::sort(r.begin(), r.end());
  }
  candidates_free(cs);
  return P;
}

}  // namespace

void copy_blocks(pum_ctx* ctx, Bsr& dst, const Bsr& src, const int* idx);

// FP64 block-FSAI factors of level l: G64 (or, nested, F064 / A1 / G164) and the
// Kaporin-type measure sum_k log det S_kk.  Precision copies and transposes are made
// when the smoother is finalised.
void fsai_setup_level(pum_ctx* ctx, pum_hier* h, int l) {
  Level& L = h->lv[l];
  L.flops_adapt = L.flops_factor = 0.0;
  const bfsai_params& fp = h->fp;
  const Pattern P0 = initial_pattern(L.A, fp.p0);
  cudaStream_t s = ctx->stream;
  L.learned = 0;
  L.gate = -1.0;
  if (!fp.nested && fp.adaptive == 2 && ctx->model && L.n >= kLearnedMinRows) {
    std::vector<double> ld0, ldL;
    const Pattern P = learned_pattern(ctx, L, P0, fp, ld0);
    L.logdet_S = fsai_factor(ctx, L.A, P, L.G64, nullptr, &L.flops_factor, &ldL);
    // the gate: Algorithm 1 on every 16th row, its gain in sum log det S_kk against the learned one
    std::vector<int> sample;
    for (int k = 0; k < L.n; k += kGateStride) sample.push_back(k);
    Pattern Pa = P0;
    if (!adaptive_patterns_device(ctx, L.A, P0.rows, fp.t_max, fp.tau, fp.tie_rel, Pa.rows, &L.flops_adapt,
                                  &sample)) {
      Pa = P0;  // no device instantiation: the step-by-step Algorithm 1 on every row
      Pa = fsai_pattern(ctx, L.A, P0, bfsai_params{fp.p0, 1, fp.t_max, fp.tau, 0, fp.tie_rel}, &L.flops_adapt);
    }
    const std::vector<double> ldA = logdet_rows(ctx, L.A, Pa, sample, &L.flops_factor);
    double num = 0.0, den = 0.0;
    for (size_t i = 0; i < sample.size(); ++i) {
      num += ldL[sample[i]] - ldA[i];
      den += ld0[sample[i]] - ldA[i];
    }
    L.gate = den > 0.0 ? num / den : 0.0;
    if (L.gate <= kGateShortfall) {
      L.learned = 1;
      return;
    }
    bsr_free(L.G64);  // the gate failed: Algorithm 1 on every row
  }
  if (!fp.nested) {
    bfsai_params a1 = fp;
    a1.adaptive = fp.adaptive ? 1 : 0;
    Pattern P;
    L.logdet_S = pattern_and_factor(ctx, L.A, P0, a1, P, L.G64, nullptr, L);
    return;
  }
  // one level of nesting: A1 = F0 A F0^T, inner FSAI of A1 with the same parameters
  Pattern Pout;
  Bsr Gout;
  pattern_and_factor(ctx, L.A, P0, fp, Pout, Gout, &L.F064, L);
  bsr_free(Gout);
  Bsr F0T64, FA;
  bsr_transpose(F0T64, L.F064, s);
  spgemm(FA, L.F064, L.A, s);
  spgemm(L.A1, FA, F0T64, s);
  bsr_free(FA);
  bsr_free(F0T64);
  // The inner FSAI needs A1 = F0 A F0^T to be numerically SPD.  On coarse Galerkin levels of
  // strongly penalised problems the computed A1 can lose that in FP64 (its small eigen-
  // directions fall below the rounding of the triple product); the level then uses the inner
  // block Jacobi, G1 = diag_B(G_outer) = S^{-1/2}, which is the non-nested FSAI (Section 2.2).
  try {
    Pattern Pin;
    L.logdet_S = pattern_and_factor(ctx, L.A1, P0, fp, Pin, L.G164, nullptr, L);
    L.nested_inner = 1;
  } catch (const Error& e) {
    if (e.st != PUM_ERR_NOT_SPD) throw;
    Bsr Gout2;
    L.logdet_S = fsai_factor(ctx, L.A, Pout, Gout2, nullptr, &L.flops_factor);
    std::vector<int> rp(L.n + 1), ci(L.n);
    for (int i = 0; i < L.n; ++i) { rp[i] = i; ci[i] = i; }
    rp[L.n] = L.n;
    bsr_alloc(L.G164, L.n, L.n, L.d, PUM_F64, rp, ci);
    // copy the diagonal blocks of the outer G (the last block of each row of a lower pattern)
    std::vector<int> src(L.n);
    for (int i = 0; i < L.n; ++i) src[i] = Gout2.h_row_ptr[i + 1] - 1;
    int* dsrc = nullptr;
    PUM_CUDA(cudaMalloc(&dsrc, sizeof(int) * L.n));
    PUM_CUDA(cudaMemcpy(dsrc, src.data(), sizeof(int) * L.n, cudaMemcpyHostToDevice));
    copy_blocks(ctx, L.G164, Gout2, dsrc);
    cudaFree(dsrc);
    bsr_free(Gout2);
    L.nested_inner = 0;
  }
}

__global__ void k_copy_blocks(double* __restrict__ dst, int dstride, const double* __restrict__ src, int sstride,
                              const int* __restrict__ idx, int dd, int64_t nblk) {
  const int64_t total = nblk * dd;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / dd;
    const int e = (int)(i - b * dd);
    dst[b * dstride + e] = src[(int64_t)idx[b] * sstride + e];
  }
}

void copy_blocks(pum_ctx* ctx, Bsr& dst, const Bsr& src, const int* idx) {
  const int64_t total = dst.nnzb * dst.d * dst.d;
  if (!total) return;
  k_copy_blocks<<<(unsigned)std::min<int64_t>((total + 255) / 256, 2048), 256, 0, ctx->stream>>>(
      (double*)dst.vals, dst.stride, (const double*)src.vals, src.stride, idx, dst.d * dst.d, dst.nnzb);
  PUM_CUDA(cudaGetLastError());
  PUM_CUDA(cudaStreamSynchronize(ctx->stream));
}

// ----------------------------------------------------------------------------- Lanczos

__global__ void k_fill_uniform(double* v, int64_t n, unsigned long long seed) {
  // SplitMix64 (Steele, Lea & Flood 2014): output i = mix(seed + (i+1) * golden gamma)
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    v[i] = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
  }
}

// w = w - coef * v, coef = sgn * c[idx] (c on device)
__global__ void k_axpy_dev(double* w, const double* v, const double* c, int idx, double sgn, int64_t n) {
  const double a = sgn * c[idx];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] -= a * v[i];
}

// beta[j] = sqrt(ww); v_prev = v; v = w / beta[j]
__global__ void k_lanczos_next(double* vprev, double* v, const double* w, const double* ww, double* beta, int j,
                               int64_t n) {
  const double b = sqrt(*ww);
  if (blockIdx.x == 0 && threadIdx.x == 0) beta[j] = b;
  const double inv = 1.0 / b;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    vprev[i] = v[i];
    v[i] = w[i] * inv;
  }
}

__global__ void k_scale_by_rsqrt(double* v, const double* ss, int64_t n) {
  const double inv = 1.0 / sqrt(*ss);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] *= inv;
}

void dot_to(pum_ctx* ctx, const double* a, const double* b, int64_t n, double* out);

namespace {
// Largest eigenvalue of the symmetric tridiagonal (alpha, beta) by Sturm-sequence bisection.
double tridiag_lmax(const std::vector<double>& al, const std::vector<double>& be) {
  const int n = (int)al.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? std::fabs(be[i - 1]) : 0.0) + (i < n - 1 ? std::fabs(be[i]) : 0.0);
    lo = std::min(lo, al[i] - r);
    hi = std::max(hi, al[i] + r);
  }
  auto count_below = [&](double x) {
    int c = 0;
    double q = al[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < n; ++i) {
      if (q == 0.0) q = 1e-300;
      q = al[i] - x - be[i - 1] * be[i - 1] / q;
      if (q < 0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 400 && hi - lo > 1e-15 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= n) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}
}  // namespace

void lanczos_level(pum_ctx* ctx, pum_hier* h, int l) {
  Level& L = h->lv[l];
  const int64_t N = (int64_t)L.n * L.d;
  const int its = (int)std::min<int64_t>(std::max(h->sp.lanczos_its, 1), N);
  cudaStream_t s = ctx->stream;
  // the operator uses the matrices at the precision the smoother stores them in
  Bsr G, GT, F0, F0T;
  const bool nested = h->fp.nested;
  // FP64 copy of a factor rounded through the smoother's storage precision
  const int gdt = level_gdt(h, l);
  auto rounded = [&](Bsr& dst, const Bsr& src64) {
    if (gdt == PUM_F64) { bsr_convert(dst, src64, PUM_F64, s); return; }
    Bsr tmp;
    bsr_convert(tmp, src64, gdt, s);
    bsr_widen(dst, tmp, s);
    // tmp's memory must not be freed (and handed to another thread's allocation) while the
    // widening kernel may still read it
    PUM_CUDA(cudaStreamSynchronize(s));
    bsr_free(tmp);
  };
  if (nested) {
    rounded(F0, L.F064);
    rounded(G, L.G164);
  } else {
    rounded(G, L.G64);
  }
  bsr_transpose(GT, G, s);
  if (nested) bsr_transpose(F0T, F0, s);
  double *v, *vp, *w, *t1, *t2, *dal, *dbe, *dss;
  PUM_CUDA(cudaMalloc(&v, sizeof(double) * N * 5));
  vp = v + N; w = vp + N; t1 = w + N; t2 = t1 + N;
  PUM_CUDA(cudaMalloc(&dal, sizeof(double) * (its + 2) * 3));
  dbe = dal + its + 2;
  dss = dbe + its + 2;
  const unsigned eg = (unsigned)std::min<int64_t>((N + 255) / 256, 2048);
  k_fill_uniform<<<eg, 256, 0, s>>>(v, N, (unsigned long long)(h->sp.lanczos_seed + (uint64_t)l));
  dot_to(ctx, v, v, N, dss);
  k_scale_by_rsqrt<<<eg, 256, 0, s>>>(v, dss, N);
  PUM_CUDA(cudaMemsetAsync(vp, 0, sizeof(double) * N, s));
  PUM_CUDA(cudaMemsetAsync(dbe, 0, sizeof(double) * (its + 2), s));
  EpiArgs e{};
  for (int j = 0; j < its; ++j) {
    // w = G A G^T v   (nested: G1 F0 A F0^T G1^T v)
    e.y = t1; bsr_mv(ctx, GT, PUM_F64, v, EPI_SET, e);
    const double* src = t1;
    if (nested) { e.y = t2; bsr_mv(ctx, F0T, PUM_F64, t1, EPI_SET, e); src = t2; }
    e.y = w; bsr_mv(ctx, L.A, PUM_F64, src, EPI_SET, e);
    if (nested) { e.y = t1; bsr_mv(ctx, F0, PUM_F64, w, EPI_SET, e); e.y = w; bsr_mv(ctx, G, PUM_F64, t1, EPI_SET, e); }
    else { e.y = t1; bsr_mv(ctx, G, PUM_F64, w, EPI_SET, e); PUM_CUDA(cudaMemcpyAsync(w, t1, sizeof(double) * N, cudaMemcpyDeviceToDevice, s)); }
    if (j > 0) k_axpy_dev<<<eg, 256, 0, s>>>(w, vp, dbe, j - 1, 1.0, N);  // w -= beta_{j-1} v_prev
    dot_to(ctx, w, v, N, dal + j);                                          // alpha_j
    k_axpy_dev<<<eg, 256, 0, s>>>(w, v, dal, j, 1.0, N);                     // w -= alpha_j v
    if (j + 1 < its) {
      dot_to(ctx, w, w, N, dss);
      k_lanczos_next<<<eg, 256, 0, s>>>(vp, v, w, dss, dbe, j, N);           // beta_j = ||w||
    } else {
      dot_to(ctx, w, w, N, dss);
      k_lanczos_next<<<1, 32, 0, s>>>(t2, t1, w, dss, dbe, j, 0);            // beta only
    }
    ctx->launches += 4;
    PUM_CUDA(cudaGetLastError());
  }
  std::vector<double> al(its), be(its);
  PUM_CUDA(cudaMemcpyAsync(al.data(), dal, sizeof(double) * its, cudaMemcpyDeviceToHost, s));
  PUM_CUDA(cudaMemcpyAsync(be.data(), dbe, sizeof(double) * its, cudaMemcpyDeviceToHost, s));
  PUM_CUDA(cudaStreamSynchronize(s));
  // truncate where beta_{j+1} <= 1e-14 ||T|| (||T|| estimated by max|alpha| + max beta + beta_{j+1})
  std::vector<double> A_, B_;
  double amax = 0.0, bmax = 0.0;
  for (int j = 0; j < its; ++j) {
    A_.push_back(al[j]);
    amax = std::max(amax, std::fabs(al[j]));
    const double bn = be[j];
    const double tn = amax + bmax + bn;
    if (bn <= 1e-14 * tn || j == its - 1) break;
    B_.push_back(bn);
    bmax = std::max(bmax, bn);
  }
  const double lmax = A_.size() == 1 ? A_[0] : tridiag_lmax(A_, B_);
  L.beta = h->sp.lanczos_safety * lmax;
  cudaFree(v);
  cudaFree(dal);
  bsr_free(G); bsr_free(GT); bsr_free(F0); bsr_free(F0T);
  PUM_CHECK(std::isfinite(L.beta) && L.beta > 0.0, PUM_ERR_BREAKDOWN, "Lanczos estimate is not positive");
}

// ----------------------------------------------------------------------------- coarse

// Dense Cholesky of the coarsest operator, one CTA, in global memory (row-major).
__global__ void k_dense_from_bsr(const int* rp, const int* ci, const double* v, int stride, int n, int d, double* D) {
  const int N = n * d;
  for (int t = threadIdx.x + blockIdx.x * blockDim.x; t < N * N; t += blockDim.x * gridDim.x) D[t] = 0.0;
  __syncthreads();
}

__global__ void k_dense_scatter(const int* rp, const int* ci, const double* v, int stride, int n, int d, double* D) {
  const int N = n * d;
  for (int i = blockIdx.x; i < n; i += gridDim.x)
    for (int b = rp[i]; b < rp[i + 1]; ++b) {
      const int j = ci[b];
      for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
        const int r = e / d, c = e - (e / d) * d;
        D[(int64_t)(i * d + r) * N + j * d + c] = v[(int64_t)b * stride + e];
      }
    }
}

__global__ void k_dense_cholesky(double* D, int N, DevStatus* st) {
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < N; ++j) {
    if (threadIdx.x == 0) {
      const double v = D[(int64_t)j * N + j];
      if (!(v > 0.0)) fail = 1;
      D[(int64_t)j * N + j] = sqrt(fmax(v, 0.0));
    }
    __syncthreads();
    if (fail) {
      if (threadIdx.x == 0) set_status(st, PUM_ERR_NOT_SPD, j, kWhereCoarse);
      return;
    }
    const double ljj = D[(int64_t)j * N + j];
    for (int i = j + 1 + threadIdx.x; i < N; i += blockDim.x) D[(int64_t)i * N + j] /= ljj;
    __syncthreads();
    for (int t = threadIdx.x; t < (N - j - 1) * (N - j - 1); t += blockDim.x) {
      const int i = j + 1 + t / (N - j - 1), l = j + 1 + t % (N - j - 1);
      if (l <= i) D[(int64_t)i * N + l] -= D[(int64_t)i * N + j] * D[(int64_t)l * N + j];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    const int i = t / N, l = t % N;
    if (l > i) D[t] = 0.0;
  }
}

void coarse_factor(pum_ctx* ctx, pum_hier* h) {
  Level& L = h->lv.back();
  const int N = L.n * L.d;
  PUM_CHECK(N <= 4096, PUM_ERR_UNSUPPORTED, "coarsest level larger than 4096 unknowns");
  if (h->coarse.L) cudaFree(h->coarse.L);
  h->coarse.N = N;
  PUM_CUDA(cudaMalloc(&h->coarse.L, sizeof(double) * (size_t)N * N));
  cudaStream_t s = ctx->stream;
  PUM_CUDA(cudaMemsetAsync(h->coarse.L, 0, sizeof(double) * (size_t)N * N, s));
  k_dense_scatter<<<std::min(L.n, 1024), 128, 0, s>>>(L.A.row_ptr, L.A.col_idx, (const double*)L.A.vals, L.A.stride,
                                                     L.n, L.d, h->coarse.L);
  k_dense_cholesky<<<1, 512, 0, s>>>(h->coarse.L, N, ctx->status);
  ctx->launches += 2;
  PUM_CUDA(cudaGetLastError());
  PUM_CUDA(cudaStreamSynchronize(s));
  check_status(ctx, "coarse Cholesky");
}

}  // namespace pum

// ----------------------------------------------------------------------------- candidates (C-ABI)

extern "C" pum_status pum_fsai_candidates(pum_ctx* ctx, pum_hier* h, int level, pum_candidates* out) {
  using namespace pum;
  if (!ctx || !h || !out) return PUM_ERR_INVALID_ARG;
  *out = pum_candidates{};
  try {
    ctx->last_error.clear();
    PUM_CUDA(cudaSetDevice(ctx->device));
    PUM_CHECK(h->setup_done, PUM_ERR_INVALID_ARG, "bfsai_setup has not run");
    PUM_CHECK(!h->fp.nested, PUM_ERR_INVALID_ARG, "candidates of a nested set-up are not supported");
    PUM_CHECK(level >= 0 && level + 1 < (int)h->lv.size(), PUM_ERR_INVALID_ARG, "level out of range or coarsest");
    Level& L = h->lv[level];
    const Pattern P0 = initial_pattern(L.A, h->fp.p0);
    Bsr G0;
    fsai_factor(ctx, L.A, P0, G0, nullptr, nullptr);
    CandidateSet cs;
    try {
      candidates_build(ctx, L.A, G0, P0.rows, L.m, cs);
    } catch (...) {
      bsr_free(G0);
      throw;
    }
    bsr_free(G0);
    // labels: membership in the level's current pattern (host copy of G's pattern)
    const Bsr& G = L.G64;
    std::vector<float> y(cs.n, 0.0f);
    for (int k = 0; k < L.n; ++k)
      for (int q = cs.rp[k]; q < cs.rp[k + 1]; ++q)
        y[q] = std::binary_search(G.h_col_idx.begin() + G.h_row_ptr[k], G.h_col_idx.begin() + G.h_row_ptr[k + 1],
                                  cs.col[q])
                   ? 1.0f
                   : 0.0f;
    float* dy = nullptr;
    PUM_CUDA(cudaMalloc(&dy, sizeof(float) * std::max<int64_t>(cs.n, 1)));
    if (cs.n) PUM_CUDA(cudaMemcpy(dy, y.data(), sizeof(float) * cs.n, cudaMemcpyHostToDevice));
    out->n = cs.n;
    out->row = cs.d_row;
    out->col = cs.d_col;
    out->x = cs.d_x;
    out->y = dy;
    return PUM_OK;
  } catch (const Error& e) {
    ctx->last_error = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    ctx->last_error = "host allocation failed";
    return PUM_ERR_OOM;
  }
}
