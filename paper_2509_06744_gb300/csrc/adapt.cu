// Algorithm 1 (adaptive block-FSAI pattern, Section 2.1) with every block row carried through
// all of its steps by one CTA, in one launch per level.
//
// The steps of Algorithm 1 change row k's pattern from row k's own scores only (the rows are
// independent: F and H of a step are formed from the patterns at its start, and row k's scores
// read A and P_k alone), so a CTA can take a row from P0_k to its final pattern without any
// global step barrier.  Inside the row, the factorisation of A[P~_k, P~_k] is grown block by
// block instead of being recomputed every step.  With the blocks of P~_k in the order they
// joined the pattern, j_0, j_1, ..., the Cholesky factor L of A[P~, P~] has block rows
// [Z_{j_q}^T, L_q], where Z_{j_q} = L_{<q}^{-1} A[{j_0..j_{q-1}}, j_q] and L_q = chol(W_{j_q}),
// W_c = A_cc - Z_c^T Z_c.  Every column c the row tracks (the row k itself, the pending blocks
// of P0, the admissible candidates) keeps Z_c = L^{-1} A[P~, c] and the d x d blocks
//     W_c = A_cc - Z_c^T Z_c,    H_kc = A_kc - Z_k^T Z_c  (= (F A)_kc, Lemma 2.8),
// and when block j_q joins, Z_c gains the block row
//     v = L_q^{-1} (A[j_q, c] - Z_{j_q}^T Z_c),   W_c -= v^T v,   H_kc -= u_q^T v,
// with u_q the block row Z_k gains (for c = k: S_kk = W_k -= u_q^T u_q).  A candidate's gain is
//     rho_c = det(W_c - H_kc^T S_kk^{-1} H_kc) / det(W_c)             (Lemma 2.8)
// from two d x d Cholesky factorisations; the argmin, the tie band and tau are Algorithm 1's
// (smallest column among rho_c <= rho_min (1 + tie_rel); stop when rho_c* >= tau).  A candidate
// whose W_c or Schur complement fails its Cholesky factorisation has no rho_c and is not chosen;
// a row without a computable candidate retires.  A failed Cholesky of a joining block's W (the
// block Cholesky of A[P~, P~]) or of S_kk reports PUM_ERR_NOT_SPD with the row, as the from-
// scratch factorisation would.
//
// Work layout: persistent CTAs take rows from an atomic counter; a row's columns live in
// "slots" of the CTA's slab in global memory (Z_c: s_cap x d, row-major; W_c, H_kc, chol(W_c)
// and the reciprocal diagonal of that factor), each warp works on whole slots, and the small
// per-row tables (columns, pattern order, scores) are in shared memory.  All arithmetic is FP64.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "pum_internal.cuh"
#include "small_dense.cuh"

namespace pum {

namespace {

constexpr int kAdaptThreads = 128;
constexpr int kAdaptWarps = kAdaptThreads / 32;

struct AdaptArgs {
  const int* arp;
  const int* aci;
  const double* av;
  int astride;
  int n;            // block rows
  const int* p0rp;  // initial pattern P0 (sorted rows, diagonal included)
  const int* p0ci;
  int t_max;
  double tau, tie_rel;
  int np_cap;       // most blocks P~_k can hold
  int slots;        // slots per CTA (1 + P0 blocks + candidates)
  int max_row;      // longest block row of A
  int64_t slot_doubles;
  double* slab;     // gridDim.x * slots * slot_doubles
  int* next_row;    // work counter (starts at 0)
  const int* work;  // block rows to process (NULL: all n, in order)
  int n_work;
  int* out_np;      // per row: |P_k| (diagonal included)
  int* out_cols;    // per row: np_cap + 1 sorted columns
  double* fmas;     // accumulated FP64 multiply-adds of the algorithm (all rows)
  double* out_g;    // optional: per row np_cap + 1 blocks of G = L_S^-1 F in ascending column order
  double* out_f;    // optional: the same blocks of F
  double* out_ld;   // with out_g: per row log det S_kk
  DevStatus* status;
};

// FP64 multiply-adds of the kernel's steps (the algorithm's arithmetic; square roots and
// reciprocals not counted): a column's update when block q joins (Gram over q D rows, the
// triangular solve, W and, for a candidate, H), a d x d Cholesky, and a candidate's score.
template <int D>
__host__ __device__ constexpr double fma_replay(int q, bool is_row) {
  return (double)q * D * D * D + 0.5 * D * D * (D - 1) + (double)D * D * D + (is_row ? 0.0 : (double)D * D * D);
}
template <int D>
__host__ __device__ constexpr double fma_chol() { return (double)(D * D * D - D) / 6.0; }
template <int D>
__host__ __device__ constexpr double fma_score() {
  return 0.5 * D * D * (D - 1) + (double)D * D * D + 2.0 * fma_chol<D>();
}

// Slot layout (doubles): Z [s_cap * D] | W [D * D] | H [D * D] | LW [D * D] | inverse diagonal of LW [D].
template <int D>
struct SlotView {
  double* Z;
  double* W;
  double* H;
  double* LW;
  double* inv;
  __device__ SlotView(double* base, int s_cap) {
    Z = base;
    W = Z + (int64_t)s_cap * D;
    H = W + D * D;
    LW = H + D * D;
    inv = LW + D * D;
  }
};

// Block j_q joins the factor; bring column c (slot sc, Z rows [0, q D) valid) up to date:
// v = L_q^{-1} (A[j_q, col] - Z_q^T Z_c), Z_c rows [q D, q D + D) = v, W_c -= v^T v, and unless
// c is the row itself, H_kc -= u_q^T v.  R: per-warp scratch of D * D doubles.
template <int D>
__device__ void warp_replay(const AdaptArgs& a, int s_cap, int q, int jq, const SlotView<D>& Q, const SlotView<D>& C,
                            int col, const double* Zk, bool is_row, double* R) {
  const int lane = threadIdx.x & 31;
  int blk = 0;
  if (lane == 0) blk = find_blk(a.arp, a.aci, jq, col);
  blk = __shfl_sync(0xffffffffu, blk, 0);
  const double* Ab = blk >= 0 ? a.av + (int64_t)blk * a.astride : nullptr;
  const int rows = q * D;
  for (int e = lane; e < D * D; e += 32) {
    const int r = e / D, c = e - (e / D) * D;
    double acc = Ab ? Ab[e] : 0.0;
    const double* zq = Q.Z + r;
    const double* zc = C.Z + c;
    for (int i = 0; i < rows; ++i) acc -= zq[(int64_t)i * D] * zc[(int64_t)i * D];
    R[e] = acc;
  }
  __syncwarp();
  warp_lsolve<D>(Q.LW, Q.inv, R);
  for (int e = lane; e < D * D; e += 32) C.Z[(int64_t)rows * D + e] = R[e];
  const double* u = Zk + (int64_t)rows * D;
  for (int e = lane; e < D * D; e += 32) {
    const int r = e / D, c = e - (e / D) * D;
    double w = C.W[e], h = is_row ? 0.0 : C.H[e];
#pragma unroll
    for (int t = 0; t < D; ++t) {
      const double vc = R[t * D + c];
      w -= R[t * D + r] * vc;
      if (!is_row) h -= u[t * D + r] * vc;
    }
    C.W[e] = w;
    if (!is_row) C.H[e] = h;
  }
  __syncwarp();
  (void)s_cap;
}

// Load A block (row, col) into dst (zero when the block is not stored).
template <int D>
__device__ void warp_load_block(const AdaptArgs& a, int row, int col, double* dst) {
  const int lane = threadIdx.x & 31;
  int blk = 0;
  if (lane == 0) blk = find_blk(a.arp, a.aci, row, col);
  blk = __shfl_sync(0xffffffffu, blk, 0);
  for (int e = lane; e < D * D; e += 32) dst[e] = blk >= 0 ? a.av[(int64_t)blk * a.astride + e] : 0.0;
}

// rho_c of Lemma 2.8 for slot C against the row's factor of S_kk (slot Kr): U = L_S^{-1} H_kc,
// X = W_c - U^T U; also leaves chol(W_c) in C.LW.  Returns -1 when rho_c is not computable.
template <int D>
__device__ double warp_score(const SlotView<D>& Kr, const SlotView<D>& C, double* R, double* X) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < D * D; e += 32) R[e] = C.H[e];
  __syncwarp();
  warp_lsolve<D>(Kr.LW, Kr.inv, R);
  for (int e = lane; e < D * D; e += 32) {
    const int r = e / D, c = e - (e / D) * D;
    double v = C.W[e];
#pragma unroll
    for (int t = 0; t < D; ++t) v -= R[t * D + r] * R[t * D + c];
    X[e] = v;
  }
  __syncwarp();
  double mx, mw;
  int ex, ew;
  const bool okx = warp_chol<D>(X, R, X + D * D, mx, ex);  // X + D*D: throwaway reciprocal diagonal
  const bool okw = warp_chol<D>(C.W, C.LW, C.inv, mw, ew);
  if (!okx || !okw) return -1.0;
  return ldexp(mx / mw, ex - ew);
}

// Scores of small blocks (D <= 10) are split in two passes so that the two d x d Cholesky
// factorisations of a score run one candidate per thread instead of one matrix per warp (whose
// pivots and shrinking trailing triangles leave most lanes idle): first, per candidate and by one
// warp, X = W_c - U^T U with U = L_S^{-1} H_kc, stored in the candidate's LW area; then, per
// candidate and by one thread, det X and chol(W_c) into LW (kept for the candidate's possible
// joining) and rho_c = det X / det W_c.  The per-thread factorisation performs the operations of
// warp_chol in the same order for every element, so the scores are the same bit for bit.
template <int D>
constexpr bool kThreadChol = D <= 10;

template <int D>
__device__ void warp_score_x(const SlotView<D>& Kr, const SlotView<D>& C, double* R) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < D * D; e += 32) R[e] = C.H[e];
  __syncwarp();
  warp_lsolve<D>(Kr.LW, Kr.inv, R);
  for (int e = lane; e < D * D; e += 32) {
    const int r = e / D, c = e - (e / D) * D;
    double v = C.W[e];
#pragma unroll
    for (int t = 0; t < D; ++t) v -= R[t * D + r] * R[t * D + c];
    C.LW[e] = v;
  }
  __syncwarp();
}

// Cholesky of the symmetric D x D matrix src (row-major, lower part read) by one thread, with the
// element operations of warp_chol in its order; the lower factor into dst and the reciprocal
// diagonal into inv when given.  det = mant * 2^expo.  False when a pivot is not positive.
template <int D>
__device__ bool thread_chol(const double* src, double* dst, double* inv, double& mant, int& expo) {
  double m[D * (D + 1) / 2];  // packed lower triangle: (i, c) at i (i + 1) / 2 + c
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int c = 0; c <= i; ++c) m[i * (i + 1) / 2 + c] = src[i * D + c];
  mant = 1.0;
  expo = 0;
  bool ok = true;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const double piv = m[j * (j + 1) / 2 + j];
    if (!(piv > 0.0)) {
      ok = false;
      break;
    }
    const double l = sqrt(piv);
    const double il = 1.0 / l;
    int ex = 0;
    mant = frexp(mant * piv, &ex);
    expo += ex;
    m[j * (j + 1) / 2 + j] = l;
    if (inv) inv[j] = il;
#pragma unroll
    for (int i = j + 1; i < D; ++i) m[i * (i + 1) / 2 + j] *= il;
#pragma unroll
    for (int i = j + 1; i < D; ++i)
#pragma unroll
      for (int c = j + 1; c <= i; ++c) m[i * (i + 1) / 2 + c] -= m[i * (i + 1) / 2 + j] * m[c * (c + 1) / 2 + j];
  }
  if (dst)
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int c = 0; c <= i; ++c) dst[i * D + c] = m[i * (i + 1) / 2 + c];
  return ok;
}

// rho_c from X (in C.LW, left by warp_score_x) and W_c, one thread; chol(W_c) into C.LW / C.inv.
template <int D>
__device__ double thread_score(const SlotView<D>& C) {
  double mx, mw;
  int ex, ew;
  const bool okx = thread_chol<D>(C.LW, nullptr, nullptr, mx, ex);
  const bool okw = thread_chol<D>(C.W, C.LW, C.inv, mw, ew);
  if (!okx || !okw) return -1.0;
  return ldexp(mx / mw, ex - ew);
}

// Four CTAs per SM (the launch's CTA count): the register cap spills a little of the d = 10
// per-thread Cholesky, which measured faster than three CTAs per SM without spills.
template <int D>
__global__ void __launch_bounds__(kAdaptThreads, 4) k_adaptive_rows(AdaptArgs a) {
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s_cap = a.np_cap * D;
  // shared tables
  double* scratch = sm;                                  // kAdaptWarps * 2 * (D*D + D)
  double* s_rho = scratch + kAdaptWarps * 2 * (D * D + D); // slots
  int* s_col = reinterpret_cast<int*>(s_rho + a.slots);  // slots: column of the slot
  int* s_state = s_col + a.slots;                        // slots: 0 free, 1 pending P0, 2 candidate, 3 in P~, 4 row
  int* s_done = s_state + a.slots;                       // slots: block rows of Z valid
  int* s_jslot = s_done + a.slots;                       // np_cap: slot of the q-th block of P~
  int* s_tmp = s_jslot + a.np_cap;                       // (np_cap + 1) * max_row: candidate build
  __shared__ int s_row, s_np, s_nslot, s_fail, s_choice, s_np0;
  __shared__ double s_fma;
  double* R = scratch + warp * 2 * (D * D + D);
  double* X = R + D * D;
  double* slab = a.slab + (int64_t)blockIdx.x * a.slots * a.slot_doubles;
  auto slot = [&](int s) { return SlotView<D>(slab + (int64_t)s * a.slot_doubles, s_cap); };

  for (;;) {
    if (threadIdx.x == 0) {
      const int w = atomicAdd(a.next_row, 1);
      s_row = w < a.n_work ? (a.work ? a.work[w] : w) : -1;
    }
    __syncthreads();
    const int k = s_row;
    if (k < 0) break;
    // ---- slots: 0 = the row (W = S_kk), then the blocks of P0~ in ascending order
    if (threadIdx.x == 0) {
      s_fail = 0;
      s_np = 0;
      s_fma = 0.0;
      int ns = 1;
      s_col[0] = k;
      s_state[0] = 4;
      s_done[0] = 0;
      for (int b = a.p0rp[k]; b < a.p0rp[k + 1] && ns < a.slots; ++b) {
        const int c = a.p0ci[b];
        if (c >= k) break;
        s_col[ns] = c;
        s_state[ns] = 1;
        s_done[ns] = 0;
        ++ns;
      }
      s_nslot = ns;
      s_np0 = ns - 1;
    }
    __syncthreads();
    if (s_np0 > a.np_cap) {
      if (threadIdx.x == 0) set_status(a.status, PUM_ERR_UNSUPPORTED, k, kWhereAdaptive);
      continue;
    }
    for (int s = warp; s < s_nslot; s += kAdaptWarps) {
      SlotView<D> C = slot(s);
      warp_load_block<D>(a, s_col[s], s_col[s], C.W);  // A_cc
      if (s > 0) warp_load_block<D>(a, k, s_col[s], C.H);  // A_kc
    }
    __syncthreads();
    const SlotView<D> Kr = slot(0);
    // ---- the blocks of P0~ join in ascending order (the block Cholesky of A[P0~, P0~])
    for (int q = 0; q < s_np0; ++q) {
      const int sq = 1 + q;
      if (warp == 0) {
        double m;
        int e;
        SlotView<D> J = slot(sq);
        if (!warp_chol<D>(J.W, J.LW, J.inv, m, e) && lane == 0) s_fail = 1;
      }
      __syncthreads();
      if (s_fail) break;
      if (threadIdx.x == 0) {
        s_jslot[q] = sq;
        s_state[sq] = 3;
      }
      const SlotView<D> Q = slot(sq);
      if (warp == 0) warp_replay<D>(a, s_cap, q, s_col[sq], Q, Kr, k, Kr.Z, true, R);
      __syncthreads();
      for (int s = 2 + q + warp; s < s_nslot; s += kAdaptWarps)
        warp_replay<D>(a, s_cap, q, s_col[sq], Q, slot(s), s_col[s], Kr.Z, false, R);
      __syncthreads();
      if (threadIdx.x == 0) {
        s_np = q + 1;
        s_fma += fma_chol<D>() + fma_replay<D>(q, true) + (s_nslot - 2 - q) * fma_replay<D>(q, false);
      }
    }
    __syncthreads();
    if (!s_fail && warp == 0) {  // L_S = chol(S_kk)
      double m;
      int e;
      if (!warp_chol<D>(Kr.W, Kr.LW, Kr.inv, m, e) && lane == 0) s_fail = 1;
      if (lane == 0) s_fma += fma_chol<D>();
    }
    __syncthreads();
    if (s_fail) {
      if (threadIdx.x == 0) set_status(a.status, PUM_ERR_NOT_SPD, k, kWhereFsai);
      __syncthreads();
      continue;
    }
    // ---- admissible set: c < k in the A-rows of P_k, not in P_k (structural, R10)
    if (threadIdx.x == 0) {
      int m = 0;
      for (int s = 0; s < s_nslot; ++s) {
        const int j = s_col[s];
        for (int b = a.arp[j]; b < a.arp[j + 1]; ++b) s_tmp[m++] = a.aci[b];
      }
      int ns = s_nslot;
      for (int t = 0; t < m; ++t) {
        const int c = s_tmp[t];
        if (c >= k) continue;
        bool seen = false;
        for (int s = 0; s < ns && !seen; ++s) seen = s_col[s] == c;
        if (seen) continue;
        if (ns >= a.slots) {
          s_fail = 2;
          break;
        }
        s_col[ns] = c;
        s_state[ns] = 2;
        s_done[ns] = 0;
        ++ns;
      }
      s_nslot = ns;
    }
    __syncthreads();
    if (s_fail) {
      if (threadIdx.x == 0) set_status(a.status, PUM_ERR_UNSUPPORTED, k, kWhereAdaptive);
      __syncthreads();
      continue;
    }
    // new candidates: A_cc, A_kc, then their Z brought up to the current factor
    for (int s = 1 + s_np0 + warp; s < s_nslot; s += kAdaptWarps) {
      SlotView<D> C = slot(s);
      warp_load_block<D>(a, s_col[s], s_col[s], C.W);
      warp_load_block<D>(a, k, s_col[s], C.H);
      __syncwarp();
      for (int q = 0; q < s_np; ++q) {
        const int sq = s_jslot[q];
        warp_replay<D>(a, s_cap, q, s_col[sq], slot(sq), C, s_col[s], Kr.Z, false, R);
      }
      if (lane == 0) s_done[s] = s_np;
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int q = 0; q < s_np; ++q) s_fma += (s_nslot - 1 - s_np0) * fma_replay<D>(q, false);
    // ---- the steps of Algorithm 1
    for (int t = 0; t < a.t_max; ++t) {
      if constexpr (kThreadChol<D>) {
        for (int s = warp; s < s_nslot; s += kAdaptWarps)
          if (s_state[s] == 2) warp_score_x<D>(Kr, slot(s), R);
        __syncthreads();
        for (int s = threadIdx.x; s < s_nslot; s += kAdaptThreads)
          if (s_state[s] == 2) s_rho[s] = thread_score<D>(slot(s));
      } else {
        for (int s = warp; s < s_nslot; s += kAdaptWarps) {
          if (s_state[s] != 2) continue;
          const double rho = warp_score<D>(Kr, slot(s), R, X);
          if (lane == 0) s_rho[s] = rho;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int s = 0; s < s_nslot; ++s) s_fma += s_state[s] == 2 ? fma_score<D>() : 0.0;
        double rmin = -1.0;
        for (int s = 0; s < s_nslot; ++s)
          if (s_state[s] == 2 && s_rho[s] >= 0.0 && (rmin < 0.0 || s_rho[s] < rmin)) rmin = s_rho[s];
        int choice = -1;
        if (rmin >= 0.0) {
          const double thr = rmin * (1.0 + a.tie_rel);
          for (int s = 0; s < s_nslot; ++s)
            if (s_state[s] == 2 && s_rho[s] >= 0.0 && s_rho[s] <= thr && (choice < 0 || s_col[s] < s_col[choice]))
              choice = s;
          // the stop test with the tie band: a gain 1 - rho below tie_rel (relative to tau) is
          // rounding, not a gain (candidates whose coupling H_kc is zero to rounding have rho = 1)
          if (!(s_rho[choice] < a.tau * (1.0 - a.tie_rel))) choice = -1;
        }
        s_choice = choice;
        if (choice >= 0) {
          if (s_np >= a.np_cap) {
            s_fail = 2;
          } else {
            s_jslot[s_np] = choice;
            s_state[choice] = 3;
          }
        }
      }
      __syncthreads();
      if (s_choice < 0 || s_fail) break;
      const int q = s_np;
      const int sq = s_choice;
      if (t == a.t_max - 1) {
        if (a.out_g && warp == 0) {  // the factor needs the row's state with the last block too
          warp_replay<D>(a, s_cap, q, s_col[sq], slot(sq), Kr, k, Kr.Z, true, R);
          double m;
          int e;
          if (!warp_chol<D>(Kr.W, Kr.LW, Kr.inv, m, e) && lane == 0) s_fail = 1;
          if (lane == 0) s_fma += fma_replay<D>(q, true) + fma_chol<D>();
        }
        if (threadIdx.x == 0) s_np = q + 1;
        __syncthreads();
        break;
      }
      // the row gains u_q; S_kk -= u_q^T u_q; L_S = chol(S_kk)
      const SlotView<D> Q = slot(sq);
      if (warp == 0) {
        warp_replay<D>(a, s_cap, q, s_col[sq], Q, Kr, k, Kr.Z, true, R);
        double m;
        int e;
        if (!warp_chol<D>(Kr.W, Kr.LW, Kr.inv, m, e) && lane == 0) s_fail = 1;
      } else if (threadIdx.x == 32) {
        // candidates new with c*: c < k in A's row c*, not yet tracked
        const int j = s_col[sq];
        int ns = s_nslot;
        for (int b = a.arp[j]; b < a.arp[j + 1]; ++b) {
          const int c = a.aci[b];
          if (c >= k) break;
          bool seen = false;
          for (int s = 0; s < ns && !seen; ++s) seen = s_col[s] == c;
          if (seen) continue;
          if (ns >= a.slots) {
            s_fail = 2;
            break;
          }
          s_col[ns] = c;
          s_state[ns] = 2;
          s_done[ns] = 0;
          ++ns;
        }
        s_nslot = ns;
      }
      __syncthreads();
      if (s_fail) break;
      // every candidate brought up to the factor with q + 1 blocks (new ones from the start)
      for (int s = warp; s < s_nslot; s += kAdaptWarps) {
        if (s_state[s] != 2) continue;
        SlotView<D> C = slot(s);
        int done = s_done[s];
        if (done == 0) {  // new with c*: A_cc and A_kc first
          warp_load_block<D>(a, s_col[s], s_col[s], C.W);
          warp_load_block<D>(a, k, s_col[s], C.H);
          __syncwarp();
        }
        double f = 0.0;
        for (; done <= q; ++done) {
          const int sj = s_jslot[done];
          warp_replay<D>(a, s_cap, done, s_col[sj], slot(sj), C, s_col[s], Kr.Z, false, R);
          f += fma_replay<D>(done, false);
        }
        if (lane == 0) {
          s_done[s] = done;
          atomicAdd(&s_fma, f);
        }
      }
      if (threadIdx.x == 0) {
        s_np = q + 1;
        atomicAdd(&s_fma, fma_replay<D>(q, true) + fma_chol<D>());
      }
      __syncthreads();
    }
    if (s_fail) {
      if (threadIdx.x == 0)
        set_status(a.status, s_fail == 1 ? PUM_ERR_NOT_SPD : PUM_ERR_UNSUPPORTED, k,
                   s_fail == 1 ? kWhereFsai : kWhereAdaptive);
      __syncthreads();
      continue;
    }
    // ---- G and F of the row from the grown factor (Definition 2.2): with L L^T = A[P~,P~] in
    // the order the blocks joined, Y = L^-T Z_k = A[P~,P~]^-1 A[P~,k], F[k,P~] = -Y^T and
    // G = L_S^-1 F, written in ascending column order (the diagonal block last)
    if (a.out_g) {
      const int np = s_np;
      int* pos = s_tmp;  // sorted position of the q-th joined block
      if (threadIdx.x == 0) {
        for (int q = 0; q < np; ++q) {
          int r = 0;
          const int cq = s_col[s_jslot[q]];
          for (int q2 = 0; q2 < np; ++q2) r += s_col[s_jslot[q2]] < cq;
          pos[q] = r;
        }
      }
      __syncthreads();
      double* gout = a.out_g + (int64_t)k * (a.np_cap + 1) * D * D;
      if (warp == 0) {
        // backward block substitution: Y_q = L_q^-T (Z_k[q] - sum_{q' > q} Z_{j_q'}[q] Y_q')
        for (int q = np - 1; q >= 0; --q) {
          for (int e = lane; e < D * D; e += 32) R[e] = Kr.Z[(int64_t)q * D * D + e];
          __syncwarp();
          for (int q2 = q + 1; q2 < np; ++q2) {
            const double* Zq2 = slot(s_jslot[q2]).Z + (int64_t)q * D * D;  // block (q, q2) of L^T
            const double* Y2 = gout + (int64_t)pos[q2] * D * D;
            for (int e = lane; e < D * D; e += 32) {
              const int r = e / D, c = e - (e / D) * D;
              double v = R[e];
#pragma unroll
              for (int t2 = 0; t2 < D; ++t2) v -= Zq2[r * D + t2] * Y2[t2 * D + c];
              R[e] = v;
            }
            __syncwarp();
          }
          const SlotView<D> Lq = slot(s_jslot[q]);
          warp_ltsolve<D>(Lq.LW, Lq.inv, R);
          for (int e = lane; e < D * D; e += 32) gout[(int64_t)pos[q] * D * D + e] = R[e];
          __syncwarp();
        }
      }
      __syncthreads();
      // F = -Y^T and G = L_S^-1 F block by block; the diagonal block F = I, G = L_S^-1
      for (int q = warp; q <= np; q += kAdaptWarps) {
        const int pq = q < np ? pos[q] : np;
        double* gb = gout + (int64_t)pq * D * D;
        for (int e = lane; e < D * D; e += 32) {
          const int r = e / D, c = e - (e / D) * D;
          R[e] = q < np ? -gb[c * D + r] : (r == c ? 1.0 : 0.0);
        }
        __syncwarp();
        if (a.out_f)
          for (int e = lane; e < D * D; e += 32) a.out_f[((int64_t)k * (a.np_cap + 1) + pq) * D * D + e] = R[e];
        warp_lsolve<D>(Kr.LW, Kr.inv, R);
        for (int e = lane; e < D * D; e += 32) gb[e] = R[e];
        __syncwarp();
      }
      if (warp == 0) {
        double m;
        int e;
        warp_chol<D>(Kr.W, X, X + D * D, m, e);  // log det S_kk (S was factored successfully)
        if (lane == 0) {
          a.out_ld[k] = log(m) + e * 0.6931471805599453;
          s_fma += (double)np * (np - 1) / 2.0 * D * D * D + np * 0.5 * D * D * (D - 1) +
                   (np + 1) * 0.5 * D * D * (D - 1) + fma_chol<D>();
        }
      }
      __syncthreads();
    }
    // ---- the final pattern P~_k + {k}, ascending
    if (threadIdx.x == 0) {
      const int np = s_np;
      int* out = a.out_cols + (int64_t)k * (a.np_cap + 1);
      for (int q = 0; q < np; ++q) {
        const int c = s_col[s_jslot[q]];
        int i = q;
        while (i > 0 && out[i - 1] > c) {
          out[i] = out[i - 1];
          --i;
        }
        out[i] = c;
      }
      out[np] = k;
      a.out_np[k] = np + 1;
      atomicAdd(a.fmas, s_fma);
    }
    __syncthreads();
  }
}

template <int D>
size_t adapt_smem(int slots, int np_cap, int max_row) {
  return sizeof(double) * ((size_t)kAdaptWarps * 2 * (D * D + D) + slots) +
         sizeof(int) * ((size_t)3 * slots + np_cap + (size_t)(np_cap + 1) * max_row);
}

template <int D>
void launch_adapt(pum_ctx* ctx, AdaptArgs& a, int ctas) {
  const size_t smem = adapt_smem<D>(a.slots, a.np_cap, a.max_row);
  const void* kern = (const void*)k_adaptive_rows<D>;
  allow_max_dynamic_smem(kern);
  k_adaptive_rows<D><<<ctas, kAdaptThreads, smem, ctx->stream>>>(a);
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
}

// Copy row k's staged blocks (ascending columns) into the BSR's row k.
__global__ void k_stage_to_bsr(double* __restrict__ dst, int dstride, const double* __restrict__ stage, int cap,
                               const int* __restrict__ rp, int dd) {
  const int k = blockIdx.x;
  const int b0 = rp[k], nb = rp[k + 1] - b0;
  for (int t = threadIdx.x; t < nb * dd; t += blockDim.x) {
    const int i = t / dd, e = t - (t / dd) * dd;
    dst[(int64_t)(b0 + i) * dstride + e] = stage[((int64_t)k * cap + i) * dd + e];
  }
}

}  // namespace

// Final patterns of Algorithm 1 for every block row of A (FP64) from the initial pattern P0
// (rows sorted, diagonal included; the nested FSAI passes lower(P(A)) for its inner level too);
// rows[k] receives P_k sorted.  Returns false (nothing launched) when the block size has no
// instantiation.
bool adaptive_patterns_device(pum_ctx* ctx, const Bsr& A, const std::vector<std::vector<int>>& P0, int t_max,
                              double tau, double tie_rel, std::vector<std::vector<int>>& rows, double* fp64_flops,
                              const std::vector<int>* work_rows, Bsr* G, Bsr* F, double* logdet) {
  const int d = A.d, n = A.n_brows;
  if (d != 3 && d != 6 && d != 10 && d != 15 && d != 20 && d != 21) return false;
  int np0 = 0;
  std::vector<int> p0rp(n + 1, 0), p0ci;
  for (int i = 0; i < n; ++i) {
    int c = 0;
    for (int j : P0[i]) c += j < i;
    np0 = std::max(np0, c);
    p0ci.insert(p0ci.end(), P0[i].begin(), P0[i].end());
    p0rp[i + 1] = (int)p0ci.size();
  }
  AdaptArgs a{};
  a.arp = A.row_ptr;
  a.aci = A.col_idx;
  a.av = (const double*)A.vals;
  a.astride = A.stride;
  a.n = n;
  a.t_max = t_max;
  a.tau = tau;
  a.tie_rel = tie_rel;
  a.np_cap = np0 + std::max(t_max, 0);
  a.max_row = std::max(A.max_row_nnzb, 1);
  PUM_CHECK(a.np_cap <= 64, PUM_ERR_UNSUPPORTED, "adaptive FSAI: row pattern longer than 64 blocks");
  // Every tracked column comes from the A-row of a member of P_k (|P_k| <= np_cap + 1), which
  // bounds the slots a row can need; a first launch uses at most 128 slots per row (enough for
  // the 3x3 and 5x5 block stencils of the PUM levels) and rows beyond that rerun with the bound.
  const int bound = std::max(1 + np0, std::min(n, 1 + np0 + (a.np_cap + 1) * a.max_row));
  const int64_t sd = (int64_t)a.np_cap * d * d + 3 * d * d + d;
  a.slot_doubles = (sd + 1) / 2 * 2;  // 16-byte aligned slots
  cudaStream_t s = ctx->stream;
  int *dp0rp = nullptr, *dp0ci = nullptr, *counter = nullptr, *out_np = nullptr, *out_cols = nullptr;
  int* dwork = nullptr;
  a.n_work = work_rows ? (int)work_rows->size() : n;
  if (work_rows && !work_rows->empty()) {
    PUM_CUDA(cudaMalloc(&dwork, sizeof(int) * work_rows->size()));
    PUM_CUDA(cudaMemcpyAsync(dwork, work_rows->data(), sizeof(int) * work_rows->size(), cudaMemcpyHostToDevice,
                             ctx->stream));
  }
  a.work = dwork;
  PUM_CHECK(!G || !work_rows, PUM_ERR_INVALID_ARG, "adaptive FSAI: factors need every row");
  double *dstage_g = nullptr, *dstage_f = nullptr, *dld = nullptr;
  if (G) {
    const size_t sb = sizeof(double) * (size_t)n * (a.np_cap + 1) * d * d;
    PUM_CUDA(cudaMalloc(&dstage_g, sb));
    if (F) PUM_CUDA(cudaMalloc(&dstage_f, sb));
    PUM_CUDA(cudaMalloc(&dld, sizeof(double) * std::max(n, 1)));
  }
  a.out_g = dstage_g;
  a.out_f = dstage_f;
  a.out_ld = dld;
  double* dfma = nullptr;
  PUM_CUDA(cudaMalloc(&dfma, sizeof(double)));
  PUM_CUDA(cudaMalloc(&dp0rp, sizeof(int) * (n + 1)));
  PUM_CUDA(cudaMalloc(&dp0ci, sizeof(int) * std::max<size_t>(p0ci.size(), 1)));
  PUM_CUDA(cudaMalloc(&counter, sizeof(int)));
  PUM_CUDA(cudaMalloc(&out_np, sizeof(int) * n));
  PUM_CUDA(cudaMalloc(&out_cols, sizeof(int) * (size_t)n * (a.np_cap + 1)));
  PUM_CUDA(cudaMemcpyAsync(dp0rp, p0rp.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
  if (!p0ci.empty())
    PUM_CUDA(cudaMemcpyAsync(dp0ci, p0ci.data(), sizeof(int) * p0ci.size(), cudaMemcpyHostToDevice, s));
  a.p0rp = dp0rp;
  a.p0ci = dp0ci;
  a.next_row = counter;
  a.out_np = out_np;
  a.out_cols = out_cols;
  a.status = ctx->status;
  std::vector<int> hnp(n), hcols((size_t)n * (a.np_cap + 1));
  DevStatus st{};
  for (int attempt = 0; attempt < 2; ++attempt) {
    a.slots = attempt == 0 ? std::min(bound, 128) : bound;
    const int ctas = std::max(1, std::min(a.n_work, ctx->sm_count * 4));
    double* slab = nullptr;
    PUM_CUDA(cudaMalloc(&slab, sizeof(double) * (size_t)ctas * a.slots * a.slot_doubles));
    a.slab = slab;
    PUM_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), s));
    PUM_CUDA(cudaMemsetAsync(dfma, 0, sizeof(double), s));
    a.fmas = dfma;
    switch (d) {
      case 3: launch_adapt<3>(ctx, a, ctas); break;
      case 6: launch_adapt<6>(ctx, a, ctas); break;
      case 10: launch_adapt<10>(ctx, a, ctas); break;
      case 15: launch_adapt<15>(ctx, a, ctas); break;
      case 20: launch_adapt<20>(ctx, a, ctas); break;
      case 21: launch_adapt<21>(ctx, a, ctas); break;
      default: PUM_CHECK(false, PUM_ERR_UNSUPPORTED, "Algorithm 1: unsupported block size");
    }
    PUM_CUDA(cudaStreamSynchronize(s));
    cudaFree(slab);
    PUM_CUDA(cudaMemcpy(&st, ctx->status, sizeof(st), cudaMemcpyDeviceToHost));
    if (st.code != 0) PUM_CUDA(cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), s));
    if (!(st.code == PUM_ERR_UNSUPPORTED && a.slots < bound)) break;
  }
  double fma = 0.0;
  if (st.code == 0) {
    PUM_CUDA(cudaMemcpy(hnp.data(), out_np, sizeof(int) * n, cudaMemcpyDeviceToHost));
    PUM_CUDA(cudaMemcpy(hcols.data(), out_cols, sizeof(int) * hcols.size(), cudaMemcpyDeviceToHost));
    PUM_CUDA(cudaMemcpy(&fma, dfma, sizeof(double), cudaMemcpyDeviceToHost));
  }
  std::vector<double> hld;
  if (st.code == 0 && G) {
    // the factors on the final pattern: BSR allocation, then the staged blocks row by row
    std::vector<int> rp(n + 1, 0), ci;
    for (int k = 0; k < n; ++k) {
      ci.insert(ci.end(), hcols.begin() + (int64_t)k * (a.np_cap + 1),
                hcols.begin() + (int64_t)k * (a.np_cap + 1) + hnp[k]);
      rp[k + 1] = (int)ci.size();
    }
    bsr_alloc(*G, n, A.n_bcols, d, PUM_F64, rp, ci);
    if (F) bsr_alloc(*F, n, A.n_bcols, d, PUM_F64, rp, ci);
    if (n > 0) {
      k_stage_to_bsr<<<n, 128, 0, s>>>((double*)G->vals, G->stride, dstage_g, a.np_cap + 1, G->row_ptr, d * d);
      count_launch(ctx);
      if (F) {
        k_stage_to_bsr<<<n, 128, 0, s>>>((double*)F->vals, F->stride, dstage_f, a.np_cap + 1, F->row_ptr, d * d);
        count_launch(ctx);
      }
      PUM_CUDA(cudaGetLastError());
    }
    hld.resize(n);
    PUM_CUDA(cudaMemcpy(hld.data(), dld, sizeof(double) * n, cudaMemcpyDeviceToHost));  // waits for the copies
    double sum = 0.0;
    for (double v : hld) sum += v;
    if (logdet) *logdet = sum;
  }
  for (void* p : {(void*)dp0rp, (void*)dp0ci, (void*)counter, (void*)out_np, (void*)out_cols, (void*)dfma,
                  (void*)dwork, (void*)dstage_g, (void*)dstage_f, (void*)dld})
    if (p) cudaFree(p);
  if (fp64_flops) *fp64_flops += 2.0 * fma;
  if (st.code != 0)
    throw Error{(pum_status)st.code,
                st.code == PUM_ERR_NOT_SPD
                    ? "adaptive FSAI: factorisation failed (non-positive pivot, Cholesky of A[P~,P~] or S_kk) at block "
                      "row " + std::to_string(st.info)
                    : "adaptive FSAI: row capacity exceeded at block row " + std::to_string(st.info)};
  rows = P0;  // rows outside the work list keep P0
  auto take = [&](int k) {
    rows[k].assign(hcols.begin() + (int64_t)k * (a.np_cap + 1), hcols.begin() + (int64_t)k * (a.np_cap + 1) + hnp[k]);
  };
  if (work_rows)
    for (int k : *work_rows) take(k);
  else
    for (int k = 0; k < n; ++k) take(k);
  return true;
}

}  // namespace pum
