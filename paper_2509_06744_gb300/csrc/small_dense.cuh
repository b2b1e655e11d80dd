// Small dense FP64 kernels-within-kernels shared by the set-up kernels: block lookup in a BSR
// row, and the Cholesky factorisation and triangular solve of one d x d block by one warp.
#pragma once

#include "pum_internal.cuh"

namespace pum {

__device__ inline int find_blk(const int* rp, const int* ci, int row, int col) {
  int lo = rp[row], hi = rp[row + 1] - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int c = ci[mid];
    if (c == col) return mid;
    if (c < col) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// Cholesky of the symmetric D x D matrix src (row-major) into dst (lower part; the strict upper
// part is left as is) by one warp; inv[j] = 1 / L_jj.  Returns false when a pivot is not
// positive.  det = mant * 2^expo (kept apart so no product of pivots over- or underflows).
template <int D>
__device__ bool warp_chol(const double* src, double* dst, double* inv, double& mant, int& expo) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < D * D; e += 32) dst[e] = src[e];
  __syncwarp();
  mant = 1.0;
  expo = 0;
  bool ok = true;
  for (int j = 0; j < D; ++j) {
    const double piv = dst[j * D + j];
    if (!(piv > 0.0)) {
      ok = false;
      break;
    }
    const double l = sqrt(piv);
    const double il = 1.0 / l;
    int ex = 0;
    mant = frexp(mant * piv, &ex);
    expo += ex;
    __syncwarp();
    if (lane == 0) {
      dst[j * D + j] = l;
      inv[j] = il;
    }
    for (int i = j + 1 + lane; i < D; i += 32) dst[i * D + j] *= il;
    __syncwarp();
    // trailing update of the lower part: (i, c), j < c <= i
    constexpr int kTri = D * (D + 1) / 2;
    for (int t = lane; t < kTri; t += 32) {
      int i = 0;
      while ((i + 1) * (i + 2) / 2 <= t) ++i;
      const int c = t - i * (i + 1) / 2;
      if (c > j) dst[i * D + c] -= dst[i * D + j] * dst[c * D + j];
    }
    __syncwarp();
  }
  __syncwarp();
  return ok;
}

// X (D x D, in place) <- L^{-1} X for the lower factor L with reciprocal diagonal inv; lanes own
// columns.
template <int D>
__device__ void warp_lsolve(const double* L, const double* inv, double* X) {
  const int lane = threadIdx.x & 31;
  if (lane < D) {
    double x[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double v = X[a * D + lane];
#pragma unroll
      for (int t = 0; t < a; ++t) v -= L[a * D + t] * x[t];
      x[a] = v * inv[a];
    }
#pragma unroll
    for (int a = 0; a < D; ++a) X[a * D + lane] = x[a];
  }
  __syncwarp();
}

// X (D x D, in place) <- L^-T X for the lower factor L with reciprocal diagonal inv (back
// substitution with L^T); lanes own columns.
template <int D>
__device__ void warp_ltsolve(const double* L, const double* inv, double* X) {
  const int lane = threadIdx.x & 31;
  if (lane < D) {
    double x[D];
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
      double v = X[a * D + lane];
#pragma unroll
      for (int t = a + 1; t < D; ++t) v -= L[t * D + a] * x[t];
      x[a] = v * inv[a];
    }
#pragma unroll
    for (int a = 0; a < D; ++a) X[a * D + lane] = x[a];
  }
  __syncwarp();
}

}  // namespace pum
