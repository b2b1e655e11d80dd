// Device helpers shared by the BSR and sliced-block product kernels: accumulation types,
// vectorised row loads and the fused epilogues (residual, Chebyshev-4 updates of Algorithm 3).
#pragma once

#include "pum_internal.cuh"

namespace pum {

// Programmatic dependent launch.  A kernel launched with programmatic stream serialization may
// start while its predecessor in the stream is still running: pdl_wait() blocks until that
// predecessor has completed and its writes are visible (every thread that touches memory the
// predecessor writes, or that later kernels read through this one, passes it first), and
// pdl_release() lets the successor start launching.  Both are no-ops for ordinary launches.
// Before its own wait a kernel touches only constant data (matrix structure and values); no
// kernel that writes a matrix triggers early, so a matrix read before the wait is complete.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Products of block size D <= 10 trigger right after their own wait, so that the successor
// becomes resident early and issues its constant loads while they run (measured on the 256^2
// biharmonic solve, d = 10: 10.15 -> 9.6 ms, most of it on the small levels).  With d = 21 the
// same placement made the triharmonic solves slower (by 3% to 24% across the variants tried),
// so larger blocks trigger after their main loop, as before.
template <int D>
constexpr bool kEarlyTrigger = D <= 10;

template <typename T> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };
template <> struct AccOf<float2> { using type = double; };  // double-float (hi, lo) matrix values

__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ double to_f(double v) { return v; }

// Load the D contiguous values starting at p (alignment known from D and the layout)
// into registers, converting to the accumulation type.
template <int D, typename T, typename AT>
__device__ __forceinline__ void load_row(const T* __restrict__ p, AT (&out)[D]) {
  if constexpr (sizeof(T) == 4 && (D % 2) == 0) {
    const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
    for (int i = 0; i < D / 2; ++i) {
      float2 v = __ldg(q + i);
      out[2 * i] = (AT)v.x;
      out[2 * i + 1] = (AT)v.y;
    }
  } else if constexpr (sizeof(T) == 8 && (D % 2) == 0) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int i = 0; i < D / 2; ++i) {
      double2 v = __ldg(q + i);
      out[2 * i] = (AT)v.x;
      out[2 * i + 1] = (AT)v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i) out[i] = (AT)to_f(p[i]);
  }
}

// (hi, lo) FP32 pair with hi + lo = v to 2^-48 relative: the split shadow the double-float
// products read instead of an FP64 vector.
__device__ __forceinline__ float2 split_df(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

// Epilogue of the product acc = (M x)_tid for output unknown tid.
template <int EPI, typename AT, typename XT, typename YT, typename X2T>
__device__ __forceinline__ void epilogue(const EpiArgs& e, int64_t tid, AT acc) {
  YT* y = (YT*)e.y;
  X2T* x2 = (X2T*)e.xo2;
  if constexpr (EPI == EPI_SET) {
    y[tid] = (YT)acc;
    if (x2) x2[tid] = (X2T)(YT)acc;  // optional copy of y in the second iterate's precision
  } else if constexpr (EPI == EPI_RESID) {
    // b - A x, formed in the accumulation precision (FP64 for an FP64 operator)
    y[tid] = (YT)((AT)((const XT*)e.b)[tid] - acc);
  } else if constexpr (EPI == EPI_ADD) {
    const YT v = (YT)((AT)y[tid] + acc);
    y[tid] = v;
    if constexpr (sizeof(YT) == 8)
      if (e.ys) ((float2*)e.ys)[tid] = split_df((double)v);
  } else if constexpr (EPI == EPI_CHEB_FIRST0) {
    YT* xo = (YT*)e.xo;
    y[tid] = (YT)acc;
    xo[tid] = (YT)((AT)e.dmu * acc);
    if (x2) {
      const X2T v = e.x2_set ? (X2T)(e.dmu * (double)acc) : (X2T)((double)x2[tid] + e.dmu * (double)acc);
      x2[tid] = v;
      if (e.x2s) ((float2*)e.x2s)[tid] = split_df((double)v);
    }
  } else if constexpr (EPI == EPI_CHEB_FIRST) {
    YT* xo = (YT*)e.xo;
    y[tid] = (YT)acc;
    xo[tid] = (YT)((AT)xo[tid] + (AT)e.dmu * acc);
    if (x2) {
      const X2T v = (X2T)((double)x2[tid] + e.dmu * (double)acc);
      x2[tid] = v;
      if (e.x2s) ((float2*)e.x2s)[tid] = split_df((double)v);
    }
  } else if constexpr (EPI == EPI_CHEB) {
    YT* xo = (YT*)e.xo;
    const AT pn = (AT)e.mu2 * (AT)y[tid] + acc;
    y[tid] = (YT)pn;
    xo[tid] = (YT)((AT)xo[tid] + (AT)e.dmu * pn);
    if (x2) {
      const X2T v = (X2T)((double)x2[tid] + e.dmu * (double)pn);
      x2[tid] = v;
      if (e.x2s) ((float2*)e.x2s)[tid] = split_df((double)v);
    }
  }
}

}  // namespace pum
