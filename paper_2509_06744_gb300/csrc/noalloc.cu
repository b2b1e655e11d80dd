// Block-FSAI application z = G^T (G r) that allocates no memory.
//
// Some callers cannot allocate device memory: an application whose device memory is
// already reserved in full by another allocator (a framework's caching pool), a host with
// a fixed memory budget decided at start-up, or a latency-bound loop that cannot take the
// device-wide synchronisation that cudaFree implies.  They still need the intermediate
// vector t = G r.  Here it lives in one file-scope device array, kNoAllocMaxUnknowns
// doubles (8 MiB), that every GPU which loads the library holds until the process exits.
//
// The array's name in host code is only a host-side stand-in, never a device address:
// its device address is looked up once per device with cudaGetSymbolAddress (on the
// first call on that device, with that device current) and passed to the kernels.
// All calls share the array, so calls whose work overlaps on the GPU (different
// streams, or several contexts on one device) race on it; calls queued on one stream
// are ordered and safe.  t is fully overwritten by every call before it is read, so
// nothing needs clearing.
#include <mutex>
#include <string>

#include "pum_internal.cuh"

namespace {

constexpr int64_t kNoAllocMaxUnknowns = int64_t(1) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxUnknowns];

double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// y = M x for a caller BSR with contiguous d x d blocks (block stride d*d), FP64.
template <int D>
__global__ void __launch_bounds__(256) k_bsr_set_f64(int n_brows, const int* __restrict__ rp, const int* __restrict__ ci,
                                                     const double* __restrict__ vals, const double* __restrict__ x,
                                                     double* __restrict__ y) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int row = (int)(tid / D);
  if (row >= n_brows) return;
  const int r = (int)(tid - (int64_t)row * D);
  double acc = 0.0;
  for (int b = rp[row]; b < rp[row + 1]; ++b) {
    const double* a = vals + (int64_t)b * (D * D) + r * D;
    const double* xv = x + (int64_t)ci[b] * D;
#pragma unroll
    for (int q = 0; q < D; ++q) acc = fma(a[q], xv[q], acc);
  }
  y[tid] = acc;
}

template <int D>
void launch_set(const pum_bsr_view& M, const double* x, double* y, cudaStream_t s) {
  const int64_t n = (int64_t)M.n_brows * D;
  if (n == 0) return;
  k_bsr_set_f64<D><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(M.n_brows, M.row_ptr, M.col_idx, M.vals, x, y);
}

bool launch_any(const pum_bsr_view& M, const double* x, double* y, cudaStream_t s) {
  switch (M.bs) {
    case 3: launch_set<3>(M, x, y, s); return true;
    case 6: launch_set<6>(M, x, y, s); return true;
    case 10: launch_set<10>(M, x, y, s); return true;
    case 15: launch_set<15>(M, x, y, s); return true;
    case 21: launch_set<21>(M, x, y, s); return true;
    default: return false;
  }
}

// Device address of the scratch array on `device` (looked up once per device).
cudaError_t scratch_for(int device, double** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" pum_status pum_fsai_apply_noalloc(pum_ctx* ctx, const pum_bsr_view* G, const pum_bsr_view* GT,
                                             const double* r, double* z) {
  if (!ctx || !G || !GT || !r || !z) return PUM_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (!G->on_device || !GT->on_device || !G->row_ptr || !GT->row_ptr || (G->nnzb && (!G->col_idx || !G->vals)) ||
      (GT->nnzb && (!GT->col_idx || !GT->vals))) {
    ctx->last_error = "pum_fsai_apply_noalloc: G and GT must be device BSR arrays";
    return PUM_ERR_INVALID_ARG;
  }
  if (G->bs != GT->bs || G->n_brows != G->n_bcols || GT->n_brows != G->n_bcols || GT->n_bcols != G->n_brows) {
    ctx->last_error = "pum_fsai_apply_noalloc: G must be square and GT its transpose";
    return PUM_ERR_INVALID_ARG;
  }
  if ((int64_t)G->n_brows * G->bs > kNoAllocMaxUnknowns) {
    ctx->last_error = "pum_fsai_apply_noalloc: more than 1048576 unknowns (the static scratch limit)";
    return PUM_ERR_INVALID_ARG;
  }
  // the kernels read float64 scalars: 8-byte alignment is what they need
  if (((uintptr_t)r & 7) || ((uintptr_t)z & 7) || ((uintptr_t)G->vals & 7) || ((uintptr_t)GT->vals & 7)) {
    ctx->last_error = "pum_fsai_apply_noalloc: vectors and values must be 8-byte aligned";
    return PUM_ERR_INVALID_ARG;
  }
  if (G->bs != 3 && G->bs != 6 && G->bs != 10 && G->bs != 15 && G->bs != 21) {
    ctx->last_error = "pum_fsai_apply_noalloc: block size must be 3, 6, 10, 15 or 21";
    return PUM_ERR_UNSUPPORTED;
  }
  if (ctx->device < 0 || ctx->device >= kMaxDevices) {
    ctx->last_error = "pum_fsai_apply_noalloc: device ordinal outside [0, 64)";
    return PUM_ERR_INVALID_ARG;
  }
  // the lookup and the launches run with the context's device current; the caller's
  // current device is put back on every path out
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && prev != ctx->device) e = cudaSetDevice(ctx->device);
  double* t = nullptr;
  if (e == cudaSuccess) e = scratch_for(ctx->device, &t);
  pum_status st = PUM_OK;
  if (e != cudaSuccess) {
    ctx->last_error = std::string("pum_fsai_apply_noalloc: device scratch lookup failed: ") + cudaGetErrorString(e);
    st = PUM_ERR_CUDA;
  } else {
    launch_any(*G, r, t, ctx->stream);
    launch_any(*GT, t, z, ctx->stream);
    ctx->launches += 2;
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      ctx->last_error = std::string("pum_fsai_apply_noalloc: kernel launch failed: ") + cudaGetErrorString(e);
      st = PUM_ERR_CUDA;
    }
  }
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return st;
}
