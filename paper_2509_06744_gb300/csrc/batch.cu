// Batched set-ups and solves over independent hierarchies.
//
// A 32x32-patch instance cannot fill 152 SMs: its kernels are latency-bound and its PCG waits on
// the host once per iteration.  Many such instances run concurrently instead: worker w drives its
// own context (its own stream) from its own host thread and takes the next hierarchy that no
// other worker holds; all items of one hierarchy (several right-hand sides) are solved by the
// same worker, one after another, since a hierarchy's work vectors and captured cycle are not
// shared.  Each item's report and status are its own; the batch returns the first non-OK status
// in item order.
#include <atomic>
#include <thread>
#include <vector>

#include "pum_internal.cuh"

using namespace pum;

namespace {

// Items grouped by hierarchy, groups in order of their first item.
std::vector<std::vector<int>> group_items(pum_hier* const* hs, int n) {
  std::vector<std::vector<int>> groups;
  std::vector<pum_hier*> keys;
  for (int i = 0; i < n; ++i) {
    size_t g = 0;
    while (g < keys.size() && keys[g] != hs[i]) ++g;
    if (g == keys.size()) {
      keys.push_back(hs[i]);
      groups.emplace_back();
    }
    groups[g].push_back(i);
  }
  return groups;
}

template <typename Work>
pum_status run_batch(pum_ctx* const* workers, int n_workers, pum_hier* const* hs, int n, pum_status* status,
                     Work work) {
  if (!workers || n_workers < 1 || !hs || n < 0) return PUM_ERR_INVALID_ARG;
  for (int w = 0; w < n_workers; ++w) {
    if (!workers[w]) return PUM_ERR_INVALID_ARG;
    for (int v = 0; v < w; ++v)  // each worker needs its own context and stream: a stream shared by
      if (workers[v] == workers[w] || workers[v]->stream == workers[w]->stream)  // two threads races
        return PUM_ERR_INVALID_ARG;                                            // (graph captures)
  }
  for (int i = 0; i < n; ++i)
    if (!hs[i]) return PUM_ERR_INVALID_ARG;
  const auto groups = group_items(hs, n);
  std::vector<pum_status> st(n, PUM_OK);
  std::atomic<int> next{0};
  auto worker = [&](int w) {
    for (int g = next.fetch_add(1); g < (int)groups.size(); g = next.fetch_add(1))
      for (int i : groups[g]) st[i] = work(workers[w], i);
  };
  const int nt = std::min<int>(n_workers, (int)groups.size());
  std::vector<std::thread> threads;
  for (int w = 1; w < nt; ++w) threads.emplace_back(worker, w);
  if (nt > 0) worker(0);
  for (auto& t : threads) t.join();
  pum_status first = PUM_OK;
  for (int i = 0; i < n; ++i) {
    if (status) status[i] = st[i];
    if (first == PUM_OK && st[i] != PUM_OK) first = st[i];
  }
  return first;
}

}  // namespace

extern "C" pum_status pum_setup_batch(pum_ctx* const* workers, int n_workers, pum_hier* const* hs, int n,
                                      const bfsai_params* fp, const smoother_params* sp, pum_status* status) {
  if (!fp || !sp) return PUM_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j)
      if (hs && hs[i] == hs[j]) return PUM_ERR_INVALID_ARG;  // one set-up per hierarchy
  return run_batch(workers, n_workers, hs, n, status,
                   [&](pum_ctx* ctx, int i) { return bfsai_setup(ctx, hs[i], fp, sp); });
}

extern "C" pum_status pum_solve_batch(pum_ctx* const* workers, int n_workers, pum_hier* const* hs, int n,
                                      const double* const* b, double* const* x, pcg_report* reps, int method,
                                      pum_status* status) {
  if (!b || !x || !reps || (method != 0 && method != 1)) return PUM_ERR_INVALID_ARG;
  return run_batch(workers, n_workers, hs, n, status, [&](pum_ctx* ctx, int i) {
    return method == 0 ? pcg_solve(ctx, hs[i], b[i], x[i], &reps[i]) : bicgstab_solve(ctx, hs[i], b[i], x[i], &reps[i]);
  });
}

extern "C" pum_status pum_solve_batch_multi(pum_ctx* const* workers, int n_workers, pum_hier* const* hs, int n,
                                            int nrhs, const double* const* B, double* const* X, pcg_report* reps,
                                            pum_status* status) {
  if (!B || !X || !reps || nrhs < 1) return PUM_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j)
      if (hs && hs[i] == hs[j]) return PUM_ERR_INVALID_ARG;  // one multi-solve per hierarchy
  return run_batch(workers, n_workers, hs, n, status, [&](pum_ctx* ctx, int i) {
    return pcg_solve_multi(ctx, hs[i], nrhs, B[i], X[i], reps + (size_t)i * nrhs);
  });
}
