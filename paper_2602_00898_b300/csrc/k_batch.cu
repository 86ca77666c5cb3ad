// Batched ordering of many meshes (fp_batch_order) and the patch-cap
// autotuner (fp_batch_autotune).
//
// One mesh's pipeline is a chain of latency-bound launches separated by a few
// host read-backs of data-dependent sizes (patch count, tree depth, node
// sizes), so it occupies a small part of the GPU. Independent meshes are
// therefore run concurrently: a pool of host workers, each with its own CUDA
// stream on the caller's device, drains a shared queue of meshes (largest
// first, so that the longest pipelines start early), and the GPU interleaves
// the kernels of all streams.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "fp_internal.cuh"

namespace fp {
namespace {

constexpr int N_CLASSES = 5;
constexpr int N_CAND = 4;
constexpr int32_t CAND_CAPS[N_CAND] = {128, 256, 384, 512};

std::mutex g_tune_mu;
int32_t g_tuned_caps[N_CLASSES] = {0, 0, 0, 0, 0};

int size_class(int32_t n) {
  return n < 8192 ? 0 : (n < 32768 ? 1 : (n < 131072 ? 2 : (n < 524288 ? 3 : 4)));
}

cudaStream_t worker_stream(int device) {
  thread_local cudaStream_t cache[128] = {};
  if (device < 0 || device >= 128) return nullptr;
  if (!cache[device] && cudaStreamCreateWithFlags(&cache[device], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    cache[device] = nullptr;
  }
  return cache[device];
}

int32_t cap_for(const fp_batch_item& it, const fp_options& base) {
  if (it.patch_cap > 0) return it.patch_cap;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const int32_t c = g_tuned_caps[size_class(it.n_vertices)];
  return c > 0 ? c : base.patch_cap;
}

fp_status run_one(const fp_batch_item& it, fp_options o, cudaStream_t s, int32_t* d_perm, int32_t* d_iperm,
                  int32_t* d_parent, int32_t* d_colcount, int64_t* nnz, int64_t* fl, int64_t* launches,
                  const int32_t* codes = nullptr, fp_batch_item* stats = nullptr) {
  fp_handle* h = nullptr;
  fp_status st = fp_create_from_faces(it.d_faces, it.n_faces, it.n_vertices, &o, s, &h);
  if (st == FP_OK && codes) st = fp_set_priority_net(h, codes);
  if (st == FP_OK) st = fp_permute(h, d_perm, d_iperm);
  if (st == FP_OK) st = fp_symbolic(h, d_parent, d_colcount, nnz, fl);
  if (st == FP_OK && stats)
    fp_learned_stats(h, &stats->learned_leaves, &stats->learned_kept, &stats->fill_plain, &stats->fill_chosen);
  if (launches) *launches = fp_launch_count(h);
  fp_destroy(h);
  return st;
}

}  // namespace
}  // namespace fp

using namespace fp;

extern "C" fp_status fp_batch_order(fp_batch_item* items, int32_t count, const fp_options* opts, int32_t n_workers) {
  return fp_batch_order_learned(items, count, opts, n_workers, nullptr);
}

extern "C" fp_status fp_batch_order_learned(fp_batch_item* items, int32_t count, const fp_options* opts,
                                            int32_t n_workers, const int32_t* h_codes) {
  if (count < 0 || (count > 0 && !items) || !opts || n_workers < 0 || n_workers > 64)
    return fail(nullptr, FP_ERR_INVALID_ARG, "bad batch arguments");
  if (count == 0) return FP_OK;
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return fail(nullptr, FP_ERR_CUDA, cudaGetErrorString(e));
  std::vector<int32_t> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return items[a].n_vertices > items[b].n_vertices; });
  // 8 workers measured best for a 256-mesh mix on B300 (more contend in the
  // driver's launch path and for the cooperative grids)
  const int T = std::min<int>(n_workers > 0 ? n_workers : 8, count);
  std::atomic<int32_t> next(0);
  const fp_options base = *opts;
  auto worker = [&]() {
    cudaSetDevice(device);
    cudaStream_t s = worker_stream(device);
    for (;;) {
      const int32_t q = next.fetch_add(1);
      if (q >= count) break;
      fp_batch_item& it = items[order[q]];
      if (!s) { it.status = FP_ERR_CUDA; continue; }
      fp_options o = base;
      o.patch_cap = cap_for(it, base);
      it.chosen_cap = o.patch_cap;
      it.nnzL = it.flops = 0;
      it.launches = 0;
      it.learned_leaves = it.learned_kept = 0;
      it.fill_plain = it.fill_chosen = 0;
      it.status = run_one(it, o, s, it.d_perm, it.d_iperm, it.d_parent, it.d_colcount, &it.nnzL, &it.flops,
                          &it.launches, h_codes, &it);
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < T; ++t) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
  for (int32_t i = 0; i < count; ++i)
    if (items[i].status != FP_OK) return (fp_status)items[i].status;
  return FP_OK;
}

extern "C" fp_status fp_batch_autotune(fp_batch_item* items, int32_t count, const fp_options* opts, int32_t* h_caps) {
  if (count < 0 || (count > 0 && !items) || !opts) return fail(nullptr, FP_ERR_INVALID_ARG, "bad autotune arguments");
  int device = 0;
  cudaGetDevice(&device);
  cudaStream_t s = worker_stream(device);
  if (!s) return fail(nullptr, FP_ERR_CUDA, "autotune stream");
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
    return fail(nullptr, FP_ERR_CUDA, "autotune events");
  int32_t chosen[N_CLASSES] = {0, 0, 0, 0, 0};
  fp_status result = FP_OK;
  for (int c = 0; c < N_CLASSES && result == FP_OK; ++c) {
    int32_t rep = -1;
    for (int32_t i = 0; i < count; ++i)
      if (size_class(items[i].n_vertices) == c && (rep < 0 || items[i].n_vertices > items[rep].n_vertices)) rep = i;
    if (rep < 0) continue;
    float best_ms[N_CAND];
    int64_t nnz[N_CAND];
    for (int k = 0; k < N_CAND && result == FP_OK; ++k) {
      fp_options o = *opts;
      o.patch_cap = CAND_CAPS[k];
      best_ms[k] = 1e30f;
      for (int r = 0; r < 2; ++r) {
        int64_t fl = 0;
        cudaEventRecord(a, s);
        const fp_status st = run_one(items[rep], o, s, nullptr, nullptr, nullptr, nullptr, &nnz[k], &fl, nullptr);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        if (st != FP_OK) { result = st; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        best_ms[k] = std::min(best_ms[k], ms);
      }
    }
    if (result != FP_OK) break;
    int64_t minnz = nnz[0];
    for (int k = 1; k < N_CAND; ++k) minnz = std::min(minnz, nnz[k]);
    int pick = -1;
    for (int k = 0; k < N_CAND; ++k)
      if ((double)nnz[k] <= 1.05 * (double)minnz && (pick < 0 || best_ms[k] < best_ms[pick])) pick = k;
    chosen[c] = CAND_CAPS[pick];
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (result != FP_OK) return result;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (int c = 0; c < N_CLASSES; ++c)
      if (chosen[c] > 0) g_tuned_caps[c] = chosen[c];
  }
  if (h_caps)
    for (int c = 0; c < N_CLASSES; ++c) h_caps[c] = chosen[c];
  return FP_OK;
}
