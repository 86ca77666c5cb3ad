// Batched ordering of many meshes (fp_batch_order) and the patch-cap
// autotuner (fp_batch_autotune).
//
// One mesh's pipeline is a chain of latency-bound launches separated by a few
// host read-backs of data-dependent sizes (patch count, tree depth, node
// sizes), so it occupies a small part of the GPU, and a host pool running
// many meshes' pipelines at once is bound by the launch rate of one CUDA
// context (about 143 launches a mesh). The fused form orders the whole batch
// as one graph instead, the disjoint union of its meshes: every stage is one
// pipeline over all meshes (the same launches as one mesh, each covering
// every mesh's vertices, patches and tree nodes), and the union's tree puts
// every mesh's dissection tree below an empty super-tree (Segments). A mesh's
// patches, separators, orders and symbolic counts depend only on its own
// vertices, with its own cap, seed threshold and vertex numbering, so each
// result equals the mesh ordered alone. The pool runs on request
// (n_workers > 0) and orders the items one by one when the fused form fails.
#include <algorithm>
#include <atomic>
#include <chrono>
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

// ---- fused batch: one pipeline over the disjoint union ----------------------------

struct FaceSeg {
  const int32_t* faces;
  int64_t foff;      // first union face
  int32_t voff;      // first union vertex
  int32_t n;         // vertices of the mesh
};

struct OutSeg {
  int32_t* perm;
  int32_t* iperm;
  int32_t* parent;
  int32_t* colcount;
};

// Union faces: every mesh's corners shifted by its first vertex. A corner out
// of its own mesh's range becomes -1, which the CSR build reports as a bad
// index (it would otherwise join two meshes).
__global__ void k_union_faces(const FaceSeg* __restrict__ seg, int32_t M, int64_t F, int32_t* __restrict__ out) {
  FP_PDL_WAIT();
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
    int32_t lo = 0, hi = M - 1;        // the last mesh whose first face is <= f
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (seg[mid].foff <= f) lo = mid; else hi = mid - 1;
    }
    const FaceSeg s = seg[lo];
    const int32_t* src = s.faces + 3 * (f - s.foff);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int32_t x = src[c];
      out[3 * f + c] = (x >= 0 && x < s.n) ? x + s.voff : -1;
    }
  }
}

__global__ void k_vertex_mesh(const int32_t* __restrict__ voff, int32_t M, int32_t n, int32_t* __restrict__ vmesh) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int32_t lo = 0, hi = M - 1;        // the last mesh whose first vertex is <= v
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (voff[mid] <= v) lo = mid; else hi = mid - 1;
    }
    vmesh[v] = lo;
  }
}

// Per-mesh outputs from the union's: position p holds union vertex v of mesh
// m; both are renumbered inside the mesh (its positions start at posoff[m],
// its vertices at voff[m]).
__global__ void k_batch_perm_out(const int32_t* __restrict__ perm, int32_t n, const int32_t* __restrict__ vmesh,
                                 const int32_t* __restrict__ voff, const int32_t* __restrict__ posoff,
                                 const OutSeg* __restrict__ outs) {
  FP_PDL_WAIT();
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int32_t v = perm[p];
    const int32_t m = vmesh[v];
    const int32_t lp = p - posoff[m], lv = v - voff[m];
    const OutSeg o = outs[m];
    if (o.perm) o.perm[lp] = lv;
    if (o.iperm) o.iperm[lv] = lp;
  }
}

// The elimination tree never leaves a mesh (no union edge joins two
// meshes): parents are renumbered like positions. nnz(L) and flops per mesh
// are the sums of colcount and colcount^2 over its positions (a warp's
// positions usually lie in one mesh: one atomic pair a warp).
__global__ void k_batch_sym_out(const int32_t* __restrict__ perm, const int32_t* __restrict__ parent,
                                const int32_t* __restrict__ colcount, int32_t n, const int32_t* __restrict__ vmesh,
                                const int32_t* __restrict__ posoff, const OutSeg* __restrict__ outs,
                                unsigned long long* __restrict__ sums) {
  FP_PDL_WAIT();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t p = base + threadIdx.x;
    const bool live = p < n;
    int32_t m = -1;
    unsigned long long c = 0, c2 = 0;
    if (live) {
      m = vmesh[perm[p]];
      const int32_t lp = (int32_t)p - posoff[m];
      const OutSeg o = outs[m];
      const int32_t cc = colcount[p];
      if (o.parent) {
        const int32_t q = parent[p];
        o.parent[lp] = q < 0 ? -1 : q - posoff[m];
      }
      if (o.colcount) o.colcount[lp] = cc;
      c = (unsigned long long)cc;
      c2 = c * c;
    }
    const int32_t m0 = __shfl_sync(0xffffffffu, m, 0);
    if (__all_sync(0xffffffffu, !live || m == m0)) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_down_sync(0xffffffffu, c, o);
        c2 += __shfl_down_sync(0xffffffffu, c2, o);
      }
      if ((threadIdx.x & 31) == 0 && m0 >= 0) {
        atomicAdd(&sums[2 * m0], c);
        atomicAdd(&sums[2 * m0 + 1], c2);
      }
    } else if (live) {
      atomicAdd(&sums[2 * m], c);
      atomicAdd(&sums[2 * m + 1], c2);
    }
  }
}

// Whether the fused form takes the batch: one DOF per vertex, no explicit
// depth, no stage records, valid items, totals within int32.
bool fused_ok(const fp_batch_item* items, int32_t count, const fp_options& o) {
  if (o.dof_per_vertex != 1 || o.nd_level != 0 || o.debug_dump != 0) return false;
  int64_t N = 0, F = 0;
  for (int32_t i = 0; i < count; ++i) {
    const fp_batch_item& it = items[i];
    if (it.n_vertices < 0 || it.n_faces < 0 || (it.n_faces > 0 && !it.d_faces)) return false;
    N += it.n_vertices;
    F += it.n_faces;
  }
  return N <= INT32_MAX && F <= INT32_MAX / 6;
}

// The union handle: union faces gathered on `s`, the CSR built by the
// single-mesh path, then the per-mesh lookups.
fp_status fused_create(const fp_batch_item* items, int32_t M, const fp_options& base, cudaStream_t s,
                       fp_handle** out) {
  *out = nullptr;
  int device = 0;
  cudaGetDevice(&device);
  std::vector<int32_t> voff(M + 1, 0), caps(M);
  std::vector<FaceSeg> fs(M);
  int64_t F = 0;
  for (int32_t m = 0; m < M; ++m) {
    caps[m] = cap_for(items[m], base);
    fs[m] = {items[m].d_faces, F, voff[m], items[m].n_vertices};
    F += items[m].n_faces;
    voff[m + 1] = voff[m] + items[m].n_vertices;
  }
  const int32_t N = voff[M];
  cudaMemPool_t pool = library_pool(device);
  int32_t* d_faces = nullptr;
  FaceSeg* d_fs = nullptr;
  if (cudaMallocFromPoolAsync((void**)&d_faces, sizeof(int32_t) * 3 * (size_t)(F > 0 ? F : 1), pool, s) != cudaSuccess ||
      cudaMallocFromPoolAsync((void**)&d_fs, sizeof(FaceSeg) * (size_t)M, pool, s) != cudaSuccess) {
    cudaGetLastError();
    if (d_faces) cudaFreeAsync(d_faces, s);
    return fail(nullptr, FP_ERR_OUT_OF_MEMORY, "batch union faces");
  }
  // pageable source: the call returns once the table is staged
  cudaMemcpyAsync(d_fs, fs.data(), sizeof(FaceSeg) * (size_t)M, cudaMemcpyHostToDevice, s);
  if (F > 0) launch_pdl(s, k_union_faces, grid_for(F, 256), 256, 0, (const FaceSeg*)d_fs, M, F, d_faces);
  fp_options o = base;
  o.patch_cap = caps[0];
  fp_handle* h = nullptr;
  fp_status st = fp_create_from_faces(d_faces, F, N, &o, s, &h);
  cudaFreeAsync(d_faces, s);
  cudaFreeAsync(d_fs, s);
  if (st != FP_OK) return st;
  if (F > 0) h->launches++;
  Segments* sg = new Segments();
  h->seg = sg;
  sg->M = M;
  sg->h_voff = voff;
  sg->h_cap = caps;
  int32_t* d_voff = (int32_t*)dev_alloc(h, sizeof(int32_t) * (size_t)(M + 1));
  int32_t* d_cap = (int32_t*)dev_alloc(h, sizeof(int32_t) * (size_t)M);
  int32_t* d_vmesh = (int32_t*)dev_alloc(h, sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
  sg->mroot = (int32_t*)dev_alloc(h, sizeof(int32_t) * (size_t)M);
  sg->d_posoff = (int32_t*)dev_alloc(h, sizeof(int32_t) * (size_t)M);
  sg->d_outs = dev_alloc(h, sizeof(OutSeg) * (size_t)M);
  if (!d_voff || !d_cap || !d_vmesh || !sg->mroot || !sg->d_posoff || !sg->d_outs) {
    fp_destroy(h);
    return fail(nullptr, FP_ERR_OUT_OF_MEMORY, "batch union arrays");
  }
  cudaMemcpyAsync(d_voff, voff.data(), sizeof(int32_t) * (size_t)(M + 1), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d_cap, caps.data(), sizeof(int32_t) * (size_t)M, cudaMemcpyHostToDevice, s);
  if (N > 0) FP_LAUNCH(h, k_vertex_mesh, grid_for(N, 256), 256, 0, (const int32_t*)d_voff, M, N, d_vmesh);
  sg->v = SegView{d_vmesh, d_voff, d_cap};
  fp_status e = check_cuda(h, cudaGetLastError(), "batch union");
  if (e != FP_OK) {
    fp_destroy(h);
    return e;
  }
  *out = h;
  return FP_OK;
}

// Uploads the items' output pointers (host vectors must stay alive until the
// copy is staged: pageable memory, so the call returns after staging).
void upload_outs(fp_handle* h, const fp_batch_item* items) {
  Segments* sg = h->seg;
  std::vector<OutSeg> outs(sg->M);
  for (int32_t m = 0; m < sg->M; ++m) outs[m] = {items[m].d_perm, items[m].d_iperm, items[m].d_parent, items[m].d_colcount};
  cudaMemcpyAsync(sg->d_outs, outs.data(), sizeof(OutSeg) * (size_t)sg->M, cudaMemcpyHostToDevice, h->stream);
}

// wait: return only when the outputs are complete (the public call); the
// fused batch goes straight on to the symbolic stage, whose host planning
// then overlaps the ordering kernels, and waits there.
fp_status fused_permute(fp_handle* h, fp_batch_item* items, bool wait) {
  Segments* sg = h->seg;
  const int32_t M = sg->M, N = h->n;
  FP_TRY(fp_permute(h, nullptr, nullptr));
  upload_outs(h, items);
  cudaMemcpyAsync(sg->d_posoff, sg->h_posoff.data(), sizeof(int32_t) * (size_t)M, cudaMemcpyHostToDevice, h->stream);
  if (N > 0)
    FP_LAUNCH(h, k_batch_perm_out, grid_for(N, 256), 256, 0, (const int32_t*)h->perm, N, sg->v.vmesh, sg->v.voff,
              (const int32_t*)sg->d_posoff, (const OutSeg*)sg->d_outs);
  FP_CHECK_LAUNCH(h, "batch permutation outputs");
  if (wait) {
    int32_t st = 0;
    FP_TRY(sync_status(h, &st));
  }
  for (int32_t m = 0; m < M; ++m) {
    fp_batch_item& it = items[m];
    it.status = FP_OK;
    it.chosen_cap = sg->h_cap[m];
    it.launches = 0;
    it.learned_leaves = it.learned_kept = 0;
    it.fill_plain = it.fill_chosen = 0;
    if (h->qnet && sg->h_learned.size() == 4 * (size_t)M) {
      const unsigned long long* L = &sg->h_learned[4 * (size_t)m];
      it.learned_kept = (int32_t)L[0];
      it.fill_plain = (int64_t)L[1];
      it.fill_chosen = (int64_t)L[2];
      it.learned_leaves = (int32_t)L[3];
    }
  }
  items[0].launches = h->launches;
  return FP_OK;
}

fp_status fused_symbolic(fp_handle* h, fp_batch_item* items) {
  Segments* sg = h->seg;
  const int32_t M = sg->M, N = h->n;
  int32_t* parent = (int32_t*)dev_alloc(h, sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
  int32_t* colcount = (int32_t*)dev_alloc(h, sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
  unsigned long long* d_sums = (unsigned long long*)dev_alloc(h, sizeof(unsigned long long) * 2 * (size_t)M);
  if (!parent || !colcount || !d_sums) return fail(h, FP_ERR_OUT_OF_MEMORY, "batch symbolic outputs");
  int64_t nnz = 0, fl = 0;
  FP_TRY(fp_symbolic(h, parent, colcount, &nnz, &fl));
  upload_outs(h, items);
  cudaMemsetAsync(d_sums, 0, sizeof(unsigned long long) * 2 * (size_t)M, h->stream);
  if (N > 0)
    FP_LAUNCH(h, k_batch_sym_out, grid_for(N, 256), 256, 0, (const int32_t*)h->perm, (const int32_t*)parent,
              (const int32_t*)colcount, N, sg->v.vmesh, (const int32_t*)sg->d_posoff, (const OutSeg*)sg->d_outs,
              d_sums);
  std::vector<unsigned long long> sums(2 * (size_t)M, 0ull);
  cudaMemcpyAsync(sums.data(), d_sums, sizeof(unsigned long long) * 2 * (size_t)M, cudaMemcpyDeviceToHost, h->stream);
  int32_t st = 0;
  FP_TRY(sync_status(h, &st));
  for (void* p : {(void*)parent, (void*)colcount, (void*)d_sums}) dev_free(h, p);
  for (int32_t m = 0; m < M; ++m) {
    items[m].nnzL = (int64_t)sums[2 * m];
    items[m].flops = (int64_t)sums[2 * m + 1];
  }
  items[0].launches = h->launches;
  return FP_OK;
}

fp_status run_fused(fp_batch_item* items, int32_t M, const fp_options& base, cudaStream_t s, const int32_t* codes) {
  fp_handle* h = nullptr;
  FP_TRY(fused_create(items, M, base, s, &h));
  fp_status st = codes ? fp_set_priority_net(h, codes) : FP_OK;
  if (st == FP_OK) st = fused_permute(h, items, false);
  if (st == FP_OK) st = fused_symbolic(h, items);
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
  if (n_workers == 0 && fused_ok(items, count, *opts)) {
    cudaStream_t s = worker_stream(device);
    if (!s) return fail(nullptr, FP_ERR_CUDA, "batch stream");
    if (run_fused(items, count, *opts, s, h_codes) == FP_OK) return FP_OK;
    // a failure: every item's own status comes from ordering it alone
  }
  std::vector<int32_t> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return items[a].n_vertices > items[b].n_vertices; });
  // the fused form's fallback runs 8 workers (8-16 measured best for the
  // pool on a 256-mesh mix: more contend in the driver's launch path)
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

namespace fp {
namespace {

// The fused batch's time (best of two, host clock: the call is synchronous)
// and total nnz(L) with the items of class c at cap caps[c] (items with their
// own cap keep it); outputs are not written.
fp_status fused_trial(const fp_batch_item* items, int32_t count, const fp_options& o, cudaStream_t s,
                      const int32_t* caps, double* ms, int64_t* nnz) {
  std::vector<fp_batch_item> tr(items, items + count);
  for (auto& it : tr) {
    if (it.patch_cap <= 0) it.patch_cap = caps[size_class(it.n_vertices)];
    it.d_perm = it.d_iperm = it.d_parent = it.d_colcount = nullptr;
  }
  *ms = 1e30;
  for (int r = 0; r < 2; ++r) {
    const auto t0 = std::chrono::steady_clock::now();
    FP_TRY(run_fused(tr.data(), count, o, s, nullptr));
    const double t = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *ms = std::min(*ms, t);
  }
  *nnz = 0;
  for (const auto& it : tr) *nnz += it.nnzL;
  return FP_OK;
}

// Tuning for the fused form, on the batch itself: a batch's time is the
// union's, not a sum of single-mesh pipelines, so the caps are timed where
// they run. First one cap for every class, the fastest whose total nnz(L) is
// within 5% of the least seen; then each class in turn tries the other caps
// with the rest fixed, kept when faster at that fill.
fp_status autotune_fused(const fp_batch_item* items, int32_t count, const fp_options& o, cudaStream_t s,
                         int32_t* chosen) {
  bool present[N_CLASSES] = {false, false, false, false, false};
  for (int32_t i = 0; i < count; ++i) present[size_class(items[i].n_vertices)] = true;
  double t[N_CAND];
  int64_t z[N_CAND];
  int32_t caps[N_CLASSES];
  for (int k = 0; k < N_CAND; ++k) {
    std::fill(caps, caps + N_CLASSES, CAND_CAPS[k]);
    FP_TRY(fused_trial(items, count, o, s, caps, &t[k], &z[k]));
  }
  int64_t minnz = *std::min_element(z, z + N_CAND);
  int pick = -1;
  for (int k = 0; k < N_CAND; ++k)
    if ((double)z[k] <= 1.05 * (double)minnz && (pick < 0 || t[k] < t[pick])) pick = k;
  std::fill(caps, caps + N_CLASSES, CAND_CAPS[pick]);
  double best = t[pick];
  for (int c = 0; c < N_CLASSES; ++c) {
    if (!present[c]) continue;
    for (int k = 0; k < N_CAND; ++k) {
      if (CAND_CAPS[k] == caps[c]) continue;
      int32_t trial[N_CLASSES];
      std::copy(caps, caps + N_CLASSES, trial);
      trial[c] = CAND_CAPS[k];
      double tk;
      int64_t zk;
      FP_TRY(fused_trial(items, count, o, s, trial, &tk, &zk));
      minnz = std::min(minnz, zk);
      if ((double)zk <= 1.05 * (double)minnz && tk < best) {
        best = tk;
        caps[c] = trial[c];
      }
    }
  }
  for (int c = 0; c < N_CLASSES; ++c) chosen[c] = present[c] ? caps[c] : 0;
  return FP_OK;
}

}  // namespace
}  // namespace fp

extern "C" fp_status fp_batch_autotune(fp_batch_item* items, int32_t count, const fp_options* opts, int32_t* h_caps) {
  if (count < 0 || (count > 0 && !items) || !opts) return fail(nullptr, FP_ERR_INVALID_ARG, "bad autotune arguments");
  int device = 0;
  cudaGetDevice(&device);
  cudaStream_t s = worker_stream(device);
  if (!s) return fail(nullptr, FP_ERR_CUDA, "autotune stream");
  if (count > 0 && fused_ok(items, count, *opts)) {
    int32_t chosen[N_CLASSES];
    FP_TRY(autotune_fused(items, count, *opts, s, chosen));
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      for (int c = 0; c < N_CLASSES; ++c)
        if (chosen[c] > 0) g_tuned_caps[c] = chosen[c];
    }
    if (h_caps)
      for (int c = 0; c < N_CLASSES; ++c) h_caps[c] = chosen[c];
    return FP_OK;
  }
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

extern "C" fp_status fp_batch_create(const fp_batch_item* items, int32_t count, const fp_options* opts, void* stream,
                                     fp_handle** out) {
  if (!out) return fail(nullptr, FP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || !items || !opts) return fail(nullptr, FP_ERR_INVALID_ARG, "bad batch arguments");
  if (!fused_ok(items, count, *opts))
    return fail(nullptr, FP_ERR_INVALID_ARG,
                "a batch handle takes dof_per_vertex 1, nd_level 0, debug_dump 0 and valid items within int32 totals");
  return fused_create(items, count, *opts, (cudaStream_t)stream, out);
}

extern "C" fp_status fp_batch_permute(fp_handle* h, fp_batch_item* items, int32_t count) {
  if (!h) return fail(nullptr, FP_ERR_INVALID_ARG, "NULL handle");
  if (!h->seg || !items || count != h->seg->M) return fail(h, FP_ERR_INVALID_ARG, "not a batch handle of this many items");
  if (h->poisoned) return fail(h, FP_ERR_STATE, "handle poisoned by an earlier failure");
  return fused_permute(h, items, true);
}

extern "C" fp_status fp_batch_symbolic(fp_handle* h, fp_batch_item* items, int32_t count) {
  if (!h) return fail(nullptr, FP_ERR_INVALID_ARG, "NULL handle");
  if (!h->seg || !items || count != h->seg->M) return fail(h, FP_ERR_INVALID_ARG, "not a batch handle of this many items");
  if (h->poisoned) return fail(h, FP_ERR_STATE, "handle poisoned by an earlier failure");
  if (!h->permuted) return fail(h, FP_ERR_STATE, "fp_batch_permute first");
  return fused_symbolic(h, items);
}
