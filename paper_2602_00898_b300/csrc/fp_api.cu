// C ABI entry points (include/fastperm.h): argument checks, handle and
// workspace management, and the order of the stages of Algorithm 1 on the
// caller's stream. Device memory comes from a library-private stream-ordered
// pool that keeps its reservation, so re-creating handles of similar size
// costs no driver allocation after the first one.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include <set>

#include "fp_internal.cuh"

namespace fp {

namespace {
std::mutex g_mu;
cudaMemPool_t g_pools[128];
bool g_pool_ok[128];
thread_local std::string g_create_err = "no error";

// stage profiling state
std::mutex g_prof_mu;
bool g_prof_on = false;
struct ProfRec { int kind; cudaEvent_t a, b; };
std::vector<ProfRec> g_prof_pending;
std::vector<cudaEvent_t> g_prof_free;
double g_prof_ms[FP_PROF_COUNT];
int64_t g_prof_n[FP_PROF_COUNT];

void prof_drain_locked() {
  for (auto& r : g_prof_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess &&
        r.kind >= 0 && r.kind < FP_PROF_COUNT) {
      g_prof_ms[r.kind] += ms;
      g_prof_n[r.kind] += 1;
    }
    cudaGetLastError();
    g_prof_free.push_back(r.a);
    g_prof_free.push_back(r.b);
  }
  g_prof_pending.clear();
}
}  // namespace

bool profiling_on() { return g_prof_on; }

cudaEvent_t prof_event() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_free.empty()) {
    cudaEvent_t e = g_prof_free.back();
    g_prof_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void prof_record(int kind, cudaEvent_t a, cudaEvent_t b) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_pending.push_back({kind, a, b});
  if (g_prof_pending.size() > 4096) prof_drain_locked();
}

cudaMemPool_t library_pool(int device) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (device < 0 || device >= 128) return nullptr;
  if (!g_pool_ok[device]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&g_pools[device], &props) != cudaSuccess) return nullptr;
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(g_pools[device], cudaMemPoolAttrReleaseThreshold, &thr);
    g_pool_ok[device] = true;
  }
  return g_pools[device];
}

void* dev_alloc(fp_handle* h, size_t bytes) {
  void* p = nullptr;
  cudaMemPool_t pool = library_pool(h->device);
  if (!pool) return nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  if (cudaMallocFromPoolAsync(&p, bytes, pool, h->stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  h->allocs.push_back(p);
  return p;
}

void dev_free(fp_handle* h, void* p) {
  if (!p) return;
  auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
  if (it == h->allocs.end()) return;
  h->allocs.erase(it);
  cudaFreeAsync(p, h->stream);
}

fp_status fail(fp_handle* h, fp_status s, const std::string& msg) {
  if (h) h->err = msg; else g_create_err = msg;
  if (h && (s == FP_ERR_CUDA || s == FP_ERR_TIMEOUT)) h->poisoned = true;
  return s;
}

fp_status check_cuda(fp_handle* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FP_OK;
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(h, FP_ERR_OUT_OF_MEMORY, m);
  return fail(h, FP_ERR_CUDA, m);
}

// Page-locked status words of the handles, carved from slabs that are
// allocated once and never returned: page-locking (and unlocking) memory per
// handle costs tens of microseconds and synchronises the device.
struct StatusWords {
  std::mutex mu;
  std::vector<int32_t*> free_words;
};
StatusWords& status_words() {
  static StatusWords sw;
  return sw;
}
int32_t* status_word_take() {
  StatusWords& sw = status_words();
  std::lock_guard<std::mutex> lk(sw.mu);
  if (sw.free_words.empty()) {
    constexpr int SLAB = 1024;
    int32_t* slab = nullptr;
    if (cudaMallocHost(&slab, SLAB * sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (int i = SLAB - 1; i >= 0; --i) sw.free_words.push_back(slab + i);
  }
  int32_t* w = sw.free_words.back();
  sw.free_words.pop_back();
  return w;
}
void status_word_give(int32_t* w) {
  StatusWords& sw = status_words();
  std::lock_guard<std::mutex> lk(sw.mu);
  sw.free_words.push_back(w);
}

int32_t* pinned_scratch() {
  thread_local int32_t* buf = nullptr;
  if (!buf && cudaMallocHost(&buf, 256 * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    buf = nullptr;
  }
  return buf;
}

int32_t* pinned_ints(int64_t count) {
  thread_local int32_t* buf = nullptr;
  thread_local int64_t cap = 0;
  if (count > cap) {
    if (buf) cudaFreeHost(buf);
    int64_t want = count > 2 * cap ? count : 2 * cap;
    if (want < 1024) want = 1024;
    buf = nullptr;
    cap = 0;
    if (cudaMallocHost(&buf, sizeof(int32_t) * want) != cudaSuccess) {
      cudaGetLastError();
      buf = nullptr;
      return nullptr;
    }
    cap = want;
  }
  return buf;
}

cudaEvent_t mark_event(int device) {
  thread_local cudaEvent_t ev[128] = {};
  if (device < 0 || device >= 128) return nullptr;
  if (!ev[device] && cudaEventCreateWithFlags(&ev[device], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    ev[device] = nullptr;
  }
  return ev[device];
}

AuxStream* aux_stream(int device, int which) {
  thread_local AuxStream cache[128][2];
  if (device < 0 || device >= 128 || which < 0 || which > 1) return nullptr;
  AuxStream& a = cache[device][which];
  if (!a.s) {
    if (cudaStreamCreateWithFlags(&a.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&a.join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      a.s = nullptr;
      return nullptr;
    }
  }
  return &a;
}

void allow_max_dynamic_smem_fn(const void* kernel) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({kernel, dev})) return;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  // these kernels live on shared memory: the largest carveout lets as many
  // CTAs be resident as their shared memory allows
  cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  done.insert({kernel, dev});
}

fp_status sync_status(fp_handle* h, int32_t* status_out) {
  cudaError_t e = cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "stream");
  *status_out = *h->h_status;
  return FP_OK;
}

int32_t* stage_buffer(fp_handle* h, int32_t stage, int32_t index, int64_t len) {
  if (!h->opt.debug_dump) return nullptr;
  int32_t* d = (int32_t*)dev_alloc(h, sizeof(int32_t) * (size_t)(len > 0 ? len : 1));
  if (!d) return nullptr;
  h->dumps.push_back({stage, index, d, len});
  return d;
}

void stage_dump(fp_handle* h, int32_t stage, int32_t index, const int32_t* src, int64_t len) {
  int32_t* d = stage_buffer(h, stage, index, len);
  if (d && len > 0) cudaMemcpyAsync(d, src, sizeof(int32_t) * (size_t)len, cudaMemcpyDeviceToDevice, h->stream);
}

void stage_clear(fp_handle* h) {
  for (auto& e : h->dumps) dev_free(h, e.d);
  h->dumps.clear();
}

}  // namespace fp

using namespace fp;

namespace {

fp_status validate_options(const fp_options* o) {
  if (!o) return FP_ERR_INVALID_ARG;
  if (o->patch_cap < 1 || o->lloyd_rounds < 0 || o->lloyd_rounds > 64 || o->nd_level < 0 || o->nd_level > 24 ||
      (o->schedule != 0 && o->schedule != 1) || o->dof_per_vertex < 1 || (o->debug_dump != 0 && o->debug_dump != 1) ||
      o->max_spin < 0)
    return FP_ERR_INVALID_ARG;
  return FP_OK;
}

fp_status new_handle(const fp_options* opts, void* stream, int32_t n, fp_handle** out) {
  fp_handle* h = new fp_handle();
  cudaGetDevice(&h->device);
  h->stream = (cudaStream_t)stream;
  h->opt = *opts;
  h->n = n;
  h->b = opts->dof_per_vertex;
  h->h_status = status_word_take();
  if (!h->h_status) {
    delete h;
    return fail(nullptr, FP_ERR_OUT_OF_MEMORY, "pinned status word");
  }
  h->d_status = (int32_t*)dev_alloc(h, sizeof(int32_t));
  if (!h->d_status) {
    status_word_give(h->h_status);
    delete h;
    return fail(nullptr, FP_ERR_OUT_OF_MEMORY, "status word");
  }
  fill_i32(h, h->d_status, 0, 1);
  *out = h;
  return FP_OK;
}

fp_status finish_create(fp_handle* h, fp_status s, fp_handle** out) {
  if (s == FP_OK) {
    const int64_t n = h->n > 0 ? h->n : 1;
    h->gmap = (int32_t*)dev_alloc(h, sizeof(int32_t) * n);
    h->node_of = (int32_t*)dev_alloc(h, sizeof(int32_t) * n);
    h->perm = (int32_t*)dev_alloc(h, sizeof(int32_t) * n);
    h->iperm = (int32_t*)dev_alloc(h, sizeof(int32_t) * n);
    if (!h->gmap || !h->node_of || !h->perm || !h->iperm) s = fail(h, FP_ERR_OUT_OF_MEMORY, "handle arrays");
  }
  if (s != FP_OK) {
    g_create_err = h->err;
    fp_destroy(h);
    *out = nullptr;
    return s;
  }
  *out = h;
  return FP_OK;
}

}  // namespace

extern "C" {

void fp_default_options(fp_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->patch_cap = 512;
  o->lloyd_rounds = 2;
  o->seed = 0;
  o->nd_level = 0;
  o->schedule = 0;
  o->dof_per_vertex = 1;
  o->debug_dump = 0;
  o->max_spin = 0;
}

fp_status fp_create_from_faces(const int32_t* d_faces, int64_t n_faces, int32_t n_vertices, const fp_options* opts,
                               void* stream, fp_handle** out) {
  if (!out) return fail(nullptr, FP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (validate_options(opts) != FP_OK) return fail(nullptr, FP_ERR_INVALID_ARG, "bad options");
  if (n_vertices < 0 || n_faces < 0 || (n_faces > 0 && !d_faces))
    return fail(nullptr, FP_ERR_INVALID_ARG, "bad sizes or NULL faces");
  if ((int64_t)n_vertices * opts->dof_per_vertex > INT32_MAX)
    return fail(nullptr, FP_ERR_UNSUPPORTED, "n * dof_per_vertex exceeds int32");
  if (n_faces > INT32_MAX / 6) return fail(nullptr, FP_ERR_UNSUPPORTED, "too many faces");
  fp_handle* h = nullptr;
  FP_TRY(new_handle(opts, stream, n_vertices, &h));
  fp_status s = build_graph_from_faces(h, d_faces, n_faces);
  return finish_create(h, s, out);
}

fp_status fp_create_from_csr(const int32_t* d_rowptr, const int32_t* d_col, int32_t n_rows, const fp_options* opts,
                             void* stream, fp_handle** out) {
  if (!out) return fail(nullptr, FP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (validate_options(opts) != FP_OK) return fail(nullptr, FP_ERR_INVALID_ARG, "bad options");
  if (n_rows < 0 || !d_rowptr || n_rows % opts->dof_per_vertex != 0)
    return fail(nullptr, FP_ERR_INVALID_ARG, "bad n_rows or NULL rowptr");
  fp_handle* h = nullptr;
  FP_TRY(new_handle(opts, stream, n_rows / opts->dof_per_vertex, &h));
  fp_status s = build_graph_from_csr(h, d_rowptr, d_col, n_rows);
  return finish_create(h, s, out);
}

fp_status fp_permute(fp_handle* h, int32_t* d_perm, int32_t* d_iperm) {
  if (!h) return fail(nullptr, FP_ERR_INVALID_ARG, "NULL handle");
  if (h->poisoned) return fail(h, FP_ERR_STATE, "handle poisoned by an earlier failure");
  h->permuted = false;
  stage_clear(h);
  numeric_release(h);
  if (h->user_k > 0) {
    // patches supplied by the caller (fp_set_patches)
    h->k = h->user_k;
    if (h->n > 0) cudaMemcpyAsync(h->gmap, h->user_gmap, sizeof(int32_t) * h->n, cudaMemcpyDeviceToDevice, h->stream);
  } else {
    FP_TRY(run_patching(h));
  }
  FP_TRY(run_nested_dissection(h));
  h->nnodes = ((int64_t)1 << (h->D + 1)) - 1;
  if (h->nnodes > h->node_cap) {
    dev_free(h, h->node_begin);
    dev_free(h, h->node_size);
    h->node_begin = (int32_t*)dev_alloc(h, sizeof(int32_t) * h->nnodes);
    h->node_size = (int32_t*)dev_alloc(h, sizeof(int32_t) * h->nnodes);
    if (!h->node_begin || !h->node_size) return fail(h, FP_ERR_OUT_OF_MEMORY, "tree arrays");
    h->node_cap = h->nnodes;
  }
  FP_TRY(run_local_order(h));
  FP_TRY(run_learned(h));
  const int64_t N = (int64_t)h->n * h->b;
  if (N > 0) {
    if (h->b == 1) {
      if (d_perm) cudaMemcpyAsync(d_perm, h->perm, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, h->stream);
      if (d_iperm) cudaMemcpyAsync(d_iperm, h->iperm, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, h->stream);
    } else {
      launch_dof_expand_perm(h, h->perm, d_perm, d_iperm);
    }
  }
  FP_CHECK_LAUNCH(h, "permute outputs");
  h->permuted = true;
  return FP_OK;
}

namespace {
// Code ranges of the priority network (see the header).
bool codes_valid(const int32_t* c) {
  const int ranges[8][3] = {{P_W1S, P_W1N, 255}, {P_W1N, P_B1, 255}, {P_B1, P_W2S, 1 << 20}, {P_W2S, P_W2N, 255},
                            {P_W2N, P_B2, 255}, {P_B2, P_W3, 1 << 20}, {P_W3, P_C, 255}, {P_C, P_COUNT, 1 << 20}};
  for (auto& r : ranges)
    for (int i = r[0]; i < r[1]; ++i)
      if (c[i] < -r[2] || c[i] > r[2]) return false;
  return true;
}
}  // namespace

fp_status fp_set_priority_net(fp_handle* h, const int32_t* h_codes) {
  if (!h) return fail(nullptr, FP_ERR_INVALID_ARG, "NULL handle");
  if (h->poisoned) return fail(h, FP_ERR_STATE, "handle poisoned by an earlier failure");
  if (!h_codes) {
    dev_free(h, h->qnet);
    h->qnet = nullptr;
    return FP_OK;
  }
  if (!codes_valid(h_codes)) return fail(h, FP_ERR_INVALID_ARG, "network code out of range");
  if (!h->qnet) h->qnet = (int32_t*)dev_alloc(h, sizeof(int32_t) * FP_GNN_NPARAMS);
  if (!h->qnet) return fail(h, FP_ERR_OUT_OF_MEMORY, "network codes");
  cudaError_t e = cudaMemcpyAsync(h->qnet, h_codes, sizeof(int32_t) * FP_GNN_NPARAMS, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return check_cuda(h, e, "network codes");
}

fp_status fp_learned_stats(const fp_handle* h, int32_t* h_leaves, int32_t* h_kept, int64_t* h_fill_plain,
                           int64_t* h_fill_chosen) {
  if (!h) return fail(nullptr, FP_ERR_INVALID_ARG, "NULL handle");
  if (h_leaves) *h_leaves = h->learned_leaves;
  if (h_kept) *h_kept = h->learned_kept;
  if (h_fill_plain) *h_fill_plain = h->fill_plain;
  if (h_fill_chosen) *h_fill_chosen = h->fill_chosen;
  return FP_OK;
}

fp_status fp_gnn_scores(fp_handle* h, const int32_t* h_codes, int32_t* d_scores, uint8_t* d_features) {
  if (!h || !h_codes) return fail(h, FP_ERR_INVALID_ARG, "NULL handle or codes");
  if (h->poisoned) return fail(h, FP_ERR_STATE, "handle poisoned by an earlier failure");
  if (!h->permuted) return fail(h, FP_ERR_STATE, "fp_gnn_scores before fp_permute");
  if (!codes_valid(h_codes)) return fail(h, FP_ERR_INVALID_ARG, "network code out of range");
  const int32_t n = h->n;
  if (n == 0) return FP_OK;
  int32_t* q = (int32_t*)dev_alloc(h, sizeof(int32_t) * FP_GNN_NPARAMS);
  uint32_t* key = (uint32_t*)dev_alloc(h, sizeof(uint32_t) * n);
  if (!q || !key) return fail(h, FP_ERR_OUT_OF_MEMORY, "score workspace");
  cudaError_t e = cudaMemcpyAsync(q, h_codes, sizeof(int32_t) * FP_GNN_NPARAMS, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "network codes");
  if (d_scores) cudaMemsetAsync(d_scores, 0, sizeof(int32_t) * n, h->stream);
  if (d_features) cudaMemsetAsync(d_features, 0, (size_t)8 * n, h->stream);
  std::vector<int32_t> hl;
  int32_t* dl = nullptr;
  int32_t mmax = 0;
  FP_TRY(leaf_list(h, hl, &dl, &mmax));
  FP_TRY(launch_gnn_score(h, dl, (int32_t)hl.size(), q, key, d_scores, d_features));
  int32_t st = 0;
  FP_TRY(sync_status(h, &st));
  for (void* p : {(void*)q, (void*)key, (void*)dl}) dev_free(h, p);
  if (st & ST_TIMEOUT) return fail(h, FP_ERR_TIMEOUT, "tensor-core wait ran out");
  return FP_OK;
}

namespace {

// Host destinations of the symbolic outputs (the host-buffer entry point):
// the columns outside the tree's top EARLY_SYM_LEVELS levels are final before
// those levels' launches run; they are expanded to DOFs and copied to the
// host on an auxiliary stream while the top levels run, and only the top
// nodes' column ranges follow at the end.
struct SymbolicHost {
  int32_t* parent;
  int32_t* colcount;
};
constexpr int EARLY_SYM_LEVELS = 5;
// below this many output bytes the copies are short and the early path's
// extra copy calls cost more than they hide
constexpr int64_t EARLY_SYM_MIN_BYTES = 16 << 20;

fp_status symbolic_impl(fp_handle* h, int32_t* d_parent, int32_t* d_colcount, int64_t* h_nnzL, int64_t* h_flops,
                        const SymbolicHost* ho) {
  if (!h) return fail(nullptr, FP_ERR_INVALID_ARG, "NULL handle");
  if (h->poisoned) return fail(h, FP_ERR_STATE, "handle poisoned by an earlier failure");
  if (!h->permuted) return fail(h, FP_ERR_STATE, "fp_symbolic before fp_permute");
  const int32_t n = h->n, b = h->b;
  const int64_t N = (int64_t)n * b;
  int32_t* par = (b == 1 && d_parent) ? d_parent : (int32_t*)dev_alloc(h, sizeof(int32_t) * (n > 0 ? n : 1));
  int32_t* cc = (b == 1 && d_colcount) ? d_colcount : (int32_t*)dev_alloc(h, sizeof(int32_t) * (n > 0 ? n : 1));
  if (!par || !cc) return fail(h, FP_ERR_OUT_OF_MEMORY, "symbolic outputs");
  AuxStream* ax = nullptr;
  int32_t* top_begin = nullptr;
  int64_t ntop = 0;
  bool queued = false;
  if (ho && N > 0 && d_parent && d_colcount && 8 * N >= EARLY_SYM_MIN_BYTES) {
    ax = aux_stream(h->device, 0);
    top_begin = pinned_scratch();
    if (!ax || !top_begin) return fail(h, FP_ERR_CUDA, "auxiliary stream");
    ntop = std::min<int64_t>(h->nnodes, ((int64_t)1 << EARLY_SYM_LEVELS) - 1);
    // read after run_symbolic's final sync
    cudaMemcpyAsync(top_begin, h->node_begin, sizeof(int32_t) * ntop, cudaMemcpyDeviceToHost, h->stream);
    h->sym_early_depth = EARLY_SYM_LEVELS;
    h->sym_early = [&](cudaEvent_t ev) {
      cudaStreamWaitEvent(ax->s, ev, 0);
      if (b > 1) launch_dof_expand_symbolic(h, par, cc, d_parent, d_colcount, 0, n, ax->s);
      if (ho->parent) cudaMemcpyAsync(ho->parent, d_parent, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, ax->s);
      if (ho->colcount) cudaMemcpyAsync(ho->colcount, d_colcount, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, ax->s);
      cudaEventRecord(ax->join, ax->s);
      queued = true;
    };
  }
  int64_t nnz = 0, fl = 0;
  fp_status st = run_symbolic(h, par, cc, &nnz, &fl);
  h->sym_early = nullptr;
  // the host copies of the early pass end before anything below writes the
  // same host ranges (and before the caller frees the device buffers)
  if (queued) cudaStreamWaitEvent(h->stream, ax->join, 0);
  FP_TRY(st);
  const bool top_only = queued && h->sym_early_fired;
  auto finish = [&](int32_t v0, int32_t v1) {
    if (b > 1) launch_dof_expand_symbolic(h, par, cc, d_parent, d_colcount, v0, v1);
    if (!ho) return;
    const size_t off = (size_t)v0 * b, len = (size_t)(v1 - v0) * b;
    if (ho->parent && len)
      cudaMemcpyAsync(ho->parent + off, d_parent + off, sizeof(int32_t) * len, cudaMemcpyDeviceToHost, h->stream);
    if (ho->colcount && len)
      cudaMemcpyAsync(ho->colcount + off, d_colcount + off, sizeof(int32_t) * len, cudaMemcpyDeviceToHost, h->stream);
  };
  if (top_only) {
    // the top nodes' column ranges, adjacent ones merged (in post-order a
    // node's columns follow its right child's)
    std::vector<std::pair<int32_t, int32_t>> r;
    for (int64_t t = 0; t < ntop; ++t) {
      const int32_t sz = h->node_size_host[t];
      if (sz > 0) r.push_back({top_begin[t], top_begin[t] + sz});
    }
    std::sort(r.begin(), r.end());
    for (size_t i = 0; i < r.size();) {
      size_t j = i + 1;
      int32_t end = r[i].second;
      while (j < r.size() && r[j].first == end) end = r[j++].second;
      finish(r[i].first, end);
      i = j;
    }
  } else if (b > 1 || ho) {
    finish(0, n);
  }
  FP_CHECK_LAUNCH(h, "dof expansion");
  if (b > 1) {
    const int64_t B = b;
    const int64_t nnz_d = B * B * nnz - (int64_t)n * B * (B - 1) / 2;
    const int64_t fl_d = B * B * B * fl - B * B * (B - 1) * nnz + (int64_t)n * (B - 1) * B * (2 * B - 1) / 6;
    nnz = nnz_d;
    fl = fl_d;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return check_cuda(h, e, "symbolic sync");
  }
  if (par != d_parent) dev_free(h, par);
  if (cc != d_colcount) dev_free(h, cc);
  if (h_nnzL) *h_nnzL = nnz;
  if (h_flops) *h_flops = fl;
  return FP_OK;
}

}  // namespace

fp_status fp_symbolic(fp_handle* h, int32_t* d_parent, int32_t* d_colcount, int64_t* h_nnzL, int64_t* h_flops) {
  return symbolic_impl(h, d_parent, d_colcount, h_nnzL, h_flops, nullptr);
}

fp_status fp_get_stage(fp_handle* h, int32_t stage, int32_t index, int32_t* d_out, int64_t cap, int64_t* h_len) {
  if (!h) return fail(nullptr, FP_ERR_INVALID_ARG, "NULL handle");
  if (h->poisoned) return fail(h, FP_ERR_STATE, "handle poisoned by an earlier failure");
  if (!h->permuted || !h->opt.debug_dump) return fail(h, FP_ERR_STATE, "no stage record: create the handle with "
                                                                    "debug_dump = 1 and call fp_permute");
  for (const auto& e : h->dumps) {
    if (e.stage != stage || e.index != index) continue;
    if (h_len) *h_len = e.len;
    if (!d_out) return FP_OK;
    if (cap < e.len) return fail(h, FP_ERR_INVALID_ARG, "stage buffer too small");
    if (e.len > 0) cudaMemcpyAsync(d_out, e.d, sizeof(int32_t) * (size_t)e.len, cudaMemcpyDeviceToDevice, h->stream);
    FP_CHECK_LAUNCH(h, "stage copy");
    return FP_OK;
  }
  return fail(h, FP_ERR_STATE, "stage not recorded by the last fp_permute");
}

fp_status fp_get_sizes(const fp_handle* h, int32_t* h_n, int32_t* h_dof, int64_t* h_nnz) {
  if (!h) return FP_ERR_INVALID_ARG;
  if (h_n) *h_n = h->n;
  if (h_dof) *h_dof = h->b;
  if (h_nnz) *h_nnz = h->nnz;
  return FP_OK;
}

fp_status fp_get_graph(fp_handle* h, int32_t* d_rowptr, int32_t* d_col) {
  if (!h) return FP_ERR_INVALID_ARG;
  if (h->poisoned) return fail(h, FP_ERR_STATE, "handle poisoned");
  if (d_rowptr) cudaMemcpyAsync(d_rowptr, h->rowptr, sizeof(int32_t) * (h->n + 1), cudaMemcpyDeviceToDevice, h->stream);
  if (d_col && h->nnz) cudaMemcpyAsync(d_col, h->col, sizeof(int32_t) * h->nnz, cudaMemcpyDeviceToDevice, h->stream);
  FP_CHECK_LAUNCH(h, "get graph");
  return FP_OK;
}

fp_status fp_get_patches(fp_handle* h, int32_t* d_gmap, int32_t* h_k) {
  if (!h) return FP_ERR_INVALID_ARG;
  if (!h->permuted) return fail(h, FP_ERR_STATE, "no permutation yet");
  if (d_gmap && h->n) cudaMemcpyAsync(d_gmap, h->gmap, sizeof(int32_t) * h->n, cudaMemcpyDeviceToDevice, h->stream);
  if (h_k) *h_k = h->k;
  FP_CHECK_LAUNCH(h, "get patches");
  return FP_OK;
}

namespace fp {
// Copies a caller's patch map, flagging labels outside [0, k).
__global__ void k_copy_labels(const int32_t* __restrict__ g, int32_t n, int32_t k, int32_t* __restrict__ out,
                              int32_t* status) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int32_t p = g[v];
    if (p < 0 || p >= k) atomicOr(status, ST_BAD_INDEX);
    out[v] = p;
  }
}
}  // namespace fp

fp_status fp_set_patches(fp_handle* h, const int32_t* d_gmap, int32_t k) {
  if (!h) return fail(nullptr, FP_ERR_INVALID_ARG, "NULL handle");
  if (h->poisoned) return fail(h, FP_ERR_STATE, "handle poisoned by an earlier failure");
  if (k < 1 || (h->n > 0 && !d_gmap)) return fail(h, FP_ERR_INVALID_ARG, "patch map: NULL map or k < 1");
  if (!h->user_gmap) {
    h->user_gmap = (int32_t*)dev_alloc(h, sizeof(int32_t) * (h->n > 0 ? h->n : 1));
    if (!h->user_gmap) return fail(h, FP_ERR_OUT_OF_MEMORY, "patch map");
  }
  if (h->n > 0) {
    int64_t g = ((int64_t)h->n + 255) / 256;
    if (g > NUM_SMS_B300 * 32) g = NUM_SMS_B300 * 32;
    FP_LAUNCH(h, k_copy_labels, (int)g, 256, 0, d_gmap, h->n, k, h->user_gmap, h->d_status);
  }
  FP_CHECK_LAUNCH(h, "patch map");
  int32_t st = 0;
  FP_TRY(sync_status(h, &st));
  h->permuted = false;
  if (st & ST_BAD_INDEX) {
    h->user_k = 0;
    cudaMemsetAsync(h->d_status, 0, sizeof(int32_t), h->stream);
    return fail(h, FP_ERR_INVALID_ARG, "patch map: a label outside [0, k)");
  }
  h->user_k = k;
  return FP_OK;
}

fp_status fp_get_tree(fp_handle* h, int32_t* h_depth, int32_t* d_node_begin, int32_t* d_node_size, int32_t* d_node_of) {
  if (!h) return FP_ERR_INVALID_ARG;
  if (!h->permuted) return fail(h, FP_ERR_STATE, "no permutation yet");
  if (h_depth) *h_depth = h->D;
  if (d_node_begin) cudaMemcpyAsync(d_node_begin, h->node_begin, sizeof(int32_t) * h->nnodes, cudaMemcpyDeviceToDevice, h->stream);
  if (d_node_size) cudaMemcpyAsync(d_node_size, h->node_size, sizeof(int32_t) * h->nnodes, cudaMemcpyDeviceToDevice, h->stream);
  if (d_node_of && h->n) cudaMemcpyAsync(d_node_of, h->node_of, sizeof(int32_t) * h->n, cudaMemcpyDeviceToDevice, h->stream);
  FP_CHECK_LAUNCH(h, "get tree");
  return FP_OK;
}

fp_status fp_order_faces_host(const int32_t* h_faces, int64_t n_faces, int32_t n_vertices, const fp_options* opts,
                              void* stream, int32_t* h_perm, int32_t* h_iperm, int32_t* h_parent, int32_t* h_colcount,
                              int64_t* h_nnzL, int64_t* h_flops) {
  if (validate_options(opts) != FP_OK || n_vertices < 0 || n_faces < 0 || (n_faces > 0 && !h_faces))
    return fail(nullptr, FP_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPool_t pool = library_pool(dev);
  const int64_t N = (int64_t)n_vertices * opts->dof_per_vertex;
  int32_t* d_faces = nullptr;
  int32_t* d_out = nullptr;
  if (cudaMallocFromPoolAsync((void**)&d_faces, sizeof(int32_t) * 3 * (n_faces > 0 ? n_faces : 1), pool, s) != cudaSuccess ||
      cudaMallocFromPoolAsync((void**)&d_out, sizeof(int32_t) * 4 * (N > 0 ? N : 1), pool, s) != cudaSuccess)
    return fail(nullptr, FP_ERR_OUT_OF_MEMORY, "staging buffers");
  if (n_faces > 0) cudaMemcpyAsync(d_faces, h_faces, sizeof(int32_t) * 3 * n_faces, cudaMemcpyHostToDevice, s);
  fp_handle* h = nullptr;
  fp_status st = fp_create_from_faces(d_faces, n_faces, n_vertices, opts, stream, &h);
  if (st == FP_OK) st = fp_permute(h, d_out, d_out + N);
  // perm and iperm are final here: their copies to the host run on an
  // auxiliary stream while the symbolic factorisation runs on `stream`
  AuxStream* ax = st == FP_OK && N > 0 ? aux_stream(dev, 1) : nullptr;
  int32_t* hs[4] = {h_perm, h_iperm, h_parent, h_colcount};
  if (ax) {
    cudaEventRecord(ax->fork, s);
    cudaStreamWaitEvent(ax->s, ax->fork, 0);
    for (int i = 0; i < 2; ++i)
      if (hs[i]) cudaMemcpyAsync(hs[i], d_out + i * N, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, ax->s);
    cudaEventRecord(ax->join, ax->s);
  }
  int64_t nnz = 0, fl = 0;
  // parent and colcount reach the host as soon as their columns are final
  const SymbolicHost ho{h_parent, h_colcount};
  if (st == FP_OK) st = symbolic_impl(h, d_out + 2 * N, d_out + 3 * N, &nnz, &fl, &ho);
  if (ax) cudaStreamWaitEvent(s, ax->join, 0);     // d_out is freed on `stream` below
  if (st != FP_OK && h) g_create_err = h->err;
  fp_destroy(h);
  cudaFreeAsync(d_faces, s);
  cudaFreeAsync(d_out, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (st == FP_OK && e != cudaSuccess) return fail(nullptr, FP_ERR_CUDA, cudaGetErrorString(e));
  if (h_nnzL) *h_nnzL = nnz;
  if (h_flops) *h_flops = fl;
  return st;
}

fp_status fp_factor(fp_handle* h, const double* d_diag, const double* d_offdiag) {
  if (!h) return fail(nullptr, FP_ERR_INVALID_ARG, "NULL handle");
  if (h->poisoned) return fail(h, FP_ERR_STATE, "handle poisoned by an earlier failure");
  if (!h->permuted) return fail(h, FP_ERR_STATE, "fp_factor before fp_permute");
  if (h->b != 1) return fail(h, FP_ERR_UNSUPPORTED, "fp_factor: dof_per_vertex > 1");
  if (h->n > 0 && (!d_diag || (h->nnz > 0 && !d_offdiag))) return fail(h, FP_ERR_INVALID_ARG, "NULL values");
  if (h->n == 0) return FP_OK;
  return run_factor(h, d_diag, d_offdiag);
}

fp_status fp_solve(fp_handle* h, const double* d_b, double* d_x) {
  if (!h) return fail(nullptr, FP_ERR_INVALID_ARG, "NULL handle");
  if (h->poisoned) return fail(h, FP_ERR_STATE, "handle poisoned by an earlier failure");
  if (!h->numeric) return fail(h, FP_ERR_STATE, "fp_solve before fp_factor");
  if (h->n > 0 && (!d_b || !d_x)) return fail(h, FP_ERR_INVALID_ARG, "NULL vector");
  if (h->n == 0) return FP_OK;
  return run_solve(h, d_b, d_x);
}

fp_status fp_factor_export(fp_handle* h, int64_t* d_colptr, int32_t* d_rows, double* d_vals, int64_t cap,
                           int64_t* h_nnz) {
  if (!h) return fail(nullptr, FP_ERR_INVALID_ARG, "NULL handle");
  if (h->poisoned) return fail(h, FP_ERR_STATE, "handle poisoned by an earlier failure");
  if (!h->numeric) return fail(h, FP_ERR_STATE, "fp_factor_export before fp_factor");
  return run_factor_export(h, d_colptr, d_rows, d_vals, cap, h_nnz);
}

fp_status fp_factor_stats(const fp_handle* h, int64_t* h_front_doubles, int64_t* h_flops, int64_t* h_nnz) {
  if (!h) return fail(nullptr, FP_ERR_INVALID_ARG, "NULL handle");
  numeric_stats(h, h_front_doubles, h_flops, h_nnz);
  return FP_OK;
}

fp_status fp_destroy(fp_handle* h) {
  if (!h) return FP_OK;
  numeric_release(h);
  for (void* p : h->allocs) cudaFreeAsync(p, h->stream);
  h->allocs.clear();
  // stream-ordered frees only: every copy into the status word was waited
  // for when it was made, and the auxiliary streams' work was joined into
  // the handle's stream before the call that launched it returned
  if (h->h_status) status_word_give(h->h_status);
  delete h->seg;
  delete h;
  return FP_OK;
}

const char* fp_last_error(const fp_handle* h) {
  if (h) return h->err.empty() ? "no error" : h->err.c_str();
  return g_create_err.c_str();
}

const char* fp_status_string(fp_status s) {
  switch (s) {
    case FP_OK: return "FP_OK";
    case FP_ERR_INVALID_ARG: return "FP_ERR_INVALID_ARG";
    case FP_ERR_NOT_SYMMETRIC: return "FP_ERR_NOT_SYMMETRIC";
    case FP_ERR_OUT_OF_MEMORY: return "FP_ERR_OUT_OF_MEMORY";
    case FP_ERR_CUDA: return "FP_ERR_CUDA";
    case FP_ERR_TIMEOUT: return "FP_ERR_TIMEOUT";
    case FP_ERR_STATE: return "FP_ERR_STATE";
    case FP_ERR_UNSUPPORTED: return "FP_ERR_UNSUPPORTED";
  }
  return "FP_ERR_UNKNOWN";
}

int64_t fp_launch_count(const fp_handle* h) { return h ? h->launches : 0; }

void fp_profiling(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
}

int fp_profile_read(double* ms, int64_t* launches, int cap) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_drain_locked();
  for (int i = 0; i < FP_PROF_COUNT && i < cap; ++i) {
    if (ms) ms[i] = g_prof_ms[i];
    if (launches) launches[i] = g_prof_n[i];
  }
  return FP_PROF_COUNT;
}

void fp_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_drain_locked();
  for (int i = 0; i < FP_PROF_COUNT; ++i) { g_prof_ms[i] = 0.0; g_prof_n[i] = 0; }
}

}  // extern "C"
