// Internal declarations of the fastperm CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <utility>
#include <vector>

#include "../../include/fastperm.h"

namespace fp {

constexpr unsigned long long KEY_INF = ~0ull;
constexpr int NUM_SMS_B300 = 148;

// Grid for a grid-stride loop over n items: one item per thread, at most
// per_sm CTAs per SM.
inline int grid_for(int64_t n, int threads, int per_sm = 32) {
  int64_t g = (n + threads - 1) / threads;
  if (g > (int64_t)NUM_SMS_B300 * per_sm) g = (int64_t)NUM_SMS_B300 * per_sm;
  return (int)(g < 1 ? 1 : g);
}

// Device status word bits (set by kernels, read by the host at sync points).
enum : int32_t {
  ST_BAD_INDEX = 1 << 0,       // an input index out of range
  ST_ROW_TOO_LONG = 1 << 1,    // a CSR row beyond the sort capacity
  ST_NOT_SYMMETRIC = 1 << 2,   // CSR pattern not symmetric
  ST_POOL_OVERFLOW = 1 << 3,   // a device bump pool ran out (host retries bigger)
  ST_NODE_TOO_BIG = 1 << 4,    // a tree node beyond the ordering kernel's limit
  ST_QUOTIENT_TOO_BIG = 1 << 5, // a patch with more cross edges than the sort capacity
  ST_TIMEOUT = 1 << 6,          // a bounded device wait ran out
  ST_NOT_SPD = 1 << 7,          // a Cholesky pivot was not positive
  ST_BAD_ROWPTR = 1 << 8        // a CSR row pointer array that is not a valid prefix
};

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output for generator state s
// is the finaliser of s + gamma.
__host__ __device__ __forceinline__ uint64_t splitmix64_state(uint64_t s) {
  uint64_t z = s + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Workspace;   // per-handle device scratch (fp_api.cu)

// A batch of meshes ordered as one graph, their disjoint union (the fused
// batch ordering, k_batch.cu). Mesh m owns the union's vertices
// [voff[m], voff[m+1]); no edge, patch or tree node joins two meshes. The few
// kernels whose result depends on a mesh's own size, cap or vertex numbering
// (the seed threshold, the cap splits, the separator tie hash) read them here;
// a single-mesh handle passes the empty view (vmesh == nullptr).
struct SegView {
  const int32_t* vmesh = nullptr;   // [n] mesh of every union vertex
  const int32_t* voff = nullptr;    // [M+1] first union vertex of every mesh
  const int32_t* mcap = nullptr;    // [M] patch cap of every mesh
};
// Host side of the union (owned by the handle). Every mesh's dissection tree
// hangs below an empty super-tree at depth D - h_m, h_m = ceil(log2 k_m), so
// that all leaves lie at depth D (a canonical prefix code of the meshes,
// largest subtree first): every node at depth d then has the cut bound
// 2^(D-d-1) of a single mesh dissected to depth D.
struct Segments {
  int32_t M = 0;
  SegView v;                         // device arrays
  int32_t* mroot = nullptr;          // [M] device: root node of every mesh's subtree
  std::vector<int32_t> h_voff;       // [M+1]
  std::vector<int32_t> h_root;       // [M] root node (-1: an empty mesh)
  std::vector<int32_t> h_k;          // [M] patches of every mesh
  std::vector<int32_t> h_posoff;     // [M] first position of every mesh in the union's order
  std::vector<int32_t> h_cap;        // [M] patch cap of every mesh
  int32_t* d_posoff = nullptr;       // [M] device copy of h_posoff
  void* d_outs = nullptr;            // [M] device table of the items' output pointers
  // learned form, per mesh: leaves considered, learned orders kept, summed
  // plain and chosen leaf fills
  std::vector<unsigned long long> h_learned;   // [M][4]
  int32_t dmin = 0;                  // shallowest root depth
};
struct NumericFactor;   // numeric Cholesky factor of a handle (k_numeric.cu)

// a10 priority network: packed parameter layout (codes or floats)
// w1s[32][6] w1n[32][6] b1[32] w2s[32][32] w2n[32][32] b2[32] w3[32] c
constexpr int GNN_FIN = 6;
constexpr int GNN_HID = 32;
constexpr int GNN_LEAF_MAX = 512;
constexpr int P_W1S = 0, P_W1N = 192, P_B1 = 384, P_W2S = 416, P_W2N = 1440, P_B2 = 2464, P_W3 = 2496,
              P_C = 2528, P_COUNT = 2529;
static_assert(P_COUNT == FP_GNN_NPARAMS, "parameter layout");

}  // namespace fp

struct fp_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  fp_options opt{};
  int32_t n = 0;         // vertices
  int32_t b = 1;         // DOFs per vertex
  int64_t nnz = 0;       // adjacency entries of G (2E)
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;

  bool permuted = false;
  bool poisoned = false;
  int32_t k = 0;         // patches
  int32_t D = 0;         // tree depth
  int64_t nnodes = 0;    // 2^(D+1)-1

  // persistent results (vertex level)
  int32_t* gmap = nullptr;        // [n]
  int32_t* node_of = nullptr;     // [n]
  int32_t* perm = nullptr;        // [n]
  int32_t* iperm = nullptr;       // [n]
  int32_t* node_begin = nullptr;  // [nnodes]
  int32_t* node_size = nullptr;   // [nnodes]
  int64_t node_cap = 0;           // allocated length of node arrays
  std::vector<int32_t> node_size_host;   // host copy of node_size (set by the ordering stage)

  int32_t* d_status = nullptr;    // device status word
  int32_t* h_status = nullptr;    // pinned mirror
  void* scratch = nullptr;        // generic scratch block
  size_t scratch_bytes = 0;

  // separators ordered early (during nested dissection, on the auxiliary
  // stream): the first early_nodes tree nodes, their vertex lists, each
  // vertex's rank inside its node, and per-node adjacency-overflow flags
  int32_t early_nodes = 0;
  int32_t *early_rank = nullptr, *early_list = nullptr, *early_start = nullptr, *early_cnt = nullptr;
  int32_t *early_fill = nullptr, *early_ovf = nullptr, *early_loc = nullptr, *early_base = nullptr;

  // patches supplied by the caller (fp_set_patches): device copy and count
  int32_t* user_gmap = nullptr;
  int32_t user_k = 0;

  // a10 learned priorities
  int32_t* qnet = nullptr;        // device codes [FP_GNN_NPARAMS], or null (plain)
  int32_t* scores = nullptr;      // optional per-position score output of the learned pass
  int32_t learned_leaves = 0, learned_kept = 0;
  int64_t fill_plain = 0, fill_chosen = 0;

  // the learned pass runs beside the separator orderings: run_local_order
  // leaves them on the auxiliary streams (join_pending), with the buffers to
  // free after the join and the vertex lists by node (positions for the
  // provisional permutation); finish_orderings joins
  bool join_pending = false;
  std::vector<void*> join_frees;
  const int32_t* pend_nvlist = nullptr;
  const int32_t* pend_nvstart = nullptr;

  // numeric factor (fp_factor), released by fp_permute and fp_destroy
  fp::NumericFactor* numeric = nullptr;

  // the disjoint union of a fused batch (null for one mesh)
  fp::Segments* seg = nullptr;

  // run_symbolic calls sym_early(event) once, on its first pass, as soon as
  // every column outside the tree's top sym_early_depth levels is final (the
  // event marks that point on the handle's stream); sym_early_fired says
  // whether that pass was the one that completed
  std::function<void(cudaEvent_t)> sym_early;
  int32_t sym_early_depth = 0;
  bool sym_early_fired = false;

  // stage boundaries kept for fp_get_stage (opt.debug_dump)
  struct StageDump {
    int32_t stage, index;
    int32_t* d;
    int64_t len;
  };
  std::vector<StageDump> dumps;

  std::string err;
  int64_t launches = 0;
  std::vector<void*> allocs;
};

namespace fp {

// ---- host helpers (fp_api.cu) ------------------------------------------------
cudaMemPool_t library_pool(int device);
void* dev_alloc(fp_handle* h, size_t bytes);      // stream-ordered, tracked; nullptr on failure
void dev_free(fp_handle* h, void* p);
fp_status fail(fp_handle* h, fp_status s, const std::string& msg);
fp_status check_cuda(fp_handle* h, cudaError_t e, const char* what);
fp_status sync_status(fp_handle* h, int32_t* status_out);   // sync stream, read status word
// Stage boundaries for fp_get_stage (no-ops unless opt.debug_dump): a new
// handle-owned buffer of `len` ints recorded as (stage, index), or a copy of
// `src` into one. stage_clear drops the records of an earlier fp_permute.
int32_t* stage_buffer(fp_handle* h, int32_t stage, int32_t index, int64_t len);
void stage_dump(fp_handle* h, int32_t stage, int32_t index, const int32_t* src, int64_t len);
void stage_clear(fp_handle* h);
// Many workspace arrays from one allocation: a layout function calls get()
// for every array twice, first to size the block (pointers come back null),
// then, after alloc(), to hand out 256-byte aligned pieces of it. One
// stream-ordered allocation and one free instead of one per array.
struct Arena {
  char* base = nullptr;
  size_t off = 0;
  template <class T>
  T* get(int64_t count) {
    const size_t bytes = ((size_t)(count > 0 ? count : 1) * sizeof(T) + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += bytes;
    return p;
  }
  bool alloc(fp_handle* h) {
    base = (char*)dev_alloc(h, off);
    off = 0;
    return base != nullptr;
  }
};
// Per-thread pinned host scratch of 256 ints (allocated once per thread).
int32_t* pinned_scratch();
// Per-thread pinned host buffer of at least `count` ints (grown on demand;
// the contents do not survive a growth). nullptr on failure.
int32_t* pinned_ints(int64_t count);
// Per-thread, per-device event without timing, for a host wait on part of a
// stream (the work queued after it keeps the GPU busy meanwhile).
cudaEvent_t mark_event(int device);
// Per-thread, per-device auxiliary streams (which = 0 or 1) with a fork and a
// join event each, created once and reused (stage kernels that overlap run on
// them).
struct AuxStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
AuxStream* aux_stream(int device, int which = 0);

// Raises a kernel's dynamic shared-memory limit to the device maximum minus its
// static shared memory and asks for the largest shared-memory carveout. Every
// caller sets the same values, so concurrent host threads launching the same
// kernel with different sizes cannot race. Done once per kernel and device,
// under a lock (fp_api.cu): setting a function attribute while the kernel runs
// on another stream can hold the host until it finishes.
void allow_max_dynamic_smem_fn(const void* kernel);
template <class K>
inline void allow_max_dynamic_smem(K kernel) {
  allow_max_dynamic_smem_fn((const void*)kernel);
}

// ---- stage profiling (fp_api.cu) -------------------------------------------------
bool profiling_on();
void prof_record(int kind, cudaEvent_t start, cudaEvent_t end);
cudaEvent_t prof_event();
// Records an event pair around a scope on `stream` when profiling is on.
struct ProfScope {
  int kind;
  cudaStream_t stream;
  cudaEvent_t a = nullptr;
  ProfScope(int k, cudaStream_t s) : kind(k), stream(s) {
    if (profiling_on()) {
      a = prof_event();
      cudaEventRecord(a, stream);
    }
  }
  void end() {
    if (a) {
      cudaEvent_t b = prof_event();
      cudaEventRecord(b, stream);
      prof_record(kind, a, b);
      a = nullptr;
    }
  }
  ~ProfScope() { end(); }
};

// ---- primitives (fp_scan.cu) ---------------------------------------------------
// Exclusive scan of in[0..n) into out[0..n]; out[n] = total. in != out.
// `tmp` needs scan_tmp_ints(n) ints.
int64_t scan_tmp_ints(int64_t n);
void scan_exclusive(fp_handle* h, const int32_t* in, int32_t* out, int64_t n, int32_t* tmp);
void fill_i32(fp_handle* h, int32_t* p, int32_t v, int64_t n);
// Exclusive scans a -> oa and b -> ob (each of n items, out[n] = total), then
// b is zeroed. One launch for short arrays.
void scan_exclusive_pair_zero(fp_handle* h, const int32_t* a, int32_t* oa, int32_t* b, int32_t* ob, int64_t n,
                              int32_t* tmp);
void iota_i32(fp_handle* h, int32_t* p, int64_t n);

// ---- stages -----------------------------------------------------------------------
// a1: CSR of G from faces or from a (block) pattern. Allocates h->rowptr/col.
fp_status build_graph_from_faces(fp_handle* h, const int32_t* d_faces, int64_t nf);
fp_status build_graph_from_csr(fp_handle* h, const int32_t* d_rowptr, const int32_t* d_col, int32_t nrows);

// a2: patching; writes h->gmap and h->k.
fp_status run_patching(fp_handle* h);
// a3 + a4: quotient graph and nested dissection; writes h->node_of, h->D.
fp_status run_nested_dissection(fp_handle* h);
// a5 + a6: tree layout, local minimum degree, perm/iperm.
fp_status run_local_order(fp_handle* h);
// Early separator ordering (k_md.cu): called by the nested dissection once the
// nodes of depth d are final; orders them on the auxiliary stream while the
// deeper levels are dissected. run_local_order places the results.
fp_status early_md_begin(fp_handle* h, int32_t levels);
fp_status launch_early_md(fp_handle* h, int32_t d);
void early_md_release(fp_handle* h);
// a7: symbolic (vertex level) into parent/colcount [n]; nnz/flops sums.
fp_status run_symbolic(fp_handle* h, int32_t* d_parent, int32_t* d_colcount, int64_t* nnzL, int64_t* flops);
// a10 (k_gnn.cu, k_md.cu, k_symbolic.cu)
fp_status run_learned(fp_handle* h);
// Joins the separator orderings that run_local_order left running (a no-op
// unless h->join_pending): the handle's stream waits for both auxiliary
// streams, then the ordering stage's buffers are freed.
fp_status finish_orderings(fp_handle* h);
// lsz (optional) receives the listed leaves' sizes, in list order.
fp_status leaf_list(fp_handle* h, std::vector<int32_t>& hl, int32_t** d_list, int32_t* mmax,
                    std::vector<int32_t>* lsz = nullptr);
// perm/iperm: the positions to read (null: the handle's own).
fp_status launch_gnn_score(fp_handle* h, const int32_t* d_leaves, int32_t nl, const int32_t* d_q, uint32_t* d_key,
                           int32_t* d_score, uint8_t* d_x, const int32_t* perm = nullptr,
                           const int32_t* iperm = nullptr);
// lsz (optional): the nodes' sizes in list order (largest first), which lets
// the leaves run in two size classes like the plain leaf orderings.
fp_status run_leaf_md_keyed(fp_handle* h, const int32_t* d_nodes, int32_t count, int32_t mmax, int32_t* vlist,
                            int32_t* loc, const uint32_t* key, int32_t* perm_out,
                            const std::vector<int32_t>* lsz = nullptr);
fp_status run_leaf_fill(fp_handle* h, const int32_t* perm, const int32_t* iperm, const int32_t* d_nodes,
                        int32_t count, int64_t* d_fill);
// f4: numeric Cholesky of P A P^T over the tree (k_numeric.cu).
fp_status run_factor(fp_handle* h, const double* d_diag, const double* d_off);
fp_status run_solve(fp_handle* h, const double* d_b, double* d_x);
fp_status run_factor_export(fp_handle* h, int64_t* d_colptr, int32_t* d_rows, double* d_vals, int64_t cap,
                            int64_t* h_nnz);
void numeric_stats(const fp_handle* h, int64_t* front_doubles, int64_t* flops, int64_t* nnz);
void numeric_release(fp_handle* h);
// a8: DOF expansion of perm/iperm/parent/colcount (b > 1).
void launch_dof_expand_perm(fp_handle* h, const int32_t* perm, int32_t* perm_d, int32_t* iperm_d);
// columns [v0, v1) (v1 < 0: to the end) on stream s (null: the handle's)
void launch_dof_expand_symbolic(fp_handle* h, const int32_t* parent, const int32_t* colcount, int32_t* parent_d,
                                int32_t* colcount_d, int32_t v0 = 0, int32_t v1 = -1, cudaStream_t s = nullptr);

}  // namespace fp

namespace fp {

// Launches on the handle's stream allow programmatic dependent launch: the
// next kernel's CTAs may be scheduled as soon as every CTA of the one before
// has exited, without waiting for the grid's completion to be processed.
// Every kernel of the library therefore starts with FP_PDL_WAIT(), which
// holds it until the previous grid has completed and its writes are visible
// (a no-op for a launch that did not allow the early start).
template <class... KArgs, class... Args>
inline void launch_pdl(cudaStream_t s, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace fp

#define FP_PDL_WAIT() asm volatile("griddepcontrol.wait;" ::: "memory")

#define FP_LAUNCH(h, kernel, grid, block, smem, ...)                                  \
  do {                                                                                \
    fp::launch_pdl((h)->stream, kernel, dim3(grid), dim3(block), (size_t)(smem), __VA_ARGS__); \
    (h)->launches++;                                                                  \
  } while (0)

#define FP_CHECK_LAUNCH(h, what)                                                      \
  do {                                                                                \
    cudaError_t e_ = cudaGetLastError();                                              \
    if (e_ != cudaSuccess) return fp::check_cuda((h), e_, (what));                    \
  } while (0)

#define FP_TRY(expr)                                                                  \
  do {                                                                                \
    fp_status s_ = (expr);                                                            \
    if (s_ != FP_OK) return s_;                                                       \
  } while (0)
