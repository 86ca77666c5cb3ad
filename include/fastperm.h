/*
 * fastperm.h — C ABI of the B300 (sm_103a) fill-reducing permutation library.
 *
 * Computes the patch-guided nested-dissection ordering of "Fast Sparse Matrix
 * Permutation for Mesh-Based Direct Solvers" (Algorithm 1: patches -> group
 * map -> elimination tree -> permutation) for the matrix of a triangle mesh,
 * plus the elimination tree and column counts of its Cholesky factor. Every
 * step runs in the library's own CUDA kernels; the host code only sequences
 * launches on the caller's stream.
 *
 * Conventions shared by all calls
 *  - Pointers named d_* are device pointers (the current CUDA device), h_*
 *    are host pointers. The caller owns every buffer it passes; the library
 *    owns the handle and the workspace it allocates (stream-ordered, from a
 *    library-private memory pool) and frees them in fp_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All work of a handle is ordered on the stream given at creation. Calls
 *    that return host values (h_*) synchronise that stream; the others do not
 *    unless noted.
 *  - perm[k] is the original vertex placed at new position k (Algorithm 3's
 *    "Append" order); iperm[perm[k]] = k. Elimination-tree parents and column
 *    counts are indexed by new position; a root has parent -1.
 *  - Errors are returned as fp_status, never thrown. After FP_ERR_CUDA or
 *    FP_ERR_TIMEOUT the handle is poisoned: further calls return
 *    FP_ERR_STATE; fp_destroy still releases it. fp_last_error() gives a
 *    message for the most recent failure.
 *  - Not thread-safe per handle; distinct handles may be used concurrently.
 */
#ifndef FASTPERM_H
#define FASTPERM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fp_handle fp_handle;

typedef enum {
  FP_OK = 0,
  FP_ERR_INVALID_ARG = 1,    /* bad pointer, size, option or face index */
  FP_ERR_NOT_SYMMETRIC = 2,  /* CSR pattern is not structurally symmetric */
  FP_ERR_OUT_OF_MEMORY = 3,  /* device allocation failed */
  FP_ERR_CUDA = 4,           /* a CUDA runtime call failed (handle poisoned) */
  FP_ERR_TIMEOUT = 5,        /* a bounded device wait ran out (handle poisoned) */
  FP_ERR_STATE = 6,          /* call order violated or handle poisoned */
  FP_ERR_UNSUPPORTED = 7     /* input beyond a documented size limit */
} fp_status;

typedef struct {
  int32_t patch_cap;       /* hard maximum patch size, >= 1 (default 512). The
                              seeding targets a mean of cap/2 ("target patch
                              size", Section 6). */
  int32_t lloyd_rounds;    /* Lloyd re-centring rounds, >= 0 (default 2) */
  uint64_t seed;           /* seeds the patch seeding hash (default 0) */
  int32_t nd_level;        /* nested-dissection depth (Section 4.2); 0 = ceil(log2 k),
                              which makes every leaf a single patch (default 0) */
  int32_t schedule;        /* 0 = post-order, 1 = level order (Section 5) */
  int32_t dof_per_vertex;  /* b >= 1: each vertex owns b consecutive unknowns
                              (Section 6.5); perm/etree/colcount are then
                              expanded to n*b entries (default 1) */
  int32_t debug_dump;      /* 0 or 1 (default 0). 1: fp_permute also keeps the
                              boundaries of its stages (seeds, labels after each
                              Lloyd round, the quotient graph, the sides and
                              moves of every dissection level) for
                              fp_get_stage; this adds device copies and one
                              host sync per patching round */
  int64_t max_spin;        /* >= 0 (default 0 = 2^24): how many times a bounded
                              device wait of the library polls before it gives
                              up. The only such wait is the tensor-core
                              completion wait of the learned-priority network
                              (fp_set_priority_net); when it runs out, the
                              kernel flags it, waits (2^24 polls at most) for
                              its tensor-core work in flight, frees its tensor
                              memory and returns, and the call returns
                              FP_ERR_TIMEOUT with the handle poisoned. The
                              grid-wide barriers of the cooperative kernels are
                              the CUDA runtime's (their co-residency is
                              guaranteed by the cooperative launch). */
} fp_options;

/* Fills *opts with the defaults above. */
void fp_default_options(fp_options* opts);

/*
 * Creates a handle from a triangle list (Section 2 / Section 4.1 step 2: G is
 * the graph of A without its diagonal; for a mesh Laplacian it is the mesh
 * adjacency). d_faces: int32 [n_faces][3] row-major, corners in
 * [0, n_vertices); a face with repeated corners contributes only its distinct
 * edges. Builds the symmetric, sorted, duplicate-free CSR of G on the device.
 * Errors: FP_ERR_INVALID_ARG (NULL out/opts, n_vertices < 0, n_faces < 0,
 * bad option, a corner out of range), FP_ERR_UNSUPPORTED (a vertex with more
 * than 4096 incident face-edges, or more than 2^31-1 adjacency entries),
 * FP_ERR_OUT_OF_MEMORY, FP_ERR_CUDA. Synchronises `stream` once (validation).
 */
fp_status fp_create_from_faces(const int32_t* d_faces, int64_t n_faces, int32_t n_vertices,
                               const fp_options* opts, void* stream, fp_handle** out);

/*
 * Creates a handle from a CSR pattern of A (Section 4.1 step 2): d_rowptr
 * [n_rows+1], d_col [rowptr[n_rows]] (int32, column order arbitrary,
 * duplicates allowed, diagonal ignored). With opts->dof_per_vertex = b > 1 the
 * pattern is the unknown-level pattern of n_rows = b*n unknowns and every
 * b x b block is merged into one vertex (Section 6.5): vertices u != v are
 * adjacent iff any entry of block (u, v) exists. The vertex graph must be
 * structurally symmetric. d_rowptr must start at 0 and not decrease (checked
 * first: FP_ERR_INVALID_ARG), and d_col must hold d_rowptr[n_rows] entries (the
 * caller's contract: a shorter buffer cannot be detected). Errors as
 * fp_create_from_faces, plus FP_ERR_NOT_SYMMETRIC, and FP_ERR_INVALID_ARG if
 * n_rows is not a multiple of b or an index is out of range. Synchronises
 * `stream` twice.
 */
fp_status fp_create_from_csr(const int32_t* d_rowptr, const int32_t* d_col, int32_t n_rows,
                             const fp_options* opts, void* stream, fp_handle** out);

/*
 * Computes the permutation (Algorithm 1 steps 1-4: patching, patch-guided
 * nested dissection over the quotient graph (Algorithm 2), local minimum-degree
 * orderings and their concatenation (Algorithm 3)). d_perm, d_iperm: int32
 * [n*b], caller-owned device buffers (either may be NULL to skip it).
 * Synchronises `stream` (the number of patches decides the tree depth).
 * Errors: FP_ERR_UNSUPPORTED (a tree node larger than 32768 vertices, which
 * happens only with a small nd_level or a huge patch_cap; or a patch with more
 * than 4096 edges to other patches, counted with multiplicity, which happens
 * only on graphs far denser than meshes), FP_ERR_OUT_OF_MEMORY, FP_ERR_CUDA,
 * FP_ERR_STATE.
 */
fp_status fp_permute(fp_handle* h, int32_t* d_perm, int32_t* d_iperm);

/*
 * Symbolic Cholesky of P (A) P^T for the last fp_permute: elimination-tree
 * parent[j] = min{ i > j : L_ij != 0 } (-1 for a root) and colcount[j] =
 * |{ i >= j : L_ij != 0 }|, both int32 [n*b] indexed by new position and
 * expanded to DOFs when b > 1 (Section 6.5). h_nnzL = sum of colcount,
 * h_flops = sum of colcount^2 (the O(sum d(i)^2) cost of Section 6.5); either
 * host pointer may be NULL. Any device pointer may be NULL to skip it.
 * Synchronises `stream`. Errors: FP_ERR_STATE (no fp_permute yet),
 * FP_ERR_OUT_OF_MEMORY, FP_ERR_CUDA.
 */
fp_status fp_symbolic(fp_handle* h, int32_t* d_parent, int32_t* d_colcount, int64_t* h_nnzL,
                      int64_t* h_flops);

/*
 * Stage boundaries of the last fp_permute, kept when the handle was created
 * with opts->debug_dump = 1 (for checking each step of Algorithm 1 against a
 * reference, not only the final permutation). `index` selects the Lloyd round
 * or dissection level; int32 arrays:
 *   FP_STAGE_SEEDS          (index 0)  seed vertex of every patch rank after
 *                                      the seeding and the unreached
 *                                      components (Section 4.1 step 1)
 *   FP_STAGE_LLOYD_SEEDS    (round r)  seed of every rank after Lloyd round r
 *   FP_STAGE_LABELS         (r = 0..R) patch of every vertex after the first
 *                                      labelling (r = 0) and after the
 *                                      relabelling of Lloyd round r (before
 *                                      the cap splits); the final map is
 *                                      fp_get_patches'
 *   FP_STAGE_QUOTIENT_WEIGHT, _ROWPTR, _COL, _EDGE_WEIGHT (index 0): the
 *                                      quotient graph of the final patches
 *                                      (Section 3 definition; Algorithm 2
 *                                      step 1): vertices per patch [k], CSR
 *                                      [k+1], neighbour patches and edge
 *                                      weights in increasing neighbour id
 *   FP_STAGE_SIDE           (depth d)  [k]: side (0 left, 1 right) each patch
 *                                      took in the node bisected at depth d
 *                                      (Algorithm 2 step 2), -1 if it took
 *                                      part in no bisection at depth d
 *   FP_STAGE_CHILD          (depth d)  [k]: the child node each patch moved to
 *                                      after depth d's separators (Algorithm 2
 *                                      step 5), -1 if it has no remaining
 *                                      vertex or was not bisected
 * d_out: caller-owned device buffer of `cap` ints (may be NULL to query the
 * length); *h_len receives the length. Stream-ordered, no sync.
 * Errors: FP_ERR_STATE (no fp_permute with debug_dump on, or the stage/index
 * was not recorded), FP_ERR_INVALID_ARG (cap below the length).
 */
typedef enum {
  FP_STAGE_SEEDS = 0,
  FP_STAGE_LLOYD_SEEDS = 1,
  FP_STAGE_LABELS = 2,
  FP_STAGE_QUOTIENT_WEIGHT = 3,
  FP_STAGE_QUOTIENT_ROWPTR = 4,
  FP_STAGE_QUOTIENT_COL = 5,
  FP_STAGE_QUOTIENT_EDGE_WEIGHT = 6,
  FP_STAGE_SIDE = 7,
  FP_STAGE_CHILD = 8
} fp_stage;

fp_status fp_get_stage(fp_handle* h, int32_t stage, int32_t index, int32_t* d_out, int64_t cap, int64_t* h_len);

/* Sizes of the handle: vertices n, DOFs per vertex b, nnz of G (2E). */
fp_status fp_get_sizes(const fp_handle* h, int32_t* h_n, int32_t* h_dof, int64_t* h_nnz);

/* Copies the CSR of the vertex graph G: d_rowptr [n+1], d_col [nnz]. */
fp_status fp_get_graph(fp_handle* h, int32_t* d_rowptr, int32_t* d_col);

/* After fp_permute: the group map (patch id per vertex, Section 4.1) into
 * d_gmap [n] (may be NULL) and the number of patches into *h_k. */
fp_status fp_get_patches(fp_handle* h, int32_t* d_gmap, int32_t* h_k);

/*
 * Supplies the patch partition instead of computing it (Section 4, opening:
 * with the patches given, the mesh is not needed). d_gmap: int32 [n], caller-
 * owned device buffer read during this call; d_gmap[v] in [0, k) is the group
 * of vertex v. Every later fp_permute on h skips the patching step
 * (Algorithm 1 step 1) and dissects over these groups: they need not be
 * connected nor bounded in size (tree nodes above 512 vertices use the
 * separator kernels; above 32768 fp_permute fails with FP_ERR_UNSUPPORTED),
 * and a label no vertex carries is an empty group that takes no part
 * (zero weight). patch_cap, seed and lloyd_rounds are then unused.
 * Errors: FP_ERR_INVALID_ARG (NULL map with n > 0, k < 1, a label outside
 * [0, k)), FP_ERR_OUT_OF_MEMORY, FP_ERR_STATE. Synchronises the stream.
 */
fp_status fp_set_patches(fp_handle* h, const int32_t* d_gmap, int32_t k);

/*
 * After fp_permute: the nested-dissection tree of Section 4.2 stored as a
 * binary tree in a 1-D array (children of node t are 2t+1 and 2t+2).
 * *h_depth = D; the tree has 2^(D+1)-1 nodes. d_node_begin / d_node_size
 * [2^(D+1)-1]: first position in perm and vertex count of each node (vertex
 * level, before DOF expansion). d_node_of [n]: the node of every vertex. Call
 * first with only h_depth to size the buffers; any pointer may be NULL.
 */
fp_status fp_get_tree(fp_handle* h, int32_t* h_depth, int32_t* d_node_begin, int32_t* d_node_size,
                      int32_t* d_node_of);

/*
 * One-shot host-buffer form (for callers without device buffers): copies
 * h_faces to the device, runs create + permute + symbolic on `stream`, copies
 * the results back and destroys the handle. h_perm/h_iperm/h_parent/
 * h_colcount [n*b] may each be NULL. Returns the first failing status.
 */
fp_status fp_order_faces_host(const int32_t* h_faces, int64_t n_faces, int32_t n_vertices,
                              const fp_options* opts, void* stream, int32_t* h_perm, int32_t* h_iperm,
                              int32_t* h_parent, int32_t* h_colcount, int64_t* h_nnzL, int64_t* h_flops);

/*
 * Batched ordering of many independent meshes (a library service; the paper
 * orders one mesh at a time). Each item is one mesh: device faces in, device
 * outputs (caller-owned, each may be NULL, DOF-expanded when
 * opts->dof_per_vertex > 1) and host results out. Every item's results equal
 * those of the single-mesh calls (create + permute + symbolic) on that mesh
 * with its chosen_cap.
 *
 * n_workers = 0 (fused): the batch is ordered as ONE graph, the disjoint union
 * of its meshes, by one pipeline whose every launch covers all meshes (each
 * mesh's dissection tree hangs below an empty super-tree; its cap, seed
 * threshold and tie hashes stay its own). Taken when opts has
 * dof_per_vertex 1, nd_level 0 and debug_dump 0 and the totals fit int32
 * (sum of n_vertices, 6 x sum of n_faces); otherwise, and when the fused
 * pipeline fails (an input error, out of memory), the items are ordered one
 * by one as below, so that each item gets its own status. The fused form
 * counts the batch's kernel launches on the first item (0 on the others).
 * n_workers = 1..64 (pool): the meshes are spread over that many host
 * threads, each with its own CUDA stream on the current device, which run
 * create + permute + symbolic + destroy for one mesh after another, largest
 * first (each item counts its own launches).
 *
 * The device faces must be complete before the call (it runs on streams of
 * its own). Synchronous: returns when every item is done. Returns FP_OK if
 * every item succeeded, else the first failing item's status (each item's own
 * status is in item->status). A patch_cap of 0 in an item selects the
 * autotuned cap of its size class (see fp_batch_autotune); item->chosen_cap
 * reports the cap used, so that a result can be reproduced with the
 * single-mesh calls.
 */
typedef struct {
  const int32_t* d_faces;   /* int32 [n_faces][3] on the device */
  int64_t n_faces;
  int32_t n_vertices;
  int32_t patch_cap;        /* > 0: this cap; 0: autotuned cap of the size class */
  int32_t* d_perm;          /* [n*b] outputs, device, may be NULL */
  int32_t* d_iperm;
  int32_t* d_parent;
  int32_t* d_colcount;
  int64_t nnzL;             /* out */
  int64_t flops;            /* out */
  int32_t chosen_cap;       /* out */
  int32_t status;           /* out: fp_status of this item */
  int64_t launches;         /* out: kernel launches issued for this item (fused: the batch's, on item 0) */
  int32_t learned_leaves;   /* out (fp_batch_order_learned): leaves considered */
  int32_t learned_kept;     /* out: leaves whose learned order was kept */
  int64_t fill_plain;       /* out: summed leaf fills under plain minimum degree */
  int64_t fill_chosen;      /* out: summed leaf fills of the chosen orders */
} fp_batch_item;

fp_status fp_batch_order(fp_batch_item* items, int32_t count, const fp_options* opts, int32_t n_workers);

/*
 * fp_batch_order with learned priorities: every mesh gets the network h_codes
 * (FP_GNN_NPARAMS codes, see fp_set_priority_net) attached before its
 * fp_permute, so each leaf keeps the lower-fill of its learned and plain
 * orders; the per-item learned_* and fill_* fields report the choices.
 * n_workers as in fp_batch_order (0: fused). h_codes NULL is fp_batch_order.
 * Errors as fp_batch_order, plus FP_ERR_INVALID_ARG for a code out of range.
 */
fp_status fp_batch_order_learned(fp_batch_item* items, int32_t count, const fp_options* opts, int32_t n_workers,
                                 const int32_t* h_codes);

/*
 * The fused batch as a handle (batch create / permute / symbolic, in three
 * calls; the paper has no batch form): fp_batch_create builds ONE handle
 * for the disjoint union of the items' meshes (device faces read on `stream`
 * during the call; patch caps as in fp_batch_order: item->patch_cap, or the
 * autotuned cap of its size class); fp_batch_permute orders it and writes
 * every item's d_perm / d_iperm (mesh-local numbering, each may be NULL) and
 * status, chosen_cap and, with a network attached by fp_set_priority_net,
 * the learned_* and fill_* fields; fp_batch_symbolic writes every item's
 * d_parent / d_colcount (indexed by the mesh's own positions, -1 for roots)
 * and nnzL, flops. item 0's `launches` counts the handle's launches so far.
 * `items` must be the array (and `count` its length) given to
 * fp_batch_create; only their output pointers may differ. The handle's
 * single-mesh calls see the union (fp_get_tree: the union's tree, with
 * every mesh's subtree below an empty super-tree; fp_permute: the union's
 * order); fp_destroy frees it. Synchronous (each call waits for its stream).
 * Errors: FP_ERR_INVALID_ARG (count < 1, NULL items or options, an item
 * with negative sizes or NULL faces, options other than dof_per_vertex 1,
 * nd_level 0 and debug_dump 0, totals beyond int32, a corner outside its
 * own mesh; permute/symbolic: not a batch handle of `count` items),
 * FP_ERR_STATE (symbolic before permute; a poisoned handle), and those of
 * fp_create_from_faces, fp_permute, fp_symbolic.
 */
fp_status fp_batch_create(const fp_batch_item* items, int32_t count, const fp_options* opts, void* stream,
                          fp_handle** out);
fp_status fp_batch_permute(fp_handle* h, fp_batch_item* items, int32_t count);
fp_status fp_batch_symbolic(fp_handle* h, fp_batch_item* items, int32_t count);

/*
 * Autotuner for fp_batch_order: one patch cap per size class of the items
 * (vertex counts below 8k, 32k, 128k, 512k, and above), from the candidates
 * {128, 256, 384, 512}. When the batch qualifies for the fused form (see
 * fp_batch_order) the caps are tuned on the fused batch itself: each
 * candidate for every class at once, keeping the fastest whose total nnz(L)
 * is within 5% of the least seen, then each class in turn with the other
 * candidates, a change kept when faster at that fill (best of two runs,
 * items with their own patch_cap keep it; no output is written). Otherwise
 * each class's largest item is ordered alone once per candidate, timing
 * create + permute + symbolic with CUDA events (best of two), and the
 * fastest cap whose nnz(L) is within 5% of the smallest nnz(L) seen for that
 * item is kept. The choices are kept process-wide and used by items with
 * patch_cap 0; h_caps (may be NULL) receives the 5 chosen caps (0 for an
 * empty class).
 */
fp_status fp_batch_autotune(fp_batch_item* items, int32_t count, const fp_options* opts, int32_t* h_caps);

/*
 * Allocation-free CSR assembly. The paper has no counterpart: this is a
 * library service for callers that cannot allocate device memory when they
 * build the graph (for example a process whose device memory is entirely
 * reserved by another framework's caching allocator, or a latency-critical
 * loop that must stay out of the CUDA allocator). It computes exactly the
 * CSR that fp_create_from_faces + fp_get_graph produce (G = graph of the face
 * list without diagonal, rows sorted and duplicate-free) into caller buffers:
 * d_rowptr [n_vertices+1] and d_col [col_cap]; *h_nnz (may be NULL) receives
 * rowptr[n_vertices]. All intermediate data live in one fixed scratch array
 * compiled into the library (about 4.5 MB of device memory, held by every GPU
 * that loads the library until the process exits); the call never allocates.
 * Limits: n_vertices <= 65536, n_faces <= 131072, and at most 256 face-edge
 * entries per vertex (FP_ERR_UNSUPPORTED beyond, with a message in
 * fp_last_error(NULL)). FP_ERR_INVALID_ARG for NULL pointers, negative sizes,
 * a corner out of range, or col_cap smaller than the number of entries.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) and keeps it for the process; make that first call
 * before any stream capture. The kept address does not survive a reset of the
 * device's primary context (cudaDeviceReset): do not call this entry point
 * after one.
 * Every call on a device shares the one scratch array: calls that may overlap
 * on the GPU (other streams, other host threads) race and must be serialised
 * by the caller. Synchronises `stream`.
 */
fp_status fp_graph_from_faces_static(const int32_t* d_faces, int64_t n_faces, int32_t n_vertices,
                                     int32_t* d_rowptr, int32_t* d_col, int64_t col_cap, int64_t* h_nnz,
                                     void* stream);

/* ---- numeric factorisation driven by the permutation ----------------------------
 *
 * The paper's purpose for the permutation is a sparse Cholesky solver
 * (Section 6: the permutation and its elimination tree are handed to cuDSS or
 * MKL). These calls factor and solve on the GPU with the handle's ordering:
 * a multifrontal Cholesky with one dense front per tree node of Section 4.2
 * (the node's columns plus the ancestor rows its subtree reaches), FP64.
 * Scalar matrices only (dof_per_vertex = 1).
 */

/*
 * Numeric Cholesky L L^T = P A P^T after fp_permute. A is symmetric positive
 * definite with the pattern of the handle's graph plus the diagonal:
 * d_diag [n] its diagonal by vertex, d_offdiag [nnz] its off-diagonal values
 * aligned with the CSR that fp_get_graph returns (entry e of row v is
 * A[v, col[e]]; both triangles, equal values). Device buffers, read during the
 * call. The factor stays in the handle until the next fp_permute or
 * fp_destroy. Synchronises the stream. Errors: FP_ERR_STATE (no fp_permute),
 * FP_ERR_UNSUPPORTED (dof_per_vertex > 1, or a front beyond the kernels'
 * limits: a node with more than 1.6M ancestor columns or an update matrix
 * above 51,200 rows), FP_ERR_INVALID_ARG (NULL values with n > 0, or a pivot
 * that is not positive: A is not positive definite), FP_ERR_OUT_OF_MEMORY.
 */
fp_status fp_factor(fp_handle* h, const double* d_diag, const double* d_offdiag);

/*
 * Solves A x = b with the factor of fp_factor: d_b [n] by vertex (read),
 * d_x [n] by vertex (written; may equal d_b). Stream-ordered, no sync.
 * Errors: FP_ERR_STATE (no factor), FP_ERR_INVALID_ARG, FP_ERR_OUT_OF_MEMORY.
 */
fp_status fp_solve(fp_handle* h, const double* d_b, double* d_x);

/*
 * The factor in compressed columns indexed by new position: d_colptr [n+1]
 * (int64), d_rows / d_vals [*h_nnz] (rows ascending, the diagonal first). The
 * rows of column j are those of its front: every later position of j's tree
 * node (where L is structurally zero the value is exactly 0.0) and the
 * ancestor rows of the node's front. Call with NULL buffers to get *h_nnz.
 * Synchronises the stream. Errors: FP_ERR_STATE (no factor),
 * FP_ERR_INVALID_ARG (cap below *h_nnz).
 */
fp_status fp_factor_export(fp_handle* h, int64_t* d_colptr, int32_t* d_rows, double* d_vals, int64_t cap,
                           int64_t* h_nnz);

/* Sizes of the factor: doubles held by the fronts, flops of their partial
 * factorisations, and entries of L as stored (each may be NULL). */
fp_status fp_factor_stats(const fp_handle* h, int64_t* h_front_doubles, int64_t* h_flops, int64_t* h_nnz);

/* Releases the handle and its workspace (stream-ordered). NULL is a no-op. */
fp_status fp_destroy(fp_handle* h);

/* Message of the last failure on h (or of the last failed create when h is
 * NULL); never NULL. Valid until the next call on the same handle. */
const char* fp_last_error(const fp_handle* h);

/* Static name of a status code. */
const char* fp_status_string(fp_status s);

/* Number of kernel launches the library issued on this handle so far. */
int64_t fp_launch_count(const fp_handle* h);

/*
 * Stage profiling (process-wide, off by default). While on, every handle
 * records a CUDA event pair around each stage's launches on the stream the
 * stage runs on; fp_profile_read() waits for those events and returns, per
 * stage kind, the summed GPU milliseconds (ms[kind]) and the number of event
 * pairs (launches[kind]); it returns FP_PROF_COUNT. Either output may be NULL;
 * `cap` bounds how many kinds are written. fp_profile_reset() discards the
 * totals. The paper reports the same breakdown (patching, separators, etree,
 * local ordering) in its patch-size study (Section 6.6).
 */
typedef enum {
  FP_PROF_GRAPH = 0,       /* a1 CSR assembly */
  FP_PROF_PATCH_BFS,       /* a2 Voronoi searches over the whole mesh (k_bfs) */
  FP_PROF_PATCH_OTHER,     /* a2 seeds, Lloyd picks, splits */
  FP_PROF_QUOTIENT,        /* a3 quotient graph */
  FP_PROF_ND_BISECT,       /* a4 bisection of the quotient graph */
  FP_PROF_ND_SEPARATOR,    /* a4 superset, refinement, weight update */
  FP_PROF_LAYOUT,          /* a6 tree layout and vertex lists */
  FP_PROF_MD_SMALL,        /* a5 minimum degree, nodes <= 512 vertices */
  FP_PROF_MD_MID,          /* a5 minimum degree, nodes <= 1344 vertices */
  FP_PROF_MD_LARGE,        /* a5 minimum degree, larger nodes */
  FP_PROF_PERM,            /* a6/a8 inverse permutation and DOF expansion */
  FP_PROF_SYMBOLIC,        /* a7 etree and column counts */
  FP_PROF_LEARNED,         /* a10 network scores, keyed orders, fill choice */
  FP_PROF_TRAIN,           /* a10 training samples and gradient steps */
  FP_PROF_PATCH_LOCAL,     /* a2 searches inside patches (Lloyd depth, splits) */
  FP_PROF_JOIN_WAIT,       /* time the handle's stream waits, after its own
                              leaf orderings, for the separator orderings that
                              run on the auxiliary streams (the part of them on
                              the critical path) */
  FP_PROF_NUMERIC,         /* numeric factorisation and solves (fp_factor, fp_solve) */
  FP_PROF_COUNT
} fp_prof_kind;

void fp_profiling(int on);
int fp_profile_read(double* ms, int64_t* launches, int cap);
void fp_profile_reset(void);

/* ---- a10 learned elimination priorities ---------------------------------------
 *
 * The paper orders every patch by (approximate) minimum degree and says
 * nothing about learned orderings. This part adds, per leaf of the tree (a
 * node with vertices and no non-empty descendant, at most 512 vertices), a
 * second candidate: exact minimum degree whose ties between equal degrees go
 * to the vertex with the higher network score (then the smaller id). The
 * candidate is kept iff its exact fill -- the sum of the leaf columns' counts
 * in L -- is smaller than plain minimum degree's. A leaf's column counts
 * depend on its own order only, so nnz(L) never exceeds the plain method's.
 *
 * The network: per leaf vertex, 6 integer feature codes (value code/64):
 * degree in the leaf/8, degree in G/8, has a neighbour outside the leaf,
 * hop depth from that boundary/(max depth+1), leaf size/patch_cap, 1. Two
 * layers h' = ReLU(Ws h + Wn mean_{u in leaf neighbours} h_u + b) of width 32
 * and a head S = w.h + c. Codes: weights value q/128 (|q| <= 255), biases and
 * c value q/8192 (|q| <= 2^20), activations value q/64 (q in [0, 255], the
 * layer output rounded to nearest even and clamped). All dot products are
 * exact integers, computed on BF16 tensor cores with FP32 accumulation.
 *
 * Parameter layout, FP_GNN_NPARAMS entries (int32 codes or float weights):
 * w1s[32][6] w1n[32][6] b1[32] w2s[32][32] w2n[32][32] b2[32] w3[32] c.
 */
#define FP_GNN_NPARAMS 2529

/*
 * Attaches a network (h_codes: host array of FP_GNN_NPARAMS codes, copied) to
 * the handle; every later fp_permute then runs the learned choice after the
 * plain ordering. NULL detaches it. Errors: FP_ERR_INVALID_ARG (a code out of
 * its range), FP_ERR_OUT_OF_MEMORY.
 */
fp_status fp_set_priority_net(fp_handle* h, const int32_t* h_codes);

/* After fp_permute with a network attached: leaves considered, leaves whose
 * learned order was kept, and the summed fills of those leaves under plain
 * minimum degree and under the chosen orders. Any pointer may be NULL. */
fp_status fp_learned_stats(const fp_handle* h, int32_t* h_leaves, int32_t* h_kept, int64_t* h_fill_plain,
                           int64_t* h_fill_chosen);

/*
 * After fp_permute: the network's scores S (int32 [n], indexed by position
 * in perm; 0 off the leaves) and feature codes (uint8 [n][8], 6 used) of the
 * leaf vertices under the current permutation, for codes h_codes (host).
 * Either output may be NULL. Synchronises the stream.
 */
fp_status fp_gnn_scores(fp_handle* h, const int32_t* h_codes, int32_t* d_scores, uint8_t* d_features);

/*
 * Training sample of the last fp_permute (call it without a network): for
 * every position p of perm (n entries), d_x [n][8] uint8 feature codes,
 * d_mask [n] uint8 (1 on leaf positions), d_target [n] float, d_rank [n]
 * int32 (may be NULL), and the within-leaf neighbour positions as CSR
 * d_lrowptr [n+1], d_lcol [lcol_cap] (*h_lnnz entries used). The target of a
 * leaf vertex at rank k of its leaf's best order among plain minimum degree
 * and n_seeds minimum-degree orders with seeded tie-break keys (the high 32
 * bits of SplitMix64 at state r*0x9E3779B97F4A7C15 + v, r = 1..n_seeds;
 * lowest fill wins, ties to the lower r) is (m-1-k)/(m-1) for an m-vertex
 * leaf (1 when m = 1). Errors: FP_ERR_STATE (no fp_permute, or a network
 * attached), FP_ERR_INVALID_ARG (n_seeds outside 0..64, lcol_cap too small:
 * *h_lnnz then holds the size needed).
 */
fp_status fp_gnn_sample(fp_handle* h, int32_t n_seeds, uint8_t* d_x, uint8_t* d_mask, float* d_target,
                        int32_t* d_rank, int32_t* d_lrowptr, int32_t* d_lcol, int64_t lcol_cap, int64_t* h_lnnz);

/* Device scratch bytes fp_gnn_train_step needs for n positions. */
int64_t fp_gnn_train_work_bytes(int32_t n);

/*
 * One gradient-descent step of the float network (same structure, no grid:
 * activations clamped to [0, 255/64]) on a sample: loss = mean squared error
 * between the score s and the target over mask positions; d_grad receives
 * the gradient (FP_GNN_NPARAMS floats), d_params is updated in place by
 * params -= lr * grad (lr = 0: gradient only), *d_loss the loss before the
 * step. All pointers are device pointers; d_work holds
 * fp_gnn_train_work_bytes(n) bytes. Deterministic: every reduction has a
 * fixed order. Runs on `stream`; does not synchronise.
 */
fp_status fp_gnn_train_step(float* d_params, float* d_grad, const uint8_t* d_x, const uint8_t* d_mask,
                            const float* d_target, const int32_t* d_lrowptr, const int32_t* d_lcol, int32_t n,
                            float lr, float* d_loss, void* d_work, int64_t work_bytes, void* stream);

/* Float weights -> codes (round to nearest, clamped to the code ranges). */
fp_status fp_gnn_quantise(const float* d_params, int32_t* d_codes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FASTPERM_H */
