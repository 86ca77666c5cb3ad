// a2 Patching (Section 4.1 step 1; Algorithm 1 GetPatches). The paper calls
// RXMesh's GPU Lloyd patcher; this library grows patches itself:
//   seeds  : v is a seed iff (h(v) >> 32) * n < k_target * 2^32, h = SplitMix64
//            at state seed*gamma + v, k_target = max(1, ceil(2n / cap));
//            ranked by vertex id.
//   labels : multi-source BFS; a vertex first reached at level d takes the
//            smallest rank among its level-(d-1) neighbours, i.e. atomicMin
//            on the packed key (d << 32 | rank).
//   unreached components get their smallest vertex as a new seed;
//   Lloyd  : R rounds of "re-seed at the vertex deepest from the patch boundary
//            (ties: lowest id), relabel";
//   cap    : every patch above cap gets a second seed at its vertex farthest
//            from its seed (ties: lowest id), ranked after all existing ranks in
//            parent-rank order, and is relabelled from its two seeds.
// Searches over the whole mesh (Voronoi labelling) are one persistent
// cooperative launch each: the level loop runs on the device with a grid
// barrier between levels, frontier queues compacted with an atomic counter.
// Searches confined to one patch (Lloyd depth, cap splits) run one CTA per
// patch with the patch's adjacency in shared memory and CTA barriers only.
#include <cooperative_groups.h>

#include <type_traits>
#include <utility>

#include "fp_device.cuh"

namespace cg = cooperative_groups;

namespace fp {
namespace {

constexpr int BFS_THREADS = 256;
constexpr int BFS_BATCH = 8;
constexpr int BFS_TAIL = 1024;   // frontiers up to this size run in one CTA
// frontiers above this size (only a batch's union reaches it) read the
// neighbours' keys before claiming: a neighbour settled at an earlier level
// needs no atomic (about half of them on a mesh), which pays where the level
// is bound by atomic throughput rather than by its round trips
constexpr int32_t BFS_PRECHECK_MIN = 1 << 18;

// Level-synchronous multi-source BFS on packed keys (dist << 32 | label).
// ctr[0] holds the size of the initial frontier `fa`. Frontier entries are
// (vertex, first edge, end edge, 0), so that a level's first round trip
// brings the edge range along with the vertex. On exit key[] holds the
// distance and the minimum label for every reached vertex.
__global__ void __launch_bounds__(BFS_THREADS, 2) k_bfs(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                                     unsigned long long* key, int4* fa, int4* fb, int32_t* ctr) {
  FP_PDL_WAIT();
  cg::grid_group grid = cg::this_grid();
  // the tail's frontiers and counters (CTA 0 only): entries past BFS_TAIL
  // spill to the global queues at the same index
  __shared__ int4 s_fr[2][BFS_TAIL];
  __shared__ int32_t s_ctr[3];
  int4* cur = fa;
  int4* nxt = fb;
  int sel = 0;
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  // one level: every frontier vertex claims its unsettled neighbours. The
  // sweep is warp-uniform (every lane of a warp runs the same number of
  // batches), so a batch's claims are appended with one atomicAdd per warp
  // (offsets by bit-plane ballots); up to BFS_BATCH neighbours are loaded
  // per round. Round trips per level: the entry; its label and neighbours;
  // the claims (atomicMin returns the old key: a vertex settled at an
  // earlier level keeps it, and only the first claim of a vertex moves it to
  // the next frontier); the queue slots, with the claimed vertices' edge
  // ranges loaded meanwhile. In the tail (kTail) the entries and the
  // counter are in shared memory, which leaves the label, neighbour, claim
  // and edge-range round trips.
  auto sweep = [&](auto tail_tag, uint32_t level, int32_t ncur, int64_t first, int64_t stride) {
    constexpr bool kTail = decltype(tail_tag)::value;
    const unsigned long long dnext = (unsigned long long)(level + 1) << 32;
    const bool pre = !kTail && ncur > BFS_PRECHECK_MIN;
    int4* scur = s_fr[sel];
    int4* snxt = s_fr[sel ^ 1];
    int32_t* cnt = kTail ? s_ctr : ctr;
    for (int64_t i0 = first - lane; i0 < ncur; i0 += stride) {
      const int64_t i = i0 + lane;
      int32_t u = 0, e = 0, e1 = 0;
      if (i < ncur) {
        const int4 q = (kTail && i < BFS_TAIL) ? scur[i] : __ldcg(&cur[i]);
        u = q.x;
        e = q.y;
        e1 = q.z;
      }
      const unsigned long long lab = i < ncur ? (__ldcg(&key[u]) & 0xffffffffull) : 0ull;
      while (__any_sync(0xffffffffu, e < e1)) {
        int32_t v[BFS_BATCH];
        unsigned long long old[BFS_BATCH];
#pragma unroll
        for (int k = 0; k < BFS_BATCH; ++k) v[k] = e + k < e1 ? col[e + k] : -1;
        if (pre) {
          // settled at a level <= this one: its key cannot change
#pragma unroll
          for (int k = 0; k < BFS_BATCH; ++k) old[k] = v[k] >= 0 ? __ldcg(&key[v[k]]) : 0ull;
#pragma unroll
          for (int k = 0; k < BFS_BATCH; ++k)
            if (v[k] >= 0 && old[k] < dnext) v[k] = -1;
        }
#pragma unroll
        for (int k = 0; k < BFS_BATCH; ++k) old[k] = v[k] >= 0 ? atomicMin(&key[v[k]], dnext | lab) : 0ull;
        uint32_t claim = 0;
#pragma unroll
        for (int k = 0; k < BFS_BATCH; ++k)
          if (old[k] == KEY_INF) claim |= 1u << k;      // first claim: goes to the next frontier
        int32_t rb[BFS_BATCH], re[BFS_BATCH];
#pragma unroll
        for (int k = 0; k < BFS_BATCH; ++k) {
          rb[k] = (claim >> k & 1u) ? rowptr[v[k]] : 0;
          re[k] = (claim >> k & 1u) ? rowptr[v[k] + 1] : 0;
        }
        const int32_t c = __popc(claim);
        int32_t ex = 0, tot = 0;
#pragma unroll
        for (int bp = 0; bp < 4; ++bp) {      // c <= BFS_BATCH = 8: four bit planes
          const unsigned bb = __ballot_sync(0xffffffffu, (c >> bp) & 1);
          ex += __popc(bb & lt) << bp;
          tot += __popc(bb) << bp;
        }
        int32_t base = 0;
        if (lane == 0 && tot) base = atomicAdd(&cnt[(level + 1) % 3], tot);
        base = __shfl_sync(0xffffffffu, base, 0) + ex;
#pragma unroll
        for (int k = 0; k < BFS_BATCH; ++k)
          if (claim >> k & 1u) {
            const int4 q = make_int4(v[k], rb[k], re[k], 0);
            if (kTail && base < BFS_TAIL) snxt[base] = q;
            else nxt[base] = q;
            ++base;
          }
        e += BFS_BATCH;
      }
    }
  };
  static_assert(BFS_BATCH <= 15, "claim counts must fit four bit planes");
  uint32_t level = 0;
  int32_t nprev = 0;
  int32_t ncur = 0;
  for (;; ++level) {
    ncur = __ldcg(&ctr[level % 3]);
    if (ncur == 0) return;
    // the frontier grows from the seeds, peaks and dies out: the shrinking
    // tail goes to one CTA (the same decision in every CTA)
    if (ncur <= BFS_TAIL && ncur < nprev) break;
    nprev = ncur;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr[(level + 2) % 3] = 0;
    sweep(std::integral_constant<bool, false>{}, level, ncur, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
          (int64_t)gridDim.x * blockDim.x);
    int4* t = cur; cur = nxt; nxt = t;
    grid.sync();
  }
  // small frontiers (the last levels): CTA 0 alone, with CTA barriers instead
  // of grid barriers; the frontier (ncur <= BFS_TAIL entries) moves to
  // shared memory
  if (blockIdx.x != 0) return;
  for (int32_t i = threadIdx.x; i < ncur; i += blockDim.x) s_fr[0][i] = __ldcg(&cur[i]);
  if (threadIdx.x == 0) {
    s_ctr[level % 3] = ncur;
    s_ctr[(level + 1) % 3] = 0;
  }
  __syncthreads();
  for (;; ++level) {
    ncur = s_ctr[level % 3];
    if (ncur == 0) return;
    if (threadIdx.x == 0) s_ctr[(level + 2) % 3] = 0;
    sweep(std::integral_constant<bool, true>{}, level, ncur, threadIdx.x, blockDim.x);
    int4* t = cur; cur = nxt; nxt = t;
    sel ^= 1;
    __syncthreads();
  }
}

// In a fused batch every vertex draws with its number, vertex count and
// k_target inside its own mesh.
__global__ void k_seed_flags(int32_t n, uint64_t kt, uint64_t seed, int32_t* __restrict__ flag, SegView sv) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int32_t lv = v;
    uint64_t nm = (uint64_t)n, ktm = kt;
    if (sv.vmesh) {
      const int32_t m = sv.vmesh[v], b = sv.voff[m];
      const uint64_t c = (uint64_t)sv.mcap[m];
      lv = v - b;
      nm = (uint64_t)(sv.voff[m + 1] - b);
      ktm = (2 * nm + c - 1) / c;
      if (ktm < 1) ktm = 1;
    }
    uint64_t h = splitmix64_state(seed * 0x9E3779B97F4A7C15ull + (uint64_t)(uint32_t)lv);
    flag[v] = ((h >> 32) * nm) < (ktm << 32) ? 1 : 0;
  }
}

// Seeds (flag[v] = 1) with rank = base + rank[v] become BFS sources.
__global__ void k_seed_sources(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ flag,
                               const int32_t* __restrict__ rank, int32_t base, unsigned long long* __restrict__ key,
                               int32_t* __restrict__ seed_of, int4* __restrict__ frontier, int32_t* ctr) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    if (flag[v]) {
      int32_t r = rank[v];
      key[v] = (unsigned long long)(uint32_t)(base + r);
      seed_of[base + r] = v;
      frontier[r] = make_int4(v, rowptr[v], rowptr[v + 1], 0);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctr[0] = rank[n];
    ctr[1] = 0;
    ctr[2] = 0;
  }
}

__global__ void k_fill_u64(unsigned long long* p, unsigned long long v, int64_t n) {
  FP_PDL_WAIT();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void k_labels_of(const unsigned long long* __restrict__ key, int32_t n, int32_t* __restrict__ label) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    label[v] = key[v] == KEY_INF ? -1 : (int32_t)(uint32_t)key[v];
}

// Labels of every vertex (all reached) and, per patch, its vertex count and
// the sum of its vertices' degrees (counts zeroed by the caller).
__global__ void k_labels_counts(const unsigned long long* __restrict__ key, const int32_t* __restrict__ rowptr,
                                int32_t n, int32_t* __restrict__ label, int32_t* __restrict__ pcnt,
                                int32_t* __restrict__ pdeg) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int32_t p = (int32_t)(uint32_t)key[v];
    label[v] = p;
    atomicAdd(&pcnt[p], 1);
    atomicAdd(&pdeg[p], rowptr[v + 1] - rowptr[v]);
  }
}

__global__ void k_zero2(int32_t* __restrict__ a, int32_t* __restrict__ b, int64_t n) {
  FP_PDL_WAIT();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    a[i] = 0;
    b[i] = 0;
  }
}

__global__ void k_count_unreached(const unsigned long long* __restrict__ key, int32_t n, int32_t* cnt) {
  FP_PDL_WAIT();
  int32_t c = 0;
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) c += key[v] == KEY_INF;
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

// Smallest vertex id of every connected component of the unreached vertices
// (label propagation with pointer jumping, one cooperative launch; at most n
// rounds, each strictly lowering some comp value until the fixed point).
__global__ void __launch_bounds__(BFS_THREADS) k_unreached_components(const int32_t* __restrict__ rowptr,
                                                                      const int32_t* __restrict__ col,
                                                                      const unsigned long long* __restrict__ key,
                                                                      int32_t n, int32_t* comp, int32_t* flags) {
  FP_PDL_WAIT();
  cg::grid_group grid = cg::this_grid();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t v = t0; v < n; v += stride) comp[v] = key[v] == KEY_INF ? (int32_t)v : -1;
  if (t0 == 0) { flags[0] = 0; flags[1] = 0; flags[2] = 0; }
  grid.sync();
  for (int32_t round = 0; round < n; ++round) {
    if (t0 == 0) flags[(round + 1) % 3] = 0;
    bool changed = false;
    for (int64_t v = t0; v < n; v += stride) {
      int32_t c = __ldcg(&comp[v]);
      if (c < 0) continue;
      int32_t m = c;
      for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
        int32_t cu = __ldcg(&comp[col[e]]);
        if (cu >= 0 && cu < m) m = cu;
      }
      int32_t cc = __ldcg(&comp[m]);     // pointer jump
      if (cc >= 0 && cc < m) m = cc;
      if (m < c) { atomicMin(&comp[v], m); changed = true; }
    }
    if (changed) flags[round % 3] = 1;
    grid.sync();
    if (__ldcg(&flags[round % 3]) == 0) break;
    grid.sync();
  }
}

__global__ void k_component_seed_flags(const int32_t* __restrict__ comp, int32_t n, int32_t* __restrict__ flag) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    flag[v] = comp[v] == v ? 1 : 0;
}

__global__ void k_lloyd_apply(const unsigned long long* __restrict__ best, int32_t k, int32_t* __restrict__ seed_of) {
  FP_PDL_WAIT();
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x)
    if (best[p]) seed_of[p] = (int32_t)(0xffffffffu - (uint32_t)best[p]);
}

// All k seeds become sources with their own rank.
__global__ void k_all_seed_sources(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ seed_of, int32_t k,
                                   unsigned long long* __restrict__ key, int4* __restrict__ frontier, int32_t* ctr) {
  FP_PDL_WAIT();
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x) {
    const int32_t v = seed_of[p];
    key[v] = (unsigned long long)(uint32_t)p;
    frontier[p] = make_int4(v, rowptr[v], rowptr[v + 1], 0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) { ctr[0] = k; ctr[1] = 0; ctr[2] = 0; }
}

__global__ void k_oversize_flags(const int32_t* __restrict__ psize, int32_t k, int32_t cap, int32_t* __restrict__ over,
                                 const int32_t* __restrict__ seed_of, SegView sv) {
  FP_PDL_WAIT();
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x)
    over[p] = psize[p] > (sv.vmesh ? sv.mcap[sv.vmesh[seed_of[p]]] : cap);
}

// Cap split: the farthest vertex of every oversize patch p becomes the seed of
// the new rank kbase + orank[p].
__global__ void k_split_seeds(const unsigned long long* __restrict__ best, const int32_t* __restrict__ over,
                              const int32_t* __restrict__ orank, int32_t kbase, int32_t* __restrict__ seed_of) {
  FP_PDL_WAIT();
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < kbase; p += gridDim.x * blockDim.x)
    if (over[p]) seed_of[kbase + orank[p]] = (int32_t)(0xffffffffu - (uint32_t)best[p]);
}

// ---- searches inside one patch: one CTA per patch, no grid barrier ---------------
//
// mode 0 (Lloyd): hop depth from the patch boundary; best[p] = max (depth, -v).
// mode 1 (cap)  : hop distance from the seed; best[p] = max (dist, -v).
// mode 2 (cap)  : two-seed Voronoi inside the patch (seed with rank p, far vertex
//                 with rank kbase + orank[p]); writes key[v] = dist << 32 | rank.
// Modes 1 and 2 only visit patches with over[p] set. A patch's vertices, its
// internal adjacency (local ids) and the BFS state live in shared memory when
// the patch has at most LOCAL_SMEM_V vertices and LOCAL_SMEM_E internal
// adjacency entries, otherwise in global scratch at the patch's offsets.
constexpr int LOCAL_THREADS = 256;
constexpr int LOCAL_SMEM_V = 1024;
constexpr int LOCAL_SMEM_E = 8192;
constexpr int PL_SLOTS = 8;      // neighbour slots a frontier vertex gets in the pair sweep

struct LocalArgs {
  int32_t k;
  const int32_t* rowptr;
  const int32_t* col;
  const int32_t* label;         // current patch of every vertex
  const int32_t* pstart;        // [k+1] vertex lists by patch
  const int32_t* pverts;
  const int32_t* pedge;         // [k+1] adjacency offsets by patch (sum of degrees)
  int32_t* g_adj;               // global fallback: internal adjacency
  int32_t* g_vtx;               // global fallback: [4n + k] (lrow, dist, fa, fb per patch)
  int32_t* loc;                 // [n] local index of a vertex in its patch
  const int32_t* over;          // modes 1, 2: patches to process
  const int32_t* orank;
  int32_t kbase;
  const int32_t* seed_of;
  unsigned long long* best;     // modes 0, 1
  unsigned long long* key;      // mode 2
  int32_t* next_over;           // mode 2: the halves still above cap (flag by new patch id)
  int32_t* next_cnt;            // mode 2: how many
  int32_t cap;
  SegView sv;                   // fused batch: the cap of the patch's own mesh
};

// Mode 0 visits every patch: five CTAs per SM keep one wave for a mesh of
// ~700 patches; modes 1 and 2 run on the few oversize patches only and may
// use more registers (four CTAs per SM) instead of spilling.
template <int kMode>
__global__ void __launch_bounds__(LOCAL_THREADS, kMode == 0 ? 5 : 4) k_patch_local(LocalArgs a) {
  FP_PDL_WAIT();
  __shared__ int32_t s_verts[LOCAL_SMEM_V];
  __shared__ int32_t s_lrow[LOCAL_SMEM_V + 1];
  __shared__ uint32_t s_dist[LOCAL_SMEM_V];
  __shared__ int32_t s_fa[LOCAL_SMEM_V];
  __shared__ int32_t s_fb[LOCAL_SMEM_V];
  __shared__ uint16_t s_adj[LOCAL_SMEM_E];
  __shared__ int32_t red[40];
  __shared__ unsigned long long red64[40];
  __shared__ int32_t s_cnt[3];
  __shared__ int32_t s_long;     // some vertex has more than PL_SLOTS internal neighbours
  const int tid = threadIdx.x;
  for (int32_t p = blockIdx.x; p < a.k; p += gridDim.x) {
    if (kMode != 0 && !a.over[p]) continue;
    const int32_t v0 = a.pstart[p], m = a.pstart[p + 1] - v0;
    const int32_t e0 = a.pedge[p], eall = a.pedge[p + 1] - e0;
    const bool small = m <= LOCAL_SMEM_V && eall <= LOCAL_SMEM_E;
    const int32_t* verts = small ? s_verts : a.pverts + v0;
    int32_t* gv = a.g_vtx + 4 * (int64_t)v0 + p;          // 4m + 1 ints of this patch
    int32_t* lrow = small ? s_lrow : gv;
    uint32_t* dist = small ? s_dist : (uint32_t*)(gv + m + 1);
    int32_t* fa = small ? s_fa : gv + 2 * m + 1;
    int32_t* fb = small ? s_fb : gv + 3 * m + 1;
    if (tid == 0) s_long = 0;
    for (int32_t i = tid; i < m; i += LOCAL_THREADS) {
      const int32_t v = a.pverts[v0 + i];
      if (small) s_verts[i] = v;
      a.loc[v] = i;
    }
    __syncthreads();
    // internal adjacency as a local CSR: one gather of every vertex's
    // neighbours' patches gives its internal degree and (mode 0) whether it
    // lies on the patch boundary, the BFS sources of that mode
    int32_t carry = 0;
    for (int32_t i0 = 0; i0 < m; i0 += LOCAL_THREADS) {
      const int32_t i = i0 + tid;
      int32_t c = 0;
      bool bnd = false;
      if (i < m)
        for_row_gather<8>(a.rowptr, a.col, verts[i], a.label, [&](int32_t, int32_t lu) {
          if (lu == p) ++c;
          else bnd = true;
        });
      if (c > PL_SLOTS) s_long = 1;
      int32_t tot;
      const int32_t ex = block_excl_scan_i32(c, &tot, red);
      if (i < m) {
        lrow[i] = carry + ex;
        dist[i] = (kMode == 0 && bnd) ? 0u : 0xffffffffu;
      }
      carry += tot;
    }
    if (tid == 0) lrow[m] = carry;
    __syncthreads();
    // rows: eight neighbours a round (ids, then their patch, then the local
    // index of the internal ones)
    for (int32_t i = tid; i < m; i += LOCAL_THREADS) {
      int32_t o = lrow[i];
      const int32_t v = verts[i];
      const int32_t ee = a.rowptr[v + 1];
      for (int32_t eb = a.rowptr[v]; eb < ee; eb += 8) {
        int32_t u[8], j[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) u[k] = eb + k < ee ? a.col[eb + k] : -1;
#pragma unroll
        for (int k = 0; k < 8; ++k) j[k] = u[k] >= 0 ? a.label[u[k]] : -1;
#pragma unroll
        for (int k = 0; k < 8; ++k) j[k] = j[k] == p ? a.loc[u[k]] : -1;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (j[k] >= 0) {
            if (small) s_adj[o++] = (uint16_t)j[k]; else a.g_adj[e0 + o++] = j[k];
          }
      }
    }
    // sources; the BFS counts level L's frontier in s_cnt[L % 3]
    if (tid == 0) {
      s_cnt[0] = 0;
      s_cnt[1] = 0;
      s_cnt[2] = 0;
    }
    __syncthreads();
    if (kMode == 0) {
      for (int32_t i = tid; i < m; i += LOCAL_THREADS)
        if (dist[i] == 0u) fa[atomicAdd(&s_cnt[0], 1)] = i;
    } else if (tid == 0) {
      const int32_t i = a.loc[a.seed_of[p]];
      dist[i] = 0u;
      fa[0] = i;
      s_cnt[0] = 1;
      if (kMode == 2) {
        const int32_t j = a.loc[a.seed_of[a.kbase + a.orank[p]]];
        dist[j] = 1u;             // packed (dist << 1 | second seed)
        fa[1] = j;
        s_cnt[0] = 2;
      }
    }
    __syncthreads();
    // level-synchronous BFS, one CTA barrier a level: eight edges a round
    // per frontier vertex, a warp's claims appended with one atomicAdd
    // (offsets by bit-plane ballots); mode 2 packs (dist << 1 | which seed)
    // and keeps the minimum
    const int lane = tid & 31;
    const unsigned lt = lanemask_lt();
    const bool long_rows = s_long != 0;
    for (uint32_t level = 0;; ++level) {
      const int32_t nf = s_cnt[level % 3];
      if (nf == 0) break;
      if (tid == 0) s_cnt[(level + 2) % 3] = 0;
      if (!long_rows) {
        // one (frontier vertex, neighbour slot) pair a thread, every row
        // having at most PL_SLOTS internal neighbours: a thread makes one
        // claim, a warp appends its claims with one atomicAdd
        const int32_t np = nf * PL_SLOTS;
        for (int32_t x0 = 0; x0 < np; x0 += LOCAL_THREADS) {
          const int32_t x = x0 + tid;
          int32_t w = -1;
          uint32_t cand = 0;
          if (x < np) {
            const int32_t u = fa[x / PL_SLOTS];
            const int32_t r = lrow[u] + x % PL_SLOTS;
            if (r < lrow[u + 1]) w = small ? (int32_t)s_adj[r] : a.g_adj[e0 + r];
            cand = kMode == 2 ? (((level + 1) << 1) | (dist[u] & 1u)) : level + 1;
          }
          bool cl = false;
          if (w >= 0) {
            if (kMode == 2) cl = (dist[w] >> 1) > level && atomicMin(&dist[w], cand) == 0xffffffffu;
            else cl = atomicCAS(&dist[w], 0xffffffffu, cand) == 0xffffffffu;
          }
          const unsigned bb = __ballot_sync(0xffffffffu, cl);
          int32_t base = 0;
          if (lane == 0 && bb) base = atomicAdd(&s_cnt[(level + 1) % 3], __popc(bb));
          base = __shfl_sync(0xffffffffu, base, 0);
          if (cl) fb[base + __popc(bb & lt)] = w;
        }
      } else
      for (int32_t i0 = 0; i0 < nf; i0 += LOCAL_THREADS) {
        const int32_t i = i0 + tid;
        int32_t r0 = 0, r1 = 0;
        uint32_t cand = 0;
        if (i < nf) {
          const int32_t u = fa[i];
          r0 = lrow[u];
          r1 = lrow[u + 1];
          cand = kMode == 2 ? (((level + 1) << 1) | (dist[u] & 1u)) : level + 1;
        }
        while (__any_sync(0xffffffffu, r0 < r1)) {
          int32_t w[8];
#pragma unroll
          for (int k = 0; k < 8; ++k)
            w[k] = r0 + k < r1 ? (small ? (int32_t)s_adj[r0 + k] : a.g_adj[e0 + r0 + k]) : -1;
          uint32_t claim = 0;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            if (w[k] < 0) continue;
            if (kMode == 2) {
              if ((dist[w[k]] >> 1) > level && atomicMin(&dist[w[k]], cand) == 0xffffffffu) claim |= 1u << k;
            } else {
              if (atomicCAS(&dist[w[k]], 0xffffffffu, cand) == 0xffffffffu) claim |= 1u << k;
            }
          }
          const int32_t c = __popc(claim);
          int32_t ex = 0, tot = 0;
#pragma unroll
          for (int bp = 0; bp < 4; ++bp) {
            const unsigned bb = __ballot_sync(0xffffffffu, (c >> bp) & 1);
            ex += __popc(bb & lt) << bp;
            tot += __popc(bb) << bp;
          }
          int32_t base = 0;
          if (lane == 0 && tot) base = atomicAdd(&s_cnt[(level + 1) % 3], tot);
          base = __shfl_sync(0xffffffffu, base, 0) + ex;
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (claim >> k & 1u) fb[base++] = w[k];
          r0 += 8;
        }
      }
      __syncthreads();
      int32_t* t = fa; fa = fb; fb = t;
    }
    __syncthreads();
    if (kMode == 2) {
      const int32_t p2 = a.kbase + a.orank[p];
      const unsigned long long r_first = (unsigned long long)(uint32_t)p;
      const unsigned long long r_second = (unsigned long long)(uint32_t)p2;
      int32_t c2 = 0;
      for (int32_t i = tid; i < m; i += LOCAL_THREADS) {
        const uint32_t d = dist[i];
        a.key[verts[i]] = ((unsigned long long)(d >> 1) << 32) | ((d & 1u) ? r_second : r_first);
        c2 += (int32_t)(d & 1u);
      }
      // sizes of the two halves decide the next round (the patch is connected,
      // so every vertex is reached from one of the two seeds)
      c2 = block_sum(c2, red);
      if (tid == 0) {
        const int32_t cap = a.sv.vmesh ? a.sv.mcap[a.sv.vmesh[a.seed_of[p]]] : a.cap;
        if (m - c2 > cap) { a.next_over[p] = 1; atomicAdd(a.next_cnt, 1); }
        if (c2 > cap) { a.next_over[p2] = 1; atomicAdd(a.next_cnt, 1); }
      }
    } else {
      unsigned long long b = 0ull;
      for (int32_t i = tid; i < m; i += LOCAL_THREADS) {
        const uint32_t d = dist[i];
        if (d == 0xffffffffu) continue;
        const unsigned long long c = ((unsigned long long)d << 32) | (0xffffffffu - (uint32_t)verts[i]);
        b = c > b ? c : b;
      }
      b = block_max(b, red64);
      if (tid == 0) a.best[p] = b;
    }
    __syncthreads();
  }
}

__global__ void k_patch_scatter(const int32_t* __restrict__ label, int32_t n, const int32_t* __restrict__ pstart,
                                int32_t* __restrict__ fill, int32_t* __restrict__ pverts) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int32_t p = label[v];
    pverts[pstart[p] + atomicAdd(&fill[p], 1)] = v;
  }
}

struct BfsLauncher {
  int grid = 0;
  int maxgrid_bfs = 0, maxgrid_cc = 0;
  fp_status init(fp_handle* h) {
    int dev = h->device, sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bfs, BFS_THREADS, 0);
    if (e != cudaSuccess) return check_cuda(h, e, "occupancy");
    maxgrid_bfs = sms * (per > 0 ? per : 1);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_unreached_components, BFS_THREADS, 0);
    if (e != cudaSuccess) return check_cuda(h, e, "occupancy");
    maxgrid_cc = sms * (per > 0 ? per : 1);
    return FP_OK;
  }
  fp_status bfs(fp_handle* h, unsigned long long* key, int4* fa, int4* fb, int32_t* ctr) {
    // frontiers peak near n/8 vertices (seeds every ~cap/2 vertices, about 25
    // levels): one CTA per SM while that fits in one pass, more CTAs (up to
    // full occupancy) for large meshes, whose frontiers are too big for 148
    // CTAs to hide the gather latency; the grid barrier is the price of
    // every extra CTA
    int g = grid_for(h->n / 8, BFS_THREADS);
    if (g < NUM_SMS_B300) g = NUM_SMS_B300;
    if (g > maxgrid_bfs) g = maxgrid_bfs;
    const int32_t* rp = h->rowptr;
    const int32_t* cl = h->col;
    void* args[] = {(void*)&rp, (void*)&cl, (void*)&key, (void*)&fa, (void*)&fb, (void*)&ctr};
    ProfScope ps(FP_PROF_PATCH_BFS, h->stream);
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_bfs, g, BFS_THREADS, args, 0, h->stream);
    h->launches++;
    if (e != cudaSuccess) return check_cuda(h, e, "bfs launch");
    return FP_OK;
  }
};

}  // namespace

fp_status run_patching(fp_handle* h) {
  const int32_t n = h->n;
  const int32_t cap = h->opt.patch_cap;
  if (n == 0) { h->k = 0; return FP_OK; }
  BfsLauncher L;
  FP_TRY(L.init(h));

  const int64_t ints = (int64_t)n + 8;
  unsigned long long *key, *best;
  int4 *fa, *fb;      // frontier queues
  int32_t *group, *flag, *rank, *seed_of, *tmp, *ctr, *pcnt, *pdeg, *pstart, *pedge, *pverts, *loc, *g_adj, *g_vtx;
  int32_t* orank;
  Arena ar;
  auto layout = [&]() {
    key = ar.get<unsigned long long>(n); best = ar.get<unsigned long long>((int64_t)n + 1);
    fa = ar.get<int4>(ints); fb = ar.get<int4>(ints);
    group = ar.get<int32_t>(ints); flag = ar.get<int32_t>(ints); rank = ar.get<int32_t>(ints);
    seed_of = ar.get<int32_t>(ints); tmp = ar.get<int32_t>(scan_tmp_ints((int64_t)n + 1)); ctr = ar.get<int32_t>(8);
    // vertex lists by patch (for the searches inside patches)
    pcnt = ar.get<int32_t>(ints); pdeg = ar.get<int32_t>(ints); pstart = ar.get<int32_t>(ints);
    pedge = ar.get<int32_t>(ints); pverts = ar.get<int32_t>(ints); loc = ar.get<int32_t>(ints);
    g_adj = ar.get<int32_t>(h->nnz + 8); g_vtx = ar.get<int32_t>(5 * (int64_t)n + 8); orank = ar.get<int32_t>(ints);
  };
  layout();
  if (!ar.alloc(h)) return fail(h, FP_ERR_OUT_OF_MEMORY, "patching workspace");
  layout();
  int32_t* hbuf = pinned_scratch();
  if (!hbuf) return fail(h, FP_ERR_OUT_OF_MEMORY, "patching workspace");

  const int G = grid_for(n, 256);
  const SegView sv = h->seg ? h->seg->v : SegView{};
  // R1 seeds
  uint64_t kt = ((uint64_t)2 * (uint64_t)n + (uint64_t)cap - 1) / (uint64_t)cap;
  if (kt < 1) kt = 1;
  {
    ProfScope ps(FP_PROF_PATCH_OTHER, h->stream);
    FP_LAUNCH(h, k_fill_u64, G, 256, 0, key, KEY_INF, (int64_t)n);
    FP_LAUNCH(h, k_seed_flags, G, 256, 0, n, kt, h->opt.seed, flag, sv);
    scan_exclusive(h, flag, rank, n, tmp);
    FP_LAUNCH(h, k_seed_sources, G, 256, 0, n, h->rowptr, flag, rank, 0, key, seed_of, fa, ctr);
  }
  FP_CHECK_LAUNCH(h, "seeds");
  // R2 Voronoi labelling
  FP_TRY(L.bfs(h, key, fa, fb, ctr));
  // R3 unreached components
  {
    ProfScope ps(FP_PROF_PATCH_OTHER, h->stream);
    fill_i32(h, ctr + 4, 0, 1);
    FP_LAUNCH(h, k_count_unreached, G, 256, 0, key, n, ctr + 4);
  }
  cudaMemcpyAsync(hbuf, rank + n, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
  cudaMemcpyAsync(hbuf + 1, ctr + 4, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
  FP_CHECK_LAUNCH(h, "voronoi");
  int32_t st = 0;
  FP_TRY(sync_status(h, &st));
  int32_t k = hbuf[0];
  if (hbuf[1] > 0) {
    int32_t* comp = (int32_t*)fb;   // fb is free between searches
    int g = L.maxgrid_cc < G ? L.maxgrid_cc : G;
    void* args[] = {(void*)&h->rowptr, (void*)&h->col, (void*)&key, (void*)&n, (void*)&comp, (void*)&ctr};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_unreached_components, g, BFS_THREADS, args, 0, h->stream);
    h->launches++;
    if (e != cudaSuccess) return check_cuda(h, e, "components launch");
    FP_LAUNCH(h, k_component_seed_flags, G, 256, 0, comp, n, flag);
    scan_exclusive(h, flag, rank, n, tmp);
    FP_LAUNCH(h, k_seed_sources, G, 256, 0, n, h->rowptr, flag, rank, k, key, seed_of, fa, ctr);
    FP_CHECK_LAUNCH(h, "component seeds");
    FP_TRY(L.bfs(h, key, fa, fb, ctr));
    cudaMemcpyAsync(hbuf, rank + n, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    FP_TRY(sync_status(h, &st));
    k += hbuf[0];
  }
  // stage record (debug_dump): the seeds after R1 + R3 and the first labels
  stage_dump(h, FP_STAGE_SEEDS, 0, seed_of, k);
  if (int32_t* lb = stage_buffer(h, FP_STAGE_LABELS, 0, n)) FP_LAUNCH(h, k_labels_of, G, 256, 0, key, n, lb);
  // vertex lists by patch: labels and counts, their scans (pdeg is cleared to
  // serve as the scatter cursors), the scatter
  auto patch_lists = [&](int32_t kk) {
    ProfScope ps(FP_PROF_PATCH_OTHER, h->stream);
    FP_LAUNCH(h, k_zero2, grid_for(kk, 256), 256, 0, pcnt, pdeg, (int64_t)kk);
    FP_LAUNCH(h, k_labels_counts, G, 256, 0, key, h->rowptr, n, group, pcnt, pdeg);
    scan_exclusive_pair_zero(h, pcnt, pstart, pdeg, pedge, kk, tmp);
    FP_LAUNCH(h, k_patch_scatter, G, 256, 0, group, n, pstart, pdeg, pverts);
  };
  LocalArgs la{0, h->rowptr, h->col, group, pstart, pverts, pedge, g_adj, g_vtx, loc, nullptr, orank, 0,
               seed_of, best, key, nullptr, nullptr, cap, sv};
  const int GL = NUM_SMS_B300 * 8;
  // R4 Lloyd rounds
  const int GK = grid_for(k, 256);
  for (int32_t it = 0; it < h->opt.lloyd_rounds; ++it) {
    patch_lists(k);
    la.k = k;
    la.over = nullptr;
    {
      ProfScope ps(FP_PROF_PATCH_LOCAL, h->stream);
      FP_LAUNCH(h, k_patch_local<0>, k < GL ? k : GL, LOCAL_THREADS, 0, la);
    }
    {
      ProfScope ps(FP_PROF_PATCH_OTHER, h->stream);
      FP_LAUNCH(h, k_lloyd_apply, GK, 256, 0, best, k, seed_of);
      FP_LAUNCH(h, k_fill_u64, G, 256, 0, key, KEY_INF, (int64_t)n);
      FP_LAUNCH(h, k_all_seed_sources, GK, 256, 0, h->rowptr, seed_of, k, key, fa, ctr);
    }
    FP_CHECK_LAUNCH(h, "lloyd");
    stage_dump(h, FP_STAGE_LLOYD_SEEDS, it, seed_of, k);
    FP_TRY(L.bfs(h, key, fa, fb, ctr));
    if (int32_t* lb = stage_buffer(h, FP_STAGE_LABELS, it + 1, n)) FP_LAUNCH(h, k_labels_of, G, 256, 0, key, n, lb);
  }
  // R5 cap: split until every patch fits. The first round counts the patch
  // sizes; every split counts its two halves, so a later round rebuilds the
  // vertex lists only when some half is still above cap.
  int32_t* over = rank;
  int32_t* over_next = flag;
  int32_t* ocnt = ctr + 5;
  patch_lists(k);
  {
    ProfScope ps(FP_PROF_PATCH_OTHER, h->stream);
    FP_LAUNCH(h, k_oversize_flags, grid_for(k, 256), 256, 0, pcnt, k, cap, over, seed_of, sv);
    scan_exclusive(h, over, orank, k, tmp);
  }
  cudaMemcpyAsync(hbuf, orank + k, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
  FP_CHECK_LAUNCH(h, "sizes");
  // the first round is queued before its count is known (with no oversize
  // patch its kernels find nothing to do); one sync then reads both counts
  int32_t nover = -1;
  for (int32_t round = 0; round < n; ++round) {
    const int GKr = grid_for(k, 256);
    la.k = k;
    la.over = over;
    la.kbase = k;
    la.next_over = over_next;
    la.next_cnt = ocnt;
    // the halves take the new ids k .. k+nover-1 (nover <= k, and k + nover
    // <= n as every patch keeps a vertex)
    const int64_t nclear = nover >= 0 ? (int64_t)k + nover : (2 * (int64_t)k < n ? 2 * (int64_t)k : (int64_t)n);
    fill_i32(h, over_next, 0, nclear);
    fill_i32(h, ocnt, 0, 1);
    {
      ProfScope ps(FP_PROF_PATCH_LOCAL, h->stream);
      FP_LAUNCH(h, k_patch_local<1>, k < GL ? k : GL, LOCAL_THREADS, 0, la);
      FP_LAUNCH(h, k_split_seeds, GKr, 256, 0, best, over, orank, k, seed_of);
      FP_LAUNCH(h, k_patch_local<2>, k < GL ? k : GL, LOCAL_THREADS, 0, la);
    }
    cudaMemcpyAsync(hbuf + 1, ocnt, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    FP_CHECK_LAUNCH(h, "split");
    FP_TRY(sync_status(h, &st));
    if (nover < 0) nover = hbuf[0];
    k += nover;
    nover = hbuf[1];
    if (nover == 0) break;
    std::swap(over, over_next);
    {
      ProfScope ps(FP_PROF_PATCH_OTHER, h->stream);
      scan_exclusive(h, over, orank, k, tmp);
    }
    patch_lists(k);
  }
  {
    ProfScope ps(FP_PROF_PATCH_OTHER, h->stream);
    FP_LAUNCH(h, k_labels_of, G, 256, 0, key, n, h->gmap);
  }
  FP_CHECK_LAUNCH(h, "labels");
  h->k = k;
  dev_free(h, ar.base);
  return FP_OK;
}

}  // namespace fp
