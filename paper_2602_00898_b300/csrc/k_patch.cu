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
// The BFS is one persistent cooperative launch per search: the level loop
// runs on the device with a grid barrier between levels, and frontier queues
// are compacted with an atomic counter.
#include <cooperative_groups.h>

#include "fp_internal.cuh"

namespace cg = cooperative_groups;

namespace fp {
namespace {

constexpr int BFS_THREADS = 256;

inline int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > NUM_SMS_B300 * 32) g = NUM_SMS_B300 * 32;
  return (int)(g < 1 ? 1 : g);
}

// Level-synchronous multi-source BFS on packed keys (dist << 32 | label).
// ctr[0] holds the size of the initial frontier `fa`. An edge {u,v} is
// followed iff group is null or group[u] == group[v]. On exit key[] holds the
// distance and the minimum label for every reached vertex.
__global__ void __launch_bounds__(BFS_THREADS) k_bfs(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                                     unsigned long long* key, const int32_t* __restrict__ group,
                                                     int32_t* fa, int32_t* fb, int32_t* ctr) {
  cg::grid_group grid = cg::this_grid();
  int32_t* cur = fa;
  int32_t* nxt = fb;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (uint32_t level = 0;; ++level) {
    const int32_t ncur = __ldcg(&ctr[level % 3]);
    if (ncur == 0) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr[(level + 2) % 3] = 0;
    const unsigned long long dnext = (unsigned long long)(level + 1) << 32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ncur; i += stride) {
      const int32_t u = __ldcg(&cur[i]);
      const unsigned long long lab = __ldcg(&key[u]) & 0xffffffffull;
      const int32_t gu = group ? group[u] : 0;
      const int32_t e1 = rowptr[u + 1];
      for (int32_t e = rowptr[u]; e < e1; ++e) {
        const int32_t v = col[e];
        if (group && group[v] != gu) continue;
        const unsigned long long kv = __ldcg(&key[v]);
        if ((kv >> 32) <= level) continue;                 // settled at an earlier level
        const unsigned long long old = atomicMin(&key[v], dnext | lab);
        if (old == KEY_INF) nxt[atomicAdd(&ctr[(level + 1) % 3], 1)] = v;
      }
    }
    int32_t* t = cur; cur = nxt; nxt = t;
    grid.sync();
  }
}

__global__ void k_seed_flags(int32_t n, uint64_t kt, uint64_t seed, int32_t* __restrict__ flag) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    uint64_t h = splitmix64_state(seed * 0x9E3779B97F4A7C15ull + (uint64_t)(uint32_t)v);
    flag[v] = ((h >> 32) * (uint64_t)n) < (kt << 32) ? 1 : 0;
  }
}

// Seeds (flag[v] = 1) with rank = base + rank[v] become BFS sources.
__global__ void k_seed_sources(int32_t n, const int32_t* __restrict__ flag, const int32_t* __restrict__ rank,
                               int32_t base, unsigned long long* __restrict__ key, int32_t* __restrict__ seed_of,
                               int32_t* __restrict__ frontier, int32_t* ctr) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    if (flag[v]) {
      int32_t r = rank[v];
      key[v] = (unsigned long long)(uint32_t)(base + r);
      seed_of[base + r] = v;
      frontier[r] = v;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctr[0] = rank[n];
    ctr[1] = 0;
    ctr[2] = 0;
  }
}

__global__ void k_fill_u64(unsigned long long* p, unsigned long long v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void k_labels_of(const unsigned long long* __restrict__ key, int32_t n, int32_t* __restrict__ label) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    label[v] = key[v] == KEY_INF ? -1 : (int32_t)(uint32_t)key[v];
}

__global__ void k_count_unreached(const unsigned long long* __restrict__ key, int32_t n, int32_t* cnt) {
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
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    flag[v] = comp[v] == v ? 1 : 0;
}

// Lloyd: boundary vertices (a neighbour with another label) are the sources
// of a BFS restricted to the patch.
__global__ void k_boundary_sources(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int32_t n,
                                   const int32_t* __restrict__ label, unsigned long long* __restrict__ key2,
                                   int32_t* __restrict__ frontier, int32_t* ctr) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int32_t lv = label[v];
    bool bnd = false;
    for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e)
      if (label[col[e]] != lv) { bnd = true; break; }
    key2[v] = bnd ? 0ull : KEY_INF;
    if (bnd) frontier[atomicAdd(&ctr[0], 1)] = v;
  }
}

// best[label] = max over reached v of (dist << 32 | ~v): the farthest vertex,
// ties to the smallest id.
__global__ void k_pick_farthest(const unsigned long long* __restrict__ key2, const int32_t* __restrict__ label, int32_t n,
                                unsigned long long* __restrict__ best) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    unsigned long long k2 = key2[v];
    if (k2 == KEY_INF) continue;
    atomicMax(&best[label[v]], (k2 & 0xffffffff00000000ull) | (unsigned long long)(0xffffffffu - (uint32_t)v));
  }
}

__global__ void k_lloyd_apply(const unsigned long long* __restrict__ best, int32_t k, int32_t* __restrict__ seed_of) {
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x)
    if (best[p]) seed_of[p] = (int32_t)(0xffffffffu - (uint32_t)best[p]);
}

// All k seeds become sources with their own rank.
__global__ void k_all_seed_sources(const int32_t* __restrict__ seed_of, int32_t k, unsigned long long* __restrict__ key,
                                   int32_t* __restrict__ frontier, int32_t* ctr) {
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x) {
    key[seed_of[p]] = (unsigned long long)(uint32_t)p;
    frontier[p] = seed_of[p];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) { ctr[0] = k; ctr[1] = 0; ctr[2] = 0; }
}

__global__ void k_patch_sizes(const int32_t* __restrict__ label, int32_t n, int32_t* __restrict__ psize) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) atomicAdd(&psize[label[v]], 1);
}

__global__ void k_oversize_flags(const int32_t* __restrict__ psize, int32_t k, int32_t cap, int32_t* __restrict__ over) {
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x) over[p] = psize[p] > cap;
}

// Sources of the "farthest from the seed" search: the seeds of oversize patches.
__global__ void k_oversize_seed_sources(const int32_t* __restrict__ seed_of, const int32_t* __restrict__ over,
                                        const int32_t* __restrict__ orank, int32_t k,
                                        unsigned long long* __restrict__ key2, int32_t* __restrict__ frontier, int32_t* ctr) {
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x)
    if (over[p]) {
      key2[seed_of[p]] = 0ull;
      frontier[orank[p]] = seed_of[p];
    }
  if (blockIdx.x == 0 && threadIdx.x == 0) { ctr[0] = orank[k]; ctr[1] = 0; ctr[2] = 0; }
}

// Reset the labels of every vertex of an oversize patch.
__global__ void k_reset_oversize(const int32_t* __restrict__ label, const int32_t* __restrict__ over, int32_t n,
                                 unsigned long long* __restrict__ key) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (over[label[v]]) key[v] = KEY_INF;
}

// Two sources per oversize patch p: its seed (rank p) and its farthest vertex
// (new rank k + orank[p]).
__global__ void k_split_sources(const unsigned long long* __restrict__ best, const int32_t* __restrict__ over,
                                const int32_t* __restrict__ orank, int32_t k, int32_t* __restrict__ seed_of,
                                unsigned long long* __restrict__ key, int32_t* __restrict__ frontier, int32_t* ctr) {
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x) {
    if (!over[p]) continue;
    int32_t r = k + orank[p];
    int32_t far = (int32_t)(0xffffffffu - (uint32_t)best[p]);
    seed_of[r] = far;
    key[seed_of[p]] = (unsigned long long)(uint32_t)p;
    key[far] = (unsigned long long)(uint32_t)r;
    frontier[2 * orank[p]] = seed_of[p];
    frontier[2 * orank[p] + 1] = far;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) { ctr[0] = 2 * orank[k]; ctr[1] = 0; ctr[2] = 0; }
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
  fp_status bfs(fp_handle* h, unsigned long long* key, const int32_t* group, int32_t* fa, int32_t* fb, int32_t* ctr) {
    int g = grid_for(h->n, BFS_THREADS);
    if (g > maxgrid_bfs) g = maxgrid_bfs;
    const int32_t* rp = h->rowptr;
    const int32_t* cl = h->col;
    void* args[] = {(void*)&rp, (void*)&cl, (void*)&key, (void*)&group, (void*)&fa, (void*)&fb, (void*)&ctr};
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

  size_t ints = (size_t)n + 8;
  unsigned long long* key = (unsigned long long*)dev_alloc(h, sizeof(unsigned long long) * n);
  unsigned long long* key2 = (unsigned long long*)dev_alloc(h, sizeof(unsigned long long) * n);
  unsigned long long* best = (unsigned long long*)dev_alloc(h, sizeof(unsigned long long) * (n + 1));
  int32_t* group = (int32_t*)dev_alloc(h, sizeof(int32_t) * ints);
  int32_t* fa = (int32_t*)dev_alloc(h, sizeof(int32_t) * ints);
  int32_t* fb = (int32_t*)dev_alloc(h, sizeof(int32_t) * ints);
  int32_t* flag = (int32_t*)dev_alloc(h, sizeof(int32_t) * ints);
  int32_t* rank = (int32_t*)dev_alloc(h, sizeof(int32_t) * ints);
  int32_t* seed_of = (int32_t*)dev_alloc(h, sizeof(int32_t) * ints);
  int32_t* tmp = (int32_t*)dev_alloc(h, sizeof(int32_t) * scan_tmp_ints(n + 1));
  int32_t* ctr = (int32_t*)dev_alloc(h, sizeof(int32_t) * 8);
  int32_t* hbuf = nullptr;
  if (!key || !key2 || !best || !group || !fa || !fb || !flag || !rank || !seed_of || !tmp || !ctr)
    return fail(h, FP_ERR_OUT_OF_MEMORY, "patching workspace");
  if (cudaMallocHost(&hbuf, 4 * sizeof(int32_t)) != cudaSuccess) return fail(h, FP_ERR_OUT_OF_MEMORY, "pinned");

  const int G = grid_for(n, 256);
  // R1 seeds
  uint64_t kt = ((uint64_t)2 * (uint64_t)n + (uint64_t)cap - 1) / (uint64_t)cap;
  if (kt < 1) kt = 1;
  {
    ProfScope ps(FP_PROF_PATCH_OTHER, h->stream);
    FP_LAUNCH(h, k_fill_u64, G, 256, 0, key, KEY_INF, (int64_t)n);
    FP_LAUNCH(h, k_seed_flags, G, 256, 0, n, kt, h->opt.seed, flag);
    scan_exclusive(h, flag, rank, n, tmp);
    FP_LAUNCH(h, k_seed_sources, G, 256, 0, n, flag, rank, 0, key, seed_of, fa, ctr);
  }
  FP_CHECK_LAUNCH(h, "seeds");
  // R2 Voronoi labelling
  FP_TRY(L.bfs(h, key, nullptr, fa, fb, ctr));
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
    int32_t* comp = fb;           // fb is free between searches
    int g = L.maxgrid_cc < G ? L.maxgrid_cc : G;
    void* args[] = {(void*)&h->rowptr, (void*)&h->col, (void*)&key, (void*)&n, (void*)&comp, (void*)&ctr};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_unreached_components, g, BFS_THREADS, args, 0, h->stream);
    h->launches++;
    if (e != cudaSuccess) return check_cuda(h, e, "components launch");
    FP_LAUNCH(h, k_component_seed_flags, G, 256, 0, comp, n, flag);
    scan_exclusive(h, flag, rank, n, tmp);
    FP_LAUNCH(h, k_seed_sources, G, 256, 0, n, flag, rank, k, key, seed_of, fa, ctr);
    FP_CHECK_LAUNCH(h, "component seeds");
    FP_TRY(L.bfs(h, key, nullptr, fa, fb, ctr));
    cudaMemcpyAsync(hbuf, rank + n, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    FP_TRY(sync_status(h, &st));
    k += hbuf[0];
  }
  // R4 Lloyd rounds
  const int GK = grid_for(k, 256);
  for (int32_t it = 0; it < h->opt.lloyd_rounds; ++it) {
    {
      ProfScope ps(FP_PROF_PATCH_OTHER, h->stream);
      FP_LAUNCH(h, k_labels_of, G, 256, 0, key, n, group);
      fill_i32(h, ctr, 0, 3);
      FP_LAUNCH(h, k_boundary_sources, G, 256, 0, h->rowptr, h->col, n, group, key2, fa, ctr);
    }
    FP_TRY(L.bfs(h, key2, group, fa, fb, ctr));
    {
      ProfScope ps(FP_PROF_PATCH_OTHER, h->stream);
      FP_LAUNCH(h, k_fill_u64, GK, 256, 0, best, 0ull, (int64_t)k);
      FP_LAUNCH(h, k_pick_farthest, G, 256, 0, key2, group, n, best);
      FP_LAUNCH(h, k_lloyd_apply, GK, 256, 0, best, k, seed_of);
      FP_LAUNCH(h, k_fill_u64, G, 256, 0, key, KEY_INF, (int64_t)n);
      FP_LAUNCH(h, k_all_seed_sources, GK, 256, 0, seed_of, k, key, fa, ctr);
    }
    FP_CHECK_LAUNCH(h, "lloyd");
    FP_TRY(L.bfs(h, key, nullptr, fa, fb, ctr));
  }
  // R5 cap: split until every patch fits
  int32_t* psize = flag;   // reuse: [k] sizes, then rank for oversize flags
  int32_t* over = rank;
  int32_t* orank = (int32_t*)dev_alloc(h, sizeof(int32_t) * ints);
  if (!orank) return fail(h, FP_ERR_OUT_OF_MEMORY, "split workspace");
  for (int32_t round = 0; round < n; ++round) {
    const int GKr = grid_for(k, 256);
    {
      ProfScope ps(FP_PROF_PATCH_OTHER, h->stream);
      FP_LAUNCH(h, k_labels_of, G, 256, 0, key, n, group);
      fill_i32(h, psize, 0, k);
      FP_LAUNCH(h, k_patch_sizes, G, 256, 0, group, n, psize);
      FP_LAUNCH(h, k_oversize_flags, GKr, 256, 0, psize, k, cap, over);
      scan_exclusive(h, over, orank, k, tmp);
    }
    cudaMemcpyAsync(hbuf, orank + k, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    FP_CHECK_LAUNCH(h, "sizes");
    FP_TRY(sync_status(h, &st));
    const int32_t nover = hbuf[0];
    if (nover == 0) break;
    {
      ProfScope ps(FP_PROF_PATCH_OTHER, h->stream);
      FP_LAUNCH(h, k_fill_u64, G, 256, 0, key2, KEY_INF, (int64_t)n);
      FP_LAUNCH(h, k_oversize_seed_sources, GKr, 256, 0, seed_of, over, orank, k, key2, fa, ctr);
    }
    FP_TRY(L.bfs(h, key2, group, fa, fb, ctr));
    {
      ProfScope ps(FP_PROF_PATCH_OTHER, h->stream);
      FP_LAUNCH(h, k_fill_u64, GKr, 256, 0, best, 0ull, (int64_t)k);
      FP_LAUNCH(h, k_pick_farthest, G, 256, 0, key2, group, n, best);
      FP_LAUNCH(h, k_reset_oversize, G, 256, 0, group, over, n, key);
      FP_LAUNCH(h, k_split_sources, GKr, 256, 0, best, over, orank, k, seed_of, key, fa, ctr);
    }
    FP_CHECK_LAUNCH(h, "split");
    FP_TRY(L.bfs(h, key, group, fa, fb, ctr));
    k += nover;
  }
  {
    ProfScope ps(FP_PROF_PATCH_OTHER, h->stream);
    FP_LAUNCH(h, k_labels_of, G, 256, 0, key, n, h->gmap);
  }
  FP_CHECK_LAUNCH(h, "labels");
  h->k = k;
  cudaFreeHost(hbuf);
  dev_free(h, key); dev_free(h, key2); dev_free(h, best); dev_free(h, group); dev_free(h, fa); dev_free(h, fb);
  dev_free(h, flag); dev_free(h, rank); dev_free(h, seed_of); dev_free(h, tmp); dev_free(h, ctr); dev_free(h, orank);
  return FP_OK;
}

}  // namespace fp
