// a5 local ordering and a6 permutation assembly (Algorithm 3; Section 5
// "Concatenation and schedules"), a8 DOF expansion (Section 6.5).
//
// Layout: node sizes -> subtree sizes -> first position of every node in the
// chosen schedule (post-order: left subtree, right subtree, node; level order:
// deepest level first, node index ascending), one CTA.
//
// LocalOrder: exact minimum degree on the node's induced subgraph (the paper
// uses AMD; ties go to the smallest original vertex id). One CTA per node holds
// the elimination graph as a bit matrix (row i = neighbours of local vertex i):
// each step takes the arg-min of (degree, local index) -- local indices follow
// the original ids -- and ORs the pivot row into every neighbour's row, which
// makes the neighbourhood a clique, then recounts those degrees with popc.
//   * small nodes (m <= 512, the leaf patches): one warp per node, rows in
//     shared memory, no CTA barriers;
//   * mid nodes (m <= 1344): 256 threads, rows in shared memory (<= 221 KB);
//   * large nodes (m <= 32768): 256 threads, rows in global memory.
// The kinds run on two streams so that the long serial separator orderings
// overlap the leaves.
#include "fp_device.cuh"

namespace fp {
namespace {

constexpr int MD_SMALL = 512;
constexpr int MD_MID = 1344;
constexpr int MD_MAX = 32768;
constexpr int MD_THREADS = 256;
constexpr uint16_t DEG_DEAD = 0xffff;

inline int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > NUM_SMS_B300 * 32) g = NUM_SMS_B300 * 32;
  return (int)(g < 1 ? 1 : g);
}

int pow2_host(int x) {
  int p = 32;
  while (p < x) p <<= 1;
  return p;
}

__global__ void k_node_sizes(const int32_t* __restrict__ node_of, int32_t n, int32_t* __restrict__ size) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) atomicAdd(&size[node_of[v]], 1);
}

__global__ void k_scatter_nodes(const int32_t* __restrict__ node_of, int32_t n, const int32_t* __restrict__ start,
                                int32_t* __restrict__ fill, int32_t* __restrict__ list) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int32_t t = node_of[v];
    list[start[t] + atomicAdd(&fill[t], 1)] = v;
  }
}

// Schedule layout (one CTA). sub: scratch [nnodes].
__global__ void k_tree_layout(int32_t D, int64_t nnodes, const int32_t* __restrict__ size, int32_t* __restrict__ sub,
                              int32_t* __restrict__ begin, int32_t schedule) {
  __shared__ int32_t red[40];
  for (int32_t d = D; d >= 0; --d) {
    const int64_t a = ((int64_t)1 << d) - 1, b = ((int64_t)1 << (d + 1)) - 1;
    for (int64_t t = a + threadIdx.x; t < b; t += blockDim.x) {
      int32_t s = size[t];
      if (2 * t + 1 < nnodes) s += sub[2 * t + 1] + sub[2 * t + 2];
      sub[t] = s;
    }
    __syncthreads();
  }
  if (schedule == 0) {
    // begin[t] temporarily holds the start of t's subtree
    if (threadIdx.x == 0) begin[0] = 0;
    __syncthreads();
    for (int32_t d = 0; d <= D; ++d) {
      const int64_t a = ((int64_t)1 << d) - 1, b = ((int64_t)1 << (d + 1)) - 1;
      for (int64_t t = a + threadIdx.x; t < b; t += blockDim.x) {
        const int32_t st = begin[t];
        int32_t kids = 0;
        if (2 * t + 1 < nnodes) {
          begin[2 * t + 1] = st;
          begin[2 * t + 2] = st + sub[2 * t + 1];
          kids = sub[2 * t + 1] + sub[2 * t + 2];
        }
        begin[t] = st + kids;
      }
      __syncthreads();
    }
  } else {
    int32_t off = 0;
    for (int32_t d = D; d >= 0; --d) {
      const int64_t a = ((int64_t)1 << d) - 1, b = ((int64_t)1 << (d + 1)) - 1;
      for (int64_t c = a; c < b; c += blockDim.x) {
        const int64_t t = c + threadIdx.x;
        int32_t s = t < b ? size[t] : 0, tot;
        int32_t ex = block_excl_scan_i32(s, &tot, red);
        if (t < b) begin[t] = off + ex;
        off += tot;
      }
    }
  }
}

struct MdArgs {
  const int32_t* rowptr;
  const int32_t* col;
  const int32_t* node_of;
  const int32_t* node_begin;
  const int32_t* node_size;
  const int32_t* nvstart;     // [nnodes+1] start of each node's vertex list
  int32_t* nvlist;            // vertices grouped by node (sorted by id per node here)
  int32_t* loc;               // [n] local index of a vertex in its node
  int32_t* perm;              // [n] output
  const int32_t* nodes;       // node ids handled by this launch
  int32_t nnodes_launch;
  uint32_t* grows;            // large kind: row storage base
  const int64_t* grow_off;    // large kind: per launched node, word offset into grows
  int32_t* gsort;             // large kind: sort scratch base
  const int64_t* gsort_off;   // large kind: per launched node, int offset into gsort
};

// Minimum degree for one node. kNT threads; kind 0 small (one warp, smem rows),
// 1 mid (smem rows), 2 large (global rows).
template <int kNT, int kKind>
__global__ void __launch_bounds__(kNT) k_md(MdArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t red32[40];
  __shared__ int32_t redi[40];
  __shared__ int32_t s_nnb;
  constexpr bool kWarp = (kNT == 32);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int kWarps = kNT / 32;

  for (int32_t li = blockIdx.x; li < a.nnodes_launch; li += gridDim.x) {
    const int32_t t = a.nodes[li];
    const int32_t m = a.node_size[t];
    const int32_t pbeg = a.node_begin[t];
    int32_t* verts = a.nvlist + a.nvstart[t];
    const int W = (m + 31) >> 5;
    // ---- shared memory carve-up
    uint32_t* rows;
    uint16_t* deg;
    uint16_t* nb;
    int32_t* sortbuf;
    const int NS = pow2_at_least(m, 32);
    if (kKind == 2) {
      deg = (uint16_t*)smem;
      nb = deg + MD_MAX;
      rows = a.grows + a.grow_off[li];
      sortbuf = a.gsort + a.gsort_off[li];
    } else {
      rows = (uint32_t*)smem;
      deg = (uint16_t*)(rows + (size_t)m * W);
      nb = deg + ((m + 1) & ~1);
      sortbuf = (int32_t*)smem;          // overlaps rows; used before they are built
    }
    // ---- sort the node's vertices by original id
    for (int i = tid; i < NS; i += kNT) sortbuf[i] = i < m ? verts[i] : INT_MAX;
    if (kWarp) __syncwarp(); else __syncthreads();
    bitonic_sort<!kWarp>(sortbuf, NS, tid, kNT);
    for (int i = tid; i < m; i += kNT) {
      const int32_t v = sortbuf[i];
      verts[i] = v;
      a.loc[v] = i;
    }
    if (kWarp) __syncwarp(); else __syncthreads();
    // ---- elimination graph = induced subgraph
    for (int64_t i = tid; i < (int64_t)m * W; i += kNT) rows[i] = 0u;
    if (kWarp) __syncwarp(); else __syncthreads();
    for (int i = tid; i < m; i += kNT) {
      const int32_t v = verts[i];
      uint32_t* r = rows + (size_t)i * W;
      int c = 0;
      for (int32_t e = a.rowptr[v]; e < a.rowptr[v + 1]; ++e) {
        const int32_t u = a.col[e];
        if (a.node_of[u] != t) continue;
        const int j = a.loc[u];
        r[j >> 5] |= 1u << (j & 31);
        ++c;
      }
      deg[i] = (uint16_t)c;
    }
    if (kWarp) __syncwarp(); else __syncthreads();
    // ---- elimination
    for (int step = 0; step < m; ++step) {
      uint32_t best = 0xffffffffu;
      for (int i = tid; i < m; i += kNT) {
        const uint16_t dg = deg[i];
        if (dg != DEG_DEAD) {
          const uint32_t key = ((uint32_t)dg << 16) | (uint32_t)i;
          best = key < best ? key : best;
        }
      }
      uint32_t kmin;
      if (kWarp) kmin = warp_min(best);
      else kmin = block_min(best, red32);
      const int p = (int)(kmin & 0xffffu);
      const uint32_t* rp = rows + (size_t)p * W;
      // neighbour list of p, in increasing local index
      if (kWarp || wid == 0) {
        int base = 0;
        for (int w0 = 0; w0 < W; w0 += 32) {
          const int w = w0 + lane;
          const uint32_t bits = w < W ? rp[w] : 0u;
          const int c = __popc(bits);
          int ex = warp_incl_scan_i32(c) - c;
          const int tot = __shfl_sync(0xffffffffu, ex + c, 31);
          uint32_t x = bits;
          while (x) {
            const int bt = __ffs(x) - 1;
            x &= x - 1;
            nb[base + ex++] = (uint16_t)(w * 32 + bt);
          }
          base += tot;
        }
        if (lane == 0) {
          s_nnb = base;
          a.perm[pbeg + step] = verts[p];
          deg[p] = DEG_DEAD;
        }
      }
      if (kWarp) __syncwarp(); else __syncthreads();
      const int nnb = s_nnb;
      // clique: row[u] |= row[p], minus u and p; one warp per neighbour
      for (int q = wid; q < nnb; q += kWarps) {
        const int u = nb[q];
        uint32_t* ru = rows + (size_t)u * W;
        int c = 0;
        for (int w = lane; w < W; w += 32) {
          uint32_t x = ru[w] | rp[w];
          if (w == (u >> 5)) x &= ~(1u << (u & 31));
          if (w == (p >> 5)) x &= ~(1u << (p & 31));
          ru[w] = x;
          c += __popc(x);
        }
        c = warp_sum(c);
        if (lane == 0) deg[u] = (uint16_t)c;
      }
      if (kWarp) __syncwarp(); else __syncthreads();
    }
    if (kWarp) __syncwarp(); else __syncthreads();
  }
}

__global__ void k_iperm(const int32_t* __restrict__ perm, int32_t n, int32_t* __restrict__ iperm) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) iperm[perm[i]] = i;
}

__global__ void k_dof_perm(const int32_t* __restrict__ perm, int32_t n, int32_t b, int32_t* __restrict__ perm_d,
                           int32_t* __restrict__ iperm_d) {
  const int64_t N = (int64_t)n * b;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = (int32_t)(i / b), c = (int32_t)(i % b);
    const int32_t v = b * perm[k] + c;
    if (perm_d) perm_d[i] = v;
    if (iperm_d) iperm_d[v] = (int32_t)i;
  }
}

__global__ void k_dof_symbolic(const int32_t* __restrict__ parent, const int32_t* __restrict__ cc, int32_t n, int32_t b,
                               int32_t* __restrict__ parent_d, int32_t* __restrict__ cc_d) {
  const int64_t N = (int64_t)n * b;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = (int32_t)(i / b), c = (int32_t)(i % b);
    if (parent_d) parent_d[i] = c < b - 1 ? (int32_t)(i + 1) : (parent[j] < 0 ? -1 : b * parent[j]);
    if (cc_d) cc_d[i] = b * cc[j] - c;
  }
}

size_t md_smem(int kind, int mmax) {
  const int W = (mmax + 31) >> 5;
  if (kind == 2) return (size_t)2 * MD_MAX * sizeof(uint16_t);
  size_t rows = (size_t)mmax * W * 4;
  size_t sortb = (size_t)pow2_host(mmax) * 4;
  size_t need = rows + 2 * (size_t)((mmax + 1) & ~1) * 2;
  return need > sortb ? need : sortb;
}

}  // namespace

fp_status run_local_order(fp_handle* h) {
  const int32_t n = h->n;
  const int64_t nn = h->nnodes;
  const int G = grid_for(n, 256);
  auto I = [&](int64_t c) { return (int32_t*)dev_alloc(h, sizeof(int32_t) * (c > 0 ? c : 1)); };
  int32_t *sub = I(nn), *nvstart = I(nn + 1), *nvfill = I(nn), *nvlist = I(n), *loc = I(n), *tmp = I(scan_tmp_ints(nn) + 8);
  if (!sub || !nvstart || !nvfill || !nvlist || !loc || !tmp) return fail(h, FP_ERR_OUT_OF_MEMORY, "ordering workspace");
  {
    ProfScope ps(FP_PROF_LAYOUT, h->stream);
    fill_i32(h, h->node_size, 0, nn);
    if (n > 0) FP_LAUNCH(h, k_node_sizes, G, 256, 0, h->node_of, n, h->node_size);
    FP_LAUNCH(h, k_tree_layout, 1, 1024, 0, h->D, nn, h->node_size, sub, h->node_begin, h->opt.schedule);
    scan_exclusive(h, h->node_size, nvstart, nn, tmp);
    fill_i32(h, nvfill, 0, nn);
    if (n > 0) FP_LAUNCH(h, k_scatter_nodes, G, 256, 0, h->node_of, n, nvstart, nvfill, nvlist);
  }
  FP_CHECK_LAUNCH(h, "tree layout");
  // plan the ordering launches from the node sizes
  std::vector<int32_t> hs(nn);
  cudaError_t e = cudaMemcpyAsync(hs.data(), h->node_size, sizeof(int32_t) * nn, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "node sizes");
  int32_t st = 0;
  FP_TRY(sync_status(h, &st));
  std::vector<int32_t> ls[3];
  std::vector<int64_t> goff, soff;
  int mmax[3] = {0, 0, 0};
  int64_t gwords = 0, gsort = 0;
  for (int64_t t = 0; t < nn; ++t) {
    const int m = hs[t];
    if (m == 0) continue;
    if (m > MD_MAX) return fail(h, FP_ERR_UNSUPPORTED, "a tree node has more than 32768 vertices");
    const int kind = m <= MD_SMALL ? 0 : (m <= MD_MID ? 1 : 2);
    ls[kind].push_back((int32_t)t);
    if (m > mmax[kind]) mmax[kind] = m;
    if (kind == 2) {
      goff.push_back(gwords);
      gwords += (int64_t)m * ((m + 31) / 32);
      soff.push_back(gsort);
      gsort += pow2_host(m);
    }
  }
  // node lists + large-kind offsets in one upload
  const int64_t nlist = (int64_t)ls[0].size() + ls[1].size() + ls[2].size();
  std::vector<int64_t> up(nlist + 2 * goff.size() + 1);
  int32_t* up32 = (int32_t*)up.data();
  int64_t o = 0;
  for (int kd = 0; kd < 3; ++kd)
    for (int32_t t : ls[kd]) up32[o++] = t;
  const int64_t off64 = (o + 1) / 2;
  for (size_t i = 0; i < goff.size(); ++i) { up[off64 + i] = goff[i]; up[off64 + goff.size() + i] = soff[i]; }
  int64_t* dup = (int64_t*)dev_alloc(h, sizeof(int64_t) * (up.size() + 1));
  uint32_t* grows = (uint32_t*)dev_alloc(h, sizeof(uint32_t) * (gwords > 0 ? gwords : 1));
  int32_t* gs = I(gsort);
  if (!dup || !grows || !gs) return fail(h, FP_ERR_OUT_OF_MEMORY, "ordering rows");
  e = cudaMemcpyAsync(dup, up.data(), sizeof(int64_t) * up.size(), cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "upload node lists");
  const int32_t* dnodes = (const int32_t*)dup;
  MdArgs base{h->rowptr, h->col, h->node_of, h->node_begin, h->node_size, nvstart, nvlist, loc, h->perm,
              nullptr, 0, grows, dup + off64, gs, dup + off64 + goff.size()};
  // second stream for the large and mid nodes
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  if (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) != cudaSuccess)
    return fail(h, FP_ERR_CUDA, "stream/event create");
  cudaEventRecord(ev_fork, h->stream);
  cudaStreamWaitEvent(s2, ev_fork, 0);
  int64_t lo = 0;
  const int64_t lo1 = (int64_t)ls[0].size(), lo2 = lo1 + (int64_t)ls[1].size();
  if (!ls[2].empty()) {
    MdArgs a = base;
    a.nodes = dnodes + lo2;
    a.nnodes_launch = (int32_t)ls[2].size();
    size_t sm = md_smem(2, mmax[2]);
    cudaFuncSetAttribute(k_md<MD_THREADS, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    ProfScope ps(FP_PROF_MD_LARGE, s2);
    k_md<MD_THREADS, 2><<<(unsigned)ls[2].size(), MD_THREADS, sm, s2>>>(a);
    h->launches++;
  }
  if (!ls[1].empty()) {
    MdArgs a = base;
    a.nodes = dnodes + lo1;
    a.nnodes_launch = (int32_t)ls[1].size();
    size_t sm = md_smem(1, mmax[1]);
    cudaFuncSetAttribute(k_md<MD_THREADS, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    ProfScope ps(FP_PROF_MD_MID, s2);
    k_md<MD_THREADS, 1><<<(unsigned)ls[1].size(), MD_THREADS, sm, s2>>>(a);
    h->launches++;
  }
  if (!ls[0].empty()) {
    MdArgs a = base;
    a.nodes = dnodes + lo;
    a.nnodes_launch = (int32_t)ls[0].size();
    size_t sm = md_smem(0, mmax[0]);
    cudaFuncSetAttribute(k_md<32, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    ProfScope ps(FP_PROF_MD_SMALL, h->stream);
    k_md<32, 0><<<(unsigned)ls[0].size(), 32, sm, h->stream>>>(a);
    h->launches++;
  }
  cudaEventRecord(ev_join, s2);
  cudaStreamWaitEvent(h->stream, ev_join, 0);
  FP_CHECK_LAUNCH(h, "minimum degree");
  if (n > 0) {
    ProfScope ps(FP_PROF_PERM, h->stream);
    FP_LAUNCH(h, k_iperm, G, 256, 0, h->perm, n, h->iperm);
  }
  FP_CHECK_LAUNCH(h, "iperm");
  cudaEventDestroy(ev_fork);
  cudaEventDestroy(ev_join);
  cudaStreamDestroy(s2);
  for (void* p : {(void*)sub, (void*)nvstart, (void*)nvfill, (void*)nvlist, (void*)loc, (void*)tmp, (void*)dup,
                  (void*)grows, (void*)gs})
    dev_free(h, p);
  return FP_OK;
}

void launch_dof_expand_perm(fp_handle* h, const int32_t* perm, int32_t* perm_d, int32_t* iperm_d) {
  const int64_t N = (int64_t)h->n * h->b;
  if (N == 0) return;
  ProfScope ps(FP_PROF_PERM, h->stream);
  FP_LAUNCH(h, k_dof_perm, grid_for(N, 256), 256, 0, perm, h->n, h->b, perm_d, iperm_d);
}

void launch_dof_expand_symbolic(fp_handle* h, const int32_t* parent, const int32_t* colcount, int32_t* parent_d,
                                int32_t* colcount_d) {
  const int64_t N = (int64_t)h->n * h->b;
  if (N == 0) return;
  ProfScope ps(FP_PROF_PERM, h->stream);
  FP_LAUNCH(h, k_dof_symbolic, grid_for(N, 256), 256, 0, parent, colcount, h->n, h->b, parent_d, colcount_d);
}

}  // namespace fp
