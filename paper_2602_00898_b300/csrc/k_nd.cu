// a3 quotient graph and a4 patch-guided nested dissection (Section 4.2;
// Algorithm 2 GetSeparator; Section 5 "Quotient graph computation" and
// "Separator set computation").
//
// The quotient graph (patches as nodes, edge weight = number of G-edges between
// two patches) is built once; each tree level then
//   1. bisects every node's patch set on the quotient graph (one CTA per node:
//      components by smallest patch id, pseudo-peripheral start r1 from two
//      BFS sweeps, order by (BFS level from r1, id), left = first ceil(m/2));
//   2. lifts the bisection to the vertices: the superset is every remaining
//      vertex with a neighbour on the other side (vertex-parallel);
//   3. refines it to the lexicographically-first maximal independent set of the
//      crossing graph under the key (cdeg, tie_hash, id) -- Jacobi "local
//      minimum" rounds in one cooperative launch; the unreleased rest is the
//      separator (a minimal vertex cover of the crossing edges);
//   4. removes the separator from the quotient graph by decrementing node and
//      edge weights (each crossing G-edge once), and moves the other vertices
//      and patches to the children 2t+1 / 2t+2.
// All nodes of one depth are processed by the same launches; the host never
// waits inside the level loop.
#include <algorithm>
#include <cooperative_groups.h>

#include "fp_device.cuh"

namespace cg = cooperative_groups;

namespace fp {
namespace {

constexpr int QCAP = 4096;          // cross-edge entries of one patch sorted on chip
constexpr int ND_THREADS = 256;
constexpr int ND_BATCH = 8;
// Tree depths whose separators are ordered early. Measured on B300 (median
// step): the root alone gives icosphere-7 5.46 -> 5.19 ms and the 1M-vertex
// torus 14.10 -> 12.42 ms; two levels 5.18 / 13.27 ms, four 5.39 / 14.72 ms
// (the extra CTAs hold whole SMs while the dissection needs them).
constexpr int EARLY_LEVELS = 1;
constexpr int EARLY_CTAS = (1 << EARLY_LEVELS) - 1;  // at most that many early ordering CTAs
constexpr int8_t VS_NONE = 0, VS_UND = 1, VS_IN = 2, VS_OUT = 3;

// ---- generic counting sort helpers ----------------------------------------------------
// Keys outside [koff, koff + nk) are skipped (-1, or a tree node at another
// depth: in a fused batch the meshes' subtrees start at different depths).
__global__ void k_count_by(const int32_t* __restrict__ key, int32_t n, int32_t koff, int32_t nk,
                           int32_t* __restrict__ cnt) {
  FP_PDL_WAIT();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t c = (uint32_t)(key[i] - koff);
    if (c < (uint32_t)nk) atomicAdd(&cnt[c], 1);
  }
}

__global__ void k_scatter_by(const int32_t* __restrict__ key, int32_t n, int32_t koff, int32_t nk,
                             const int32_t* __restrict__ start, int32_t* __restrict__ fill,
                             int32_t* __restrict__ list) {
  FP_PDL_WAIT();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t c = (uint32_t)(key[i] - koff);
    if (c < (uint32_t)nk) list[start[c] + atomicAdd(&fill[c], 1)] = i;
  }
}

// The three steps above in one CTA (one launch) when the keys span at most
// GROUP_SMALL_MAX values: counts in shared memory, their exclusive scan, then
// the scatter. start gets nk+1 entries; list order within a key is arbitrary.
constexpr int GROUP_SMALL_MAX = 8192;
__global__ void __launch_bounds__(1024) k_group_small(const int32_t* __restrict__ key, int32_t n, int32_t koff,
                                                      int32_t nk, int32_t* __restrict__ start,
                                                      int32_t* __restrict__ list, int32_t* __restrict__ zero4) {
  FP_PDL_WAIT();
  extern __shared__ int32_t gsm[];
  __shared__ int32_t red[40];
  int32_t* cnt = gsm;          // [nk]
  int32_t* pos = gsm + nk;     // [nk]
  if (zero4 && threadIdx.x < 4) zero4[threadIdx.x] = 0;   // the caller's next counters
  for (int32_t i = threadIdx.x; i < nk; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const uint32_t c = (uint32_t)(key[i] - koff);
    if (c < (uint32_t)nk) atomicAdd(&cnt[c], 1);
  }
  __syncthreads();
  int32_t carry = 0;
  for (int32_t b = 0; b < nk; b += blockDim.x) {
    const int32_t i = b + threadIdx.x;
    const int32_t x = i < nk ? cnt[i] : 0;
    int32_t tot;
    const int32_t ex = block_excl_scan_i32(x, &tot, red) + carry;
    if (i < nk) {
      start[i] = ex;
      pos[i] = ex;
    }
    carry += tot;
  }
  if (threadIdx.x == 0) start[nk] = carry;
  __syncthreads();
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const uint32_t c = (uint32_t)(key[i] - koff);
    if (c < (uint32_t)nk) list[atomicAdd(&pos[c], 1)] = i;
  }
}

// ---- a3 quotient graph --------------------------------------------------------------
// One CTA per patch: gather the patch ids across its cross edges, sort them on
// chip and run-length encode, in one pass: the row (neighbour patches and edge
// weights) goes to a scratch stretch taken with one atomic, its length to
// qdeg; after the scan of qdeg, k_quotient_pack moves every row into place.
__global__ void __launch_bounds__(ND_THREADS) k_quotient_rows(const int32_t* __restrict__ pstart,
                                                              const int32_t* __restrict__ pverts,
                                                              const int32_t* __restrict__ rowptr,
                                                              const int32_t* __restrict__ col,
                                                              const int32_t* __restrict__ gmap, int32_t k,
                                                              int32_t* __restrict__ qdeg, int32_t* __restrict__ qtoff,
                                                              int32_t* __restrict__ tcol, int32_t* __restrict__ tw,
                                                              int32_t* tctr, int32_t* status,
                                                              int8_t* __restrict__ bnd) {
  FP_PDL_WAIT();
  __shared__ int32_t buf[QCAP];
  __shared__ int32_t starts[QCAP + 1];
  __shared__ int32_t red[40];
  __shared__ int32_t cnt, s_off;
  for (int32_t p = blockIdx.x; p < k; p += gridDim.x) {
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int32_t i = pstart[p] + threadIdx.x; i < pstart[p + 1]; i += blockDim.x) {
      const int32_t v = pverts[i];
      bool outside = false;
      for_row_gather<8>(rowptr, col, v, gmap, [&](int32_t, int32_t q) {
        if (q != p) {
          outside = true;
          int32_t s = atomicAdd(&cnt, 1);
          if (s < QCAP) buf[s] = q;
        }
      });
      bnd[v] = outside;        // on its patch's boundary
    }
    __syncthreads();
    const int32_t L = cnt;
    if (L > QCAP) {
      if (threadIdx.x == 0) {
        atomicOr(status, ST_QUOTIENT_TOO_BIG);
        qdeg[p] = 0;
        qtoff[p] = 0;
      }
      __syncthreads();
      continue;
    }
    const int N = pow2_at_least(L, 32);
    for (int i = L + threadIdx.x; i < N; i += blockDim.x) buf[i] = INT_MAX;
    __syncthreads();
    bitonic_sort<true>(buf, N, threadIdx.x, blockDim.x);
    int32_t base = 0;
    for (int32_t i0 = 0; i0 < L; i0 += blockDim.x) {
      int32_t i = i0 + threadIdx.x;
      int32_t f = (i < L && (i == 0 || buf[i] != buf[i - 1])) ? 1 : 0;
      int32_t tot;
      int32_t ex = block_excl_scan_i32(f, &tot, red);
      if (f) starts[base + ex] = i;
      base += tot;
    }
    if (threadIdx.x == 0) {
      starts[base] = L;
      qdeg[p] = base;
      s_off = base > 0 ? atomicAdd(tctr, base) : 0;
      qtoff[p] = s_off;
    }
    __syncthreads();
    const int32_t o = s_off;
    for (int32_t j = threadIdx.x; j < base; j += blockDim.x) {
      tcol[o + j] = buf[starts[j]];
      tw[o + j] = starts[j + 1] - starts[j];
    }
    __syncthreads();
  }
}

// Rows from the scratch stretches to their places q_rowptr[p]: one warp per
// patch.
__global__ void k_quotient_pack(const int32_t* __restrict__ q_rowptr, const int32_t* __restrict__ qdeg,
                                const int32_t* __restrict__ qtoff, const int32_t* __restrict__ tcol,
                                const int32_t* __restrict__ tw, int32_t k, int32_t* __restrict__ q_col,
                                int32_t* __restrict__ q_w) {
  FP_PDL_WAIT();
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < k; p += nwarps) {
    const int32_t d = qdeg[p], o = q_rowptr[p], t = qtoff[p];
    for (int32_t j = lane; j < d; j += 32) {
      q_col[o + j] = tcol[t + j];
      q_w[o + j] = tw[t + j];
    }
  }
}

// ---- a4 step 1: bisection of every node's patch set ----------------------------------

struct BisectArgs {
  int32_t t0, T;
  const int32_t* npstart;
  int32_t* nplist;
  int32_t* sortbuf;            // [2k + 64]
  const int32_t* q_rowptr;
  const int32_t* q_col;
  const int32_t* q_w;
  const int32_t* patch_node;
  int32_t* loc;                // [k] patch -> local index
  int32_t* ldeg;               // [k] by list position
  int32_t* lbeg;               // [k] by list position: row start in ladj
  int32_t* ladj;               // [Q] local adjacency inside each patch's quotient row
  int32_t* lvl;                // [k]
  int32_t* qa;                 // [k] frontier
  int32_t* qb;                 // [k] frontier
  int8_t* mark;                // [k] 0 untouched, 2 current component, 1 done
  int32_t* hist;               // [k]
  int32_t* side;               // [k] by patch id
  int32_t* split;              // [T]
  int8_t* cross;               // [k] by patch id: some local neighbour lies on the other side
  int32_t mcap, ecap;          // shared-memory staging limits of this launch
  int32_t k;                   // patches
  int32_t smem_ints;           // dynamic shared memory of the launch, in ints
  const int32_t* w;            // [k] remaining vertices of every patch
  int32_t cap_log;             // a child of a node at this depth keeps at most 2^cap_log patches
  int32_t* status;             // k_nd_bisect_warp: ST_NODE_TOO_BIG for a node above 32 patches
};

// Per-node working set: in shared memory when the node has <= mcap patches and
// <= ecap local adjacency entries, else in the global arrays at the node's
// list offset.
struct BisectView {
  int32_t* L;
  int32_t *lvl, *qa, *qb, *hist, *rbeg, *rlen, *adj;
  int8_t* mark;
  int8_t* sd;                  // side by local index (shared-memory layout only)
};

// Level-synchronous BFS over the node's local quotient graph from local `src`.
// lvl must be -1 on the component. Returns the number of levels. One barrier
// per level: level l reads its frontier size from scnt[l % 3], appends to
// scnt[(l + 1) % 3] and clears scnt[(l + 2) % 3], which nobody touches during
// level l. Eight lanes share a frontier patch, one edge each per round, so a
// patch's claims go out together instead of one after another; a warp's
// claims (four patches) are appended with one shared atomic, their offsets
// from a ballot. The levels do not depend on the order of the claims.
constexpr int BFS_LANES = 8;
__device__ int block_bfs(const BisectView& v, int32_t src, int32_t* scnt) {
  int32_t* fa = v.qa;
  int32_t* fb = v.qb;
  if (threadIdx.x == 0) {
    v.lvl[src] = 0;
    fa[0] = src;
    scnt[0] = 1;
    scnt[1] = 0;
    scnt[2] = 0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int sub = lane / BFS_LANES, k = lane % BFS_LANES;
  constexpr int PER_WARP = 32 / BFS_LANES;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int level = 0;
  for (;;) {
    const int32_t nf = scnt[level % 3];
    if (nf == 0) break;
    if (threadIdx.x == 0) scnt[(level + 2) % 3] = 0;
    int32_t* nxt_cnt = &scnt[(level + 1) % 3];
    // warp-uniform sweep: PER_WARP frontier patches a warp per pass
    for (int32_t i0 = warp * PER_WARP; i0 < nf; i0 += nwarps * PER_WARP) {
      const int32_t i = i0 + sub;
      int32_t e0 = 0, len = 0;
      if (i < nf) {
        const int32_t u = fa[i];
        e0 = v.rbeg[u];
        len = v.rlen[u];
      }
      for (int32_t e = k; __any_sync(0xffffffffu, e < len); e += BFS_LANES) {
        const int32_t w = e < len ? v.adj[e0 + e] : -1;
        const bool got = w >= 0 && atomicCAS(&v.lvl[w], -1, level + 1) == -1;
        const unsigned bb = __ballot_sync(0xffffffffu, got);
        int32_t o = 0;
        if (lane == 0 && bb) o = atomicAdd(nxt_cnt, __popc(bb));
        o = __shfl_sync(0xffffffffu, o, 0);
        if (got) fb[o + __popc(bb & lt)] = w;
      }
    }
    __syncthreads();
    int32_t* t = fa; fa = fb; fb = t;
    ++level;
  }
  return level;
}

__global__ void __launch_bounds__(1024) k_nd_bisect(BisectArgs a) {
  FP_PDL_WAIT();
  extern __shared__ __align__(16) int32_t bsm[];
  __shared__ int64_t red64[40];
  __shared__ int32_t red[40];
  __shared__ int32_t scnt[3];
  __shared__ int32_t s_lstar, s_rem, s_jstar;
  __shared__ int64_t s_cumw;
  for (int32_t ni = blockIdx.x; ni < a.T; ni += gridDim.x) {
    const int32_t t = a.t0 + ni;
    const int32_t base = a.npstart[ni];
    const int32_t m = a.npstart[ni + 1] - base;
    int32_t* Lg = a.nplist + base;
    if (m < 2) {
      if (threadIdx.x == 0) a.split[ni] = 0;
      continue;
    }
    if (threadIdx.x == 0) a.split[ni] = 1;
    // sort the node's patches by id (local index order = id order): marks in
    // a bitmap over all patch ids, read back in order through prefix
    // popcounts, when it fits in shared memory and is not much longer than
    // the node (a fused batch has many patch ids); else a bitonic sort
    const int32_t kw = (a.k + 31) >> 5;
    if (2 * (int64_t)kw <= a.smem_ints && (kw <= 1024 || kw <= 8 * m)) {
      uint32_t* bm = reinterpret_cast<uint32_t*>(bsm);
      int32_t* pre = bsm + kw;
      for (int32_t w = threadIdx.x; w < kw; w += blockDim.x) bm[w] = 0u;
      __syncthreads();
      for (int32_t i = threadIdx.x; i < m; i += blockDim.x) {
        const int32_t p = Lg[i];
        atomicOr(&bm[p >> 5], 1u << (p & 31));
      }
      __syncthreads();
      int32_t carry = 0;
      for (int32_t w0 = 0; w0 < kw; w0 += blockDim.x) {
        const int32_t w = w0 + threadIdx.x;
        const int32_t c = w < kw ? __popc(bm[w]) : 0;
        int32_t tot;
        const int32_t ex = block_excl_scan_i32(c, &tot, red);
        if (w < kw) pre[w] = carry + ex;
        carry += tot;
      }
      __syncthreads();
      for (int32_t w = threadIdx.x; w < kw; w += blockDim.x) {
        uint32_t x = bm[w];
        int32_t r = pre[w];
        while (x) {
          const int32_t id = w * 32 + __ffs(x) - 1;
          x &= x - 1;
          Lg[r] = id;
          a.loc[id] = r++;
        }
      }
      __syncthreads();
    } else {
      int32_t* sb = (m <= a.mcap) ? bsm : a.sortbuf + 2 * (int64_t)base;
      const int N = pow2_at_least(m, 2);
      for (int32_t i = threadIdx.x; i < N; i += blockDim.x) sb[i] = i < m ? Lg[i] : INT_MAX;
      __syncthreads();
      bitonic_sort<true>(sb, N, threadIdx.x, blockDim.x);
      for (int32_t i = threadIdx.x; i < m; i += blockDim.x) Lg[i] = sb[i];
      __syncthreads();
      for (int32_t i = threadIdx.x; i < m; i += blockDim.x) a.loc[Lg[i]] = i;
      __syncthreads();
    }
    // local quotient subgraph: neighbours in this node with remaining edge weight
    int32_t E = 0;
    if (m == a.k) {
      // the root holding every patch: its local graph is the quotient graph
      // itself (local index = patch id, every patch in this node, and before
      // the first separator every edge has weight), copied edge by edge
      E = a.q_rowptr[m];
      for (int32_t e = threadIdx.x; e < E; e += blockDim.x) a.ladj[e] = a.q_col[e];
      for (int32_t i = threadIdx.x; i < m; i += blockDim.x) {
        const int32_t e0 = a.q_rowptr[i];
        a.ldeg[base + i] = a.q_rowptr[i + 1] - e0;
        a.lbeg[base + i] = e0;
      }
      __syncthreads();
    } else {
      for (int32_t i = threadIdx.x; i < m; i += blockDim.x) {
        const int32_t p = Lg[i];
        int32_t c = 0;
        const int32_t e0 = a.q_rowptr[p], e1 = a.q_rowptr[p + 1];
        // ND_BATCH quotient edges per round: their ends and weights, then the
        // ends' node and local index
        for (int32_t eb = e0; eb < e1; eb += ND_BATCH) {
          int32_t q[ND_BATCH], wq[ND_BATCH], nq[ND_BATCH], lq[ND_BATCH];
#pragma unroll
          for (int k = 0; k < ND_BATCH; ++k) {
            q[k] = eb + k < e1 ? a.q_col[eb + k] : -1;
            wq[k] = eb + k < e1 ? a.q_w[eb + k] : 0;
          }
#pragma unroll
          for (int k = 0; k < ND_BATCH; ++k) {
            const bool live = q[k] >= 0 && wq[k] > 0;
            nq[k] = live ? a.patch_node[q[k]] : -1;
            lq[k] = live ? a.loc[q[k]] : 0;
          }
#pragma unroll
          for (int k = 0; k < ND_BATCH; ++k)
            if (nq[k] == t) a.ladj[e0 + c++] = lq[k];
        }
        a.ldeg[base + i] = c;
        a.lbeg[base + i] = e0;
        E += c;
      }
      E = block_sum(E, red);
    }
    const bool sm = m <= a.mcap && E <= a.ecap;
    BisectView v;
    if (sm) {
      // shared layout: lvl, qa, qb, hist (row lengths), rbeg [mcap+1], adj
      // [ecap] as int32, then mark [mcap] as int8; the patch ids stay in
      // global memory (read only to write the sides)
      int32_t* q = bsm;
      v.L = Lg;
      v.lvl = q; q += a.mcap;
      v.qa = q; q += a.mcap;
      v.qb = q; q += a.mcap;
      v.hist = q; q += a.mcap;
      v.rbeg = q; q += a.mcap + 1;
      v.rlen = a.ldeg + base;        // read once below into the compact rows
      v.adj = q;
      v.mark = (int8_t*)(q + a.ecap);
      v.sd = v.mark + a.mcap;
      // compact CSR in shared memory
      int32_t carry = 0;
      for (int32_t i0 = 0; i0 < m; i0 += blockDim.x) {
        const int32_t i = i0 + threadIdx.x;
        const int32_t c = i < m ? a.ldeg[base + i] : 0;
        int32_t tot;
        const int32_t ex = block_excl_scan_i32(c, &tot, red);
        if (i < m) v.rbeg[i] = carry + ex;
        carry += tot;
      }
      __syncthreads();
      for (int32_t i = threadIdx.x; i < m; i += blockDim.x) {
        const int32_t e0 = a.lbeg[base + i], c = a.ldeg[base + i], o = v.rbeg[i];
        for (int32_t j = 0; j < c; ++j) v.adj[o + j] = a.ladj[e0 + j];
        v.hist[i] = a.ldeg[base + i];   // row lengths, kept in shared memory
      }
      v.rlen = v.hist;
      // hist doubles as the row-length array; the split histogram uses qb's
      // sibling region below once the BFS sweeps are done (see `hist2`).
    } else {
      v.L = Lg;
      v.lvl = a.lvl + base;
      v.qa = a.qa + base;
      v.qb = a.qb + base;
      v.mark = a.mark + base;
      v.hist = a.hist + base;
      v.rbeg = a.lbeg + base;
      v.rlen = a.ldeg + base;
      v.adj = a.ladj;
      v.sd = nullptr;
    }
    for (int32_t i = threadIdx.x; i < m; i += blockDim.x) {
      v.lvl[i] = -1;
      v.mark[i] = 0;
    }
    __syncthreads();
    // R8 balance: the cut j of the node's order (the number of patches on
    // the left) minimises |2 P_j - W| over J = [lo, hi], P_j the weight of
    // the first j patches, ties to the smaller j. The cost is unimodal in j,
    // so the answer is the first crossing (2 P_j >= W) or the patch before
    // it, clamped into J. Components come in order; the cut is fixed in the
    // component holding the crossing (or at hi, if that comes first), and
    // every component is then assigned against the cut.
    int32_t lo = 1, hi = m - 1;
    if (a.cap_log < 30) {
      const int32_t c = 1 << a.cap_log;
      const int32_t l2 = m - c > 1 ? m - c : 1, h2 = m - 1 < c ? m - 1 : c;
      if (l2 <= h2) { lo = l2; hi = h2; }
    }
    int64_t W = -1;            // the node's weight, once needed
    int32_t jstar = lo == hi ? lo : -1;   // the cut, once fixed
    int32_t pos = 0;           // patches ordered before this component
    int64_t posw = 0;          // and their weight
    for (;;) {
      // next component: smallest untouched local index
      int32_t c0 = INT_MAX;
      for (int32_t i = threadIdx.x; i < m; i += blockDim.x)
        if (v.mark[i] == 0) { c0 = i; break; }
      c0 = block_min(c0, red);
      if (c0 == INT_MAX) break;
      // the sweep from r0 = min (degree, id) of c0's component: tried first
      // from the minimum over all untouched patches, which is r0 whenever its
      // sweep reaches c0 (the usual, connected case), so that the discovery
      // sweep is needed only when the minimum lies in another component
      int64_t best = INT64_MAX;
      for (int32_t i = threadIdx.x; i < m; i += blockDim.x)
        if (v.mark[i] == 0) {
          const int64_t key = ((int64_t)v.rlen[i] << 32) | i;
          best = key < best ? key : best;
        }
      const int32_t ra = (int32_t)(block_min(best, red64) & 0xffffffff);
      int32_t nl0 = block_bfs(v, ra, scnt);
      if (v.lvl[c0] >= 0) {
        // ra's component is c0's: its levels are those of the sweep from r0 = ra
        for (int32_t i = threadIdx.x; i < m; i += blockDim.x)
          if (v.mark[i] == 0 && v.lvl[i] >= 0) v.mark[i] = 2;
        __syncthreads();
      } else {
        for (int32_t i = threadIdx.x; i < m; i += blockDim.x)
          if (v.mark[i] == 0 && v.lvl[i] >= 0) v.lvl[i] = -1;
        __syncthreads();
        // sweep 0: discover c0's component
        block_bfs(v, c0, scnt);
        best = INT64_MAX;
        for (int32_t i = threadIdx.x; i < m; i += blockDim.x)
          if (v.mark[i] == 0 && v.lvl[i] >= 0) {
            v.mark[i] = 2;
            v.lvl[i] = -1;
            const int64_t key = ((int64_t)v.rlen[i] << 32) | i;
            best = key < best ? key : best;
          }
        const int32_t r0 = (int32_t)(block_min(best, red64) & 0xffffffff);
        // sweep 1: from r0 (minimum degree, then id)
        nl0 = block_bfs(v, r0, scnt);
      }
      // r1 = min (degree, id) on the last level of the sweep from r0
      best = INT64_MAX;
      for (int32_t i = threadIdx.x; i < m; i += blockDim.x)
        if (v.mark[i] == 2 && v.lvl[i] == nl0 - 1) {
          const int64_t key = ((int64_t)v.rlen[i] << 32) | i;
          best = key < best ? key : best;
        }
      const int32_t r1 = (int32_t)(block_min(best, red64) & 0xffffffff);
      for (int32_t i = threadIdx.x; i < m; i += blockDim.x)
        if (v.mark[i] == 2) v.lvl[i] = -1;
      __syncthreads();
      // sweep 2: the order of the component is (level from r1, id)
      block_bfs(v, r1, scnt);
      // count and weight of the component in one reduction
      int64_t pk = 0;
      for (int32_t i = threadIdx.x; i < m; i += blockDim.x)
        if (v.mark[i] == 2) pk += ((int64_t)1 << 32) | (uint32_t)a.w[v.L[i]];
      pk = block_sum(pk, red64);
      const int32_t cs = (int32_t)(pk >> 32);
      const int64_t cw = pk & 0xffffffffll;
      // left-set rule of this component: lvl < lstar, or lvl == lstar and
      // (local index < istar, or == istar when incl); -1 = by count below
      int32_t d_lstar = -1, d_istar = 0, d_incl = 0;
      if (jstar < 0) {
        if (W < 0) {
          if (pos == 0 && cs == m) {
            W = cw;
          } else {
            int32_t ws = 0;
            for (int32_t i = threadIdx.x; i < m; i += blockDim.x) ws += a.w[v.L[i]];
            W = block_sum(ws, red);
          }
        }
        if (2 * (posw + cw) >= W) {
          // the crossing lies in this component: levels by weight (and
          // count), then the patches of the crossing level in id order
          const int64_t T2 = W - 2 * posw;        // > 0: need 2 * (prefix) >= T2
          int32_t* hc = v.qa;                     // counts per level
          int32_t* hw = v.qb;                     // weights per level
          for (int32_t i = threadIdx.x; i < m; i += blockDim.x) { hc[i] = 0; hw[i] = 0; }
          __syncthreads();
          for (int32_t i = threadIdx.x; i < m; i += blockDim.x)
            if (v.mark[i] == 2) { atomicAdd(&hc[v.lvl[i]], 1); atomicAdd(&hw[v.lvl[i]], a.w[v.L[i]]); }
          __syncthreads();
          if (threadIdx.x == 0) {
            int64_t cumw = 0;
            int32_t cumc = 0, l = 0;
            while (2 * (cumw + hw[l]) < T2) { cumw += hw[l]; cumc += hc[l]; ++l; }
            s_lstar = l;
            s_rem = cumc;
            s_cumw = cumw;
            s_jstar = hc[l];
          }
          __syncthreads();
          const int32_t lstar = s_lstar, cumc = s_rem, nlev = s_jstar;
          const int64_t cumw = s_cumw;
          int32_t beforew = 0;
          for (int32_t i0 = 0; i0 < m; i0 += blockDim.x) {
            const int32_t i = i0 + threadIdx.x;
            const bool at = i < m && v.mark[i] == 2 && v.lvl[i] == lstar;
            const int32_t wi = at ? a.w[v.L[i]] : 0;
            int32_t totw;
            const int32_t exw = block_excl_scan_i32(wi, &totw, red) + beforew;
            if (at && 2 * (cumw + exw) < T2 && 2 * (cumw + exw + wi) >= T2) {
              // the first patch whose prefix reaches half the weight: keep it
              // on the left iff that cut is strictly closer to the half
              const int64_t p1 = posw + cumw + exw + wi;
              s_lstar = i;
              s_rem = (2 * p1 - W) < (W - 2 * (p1 - wi)) ? 1 : 0;
            }
            beforew += totw;
          }
          __syncthreads();
          const int32_t istar = s_lstar, incl = s_rem;
          // the cut's position j0 lies in [pos + cumc, pos + cumc + nlev];
          // its exact rank is needed only when the clamp may bind
          int32_t j0lo = pos + cumc, j0hi = pos + cumc + nlev;
          if (j0lo < lo || j0hi > hi) {
            int32_t r = 0;
            for (int32_t i = threadIdx.x; i < istar; i += blockDim.x) r += v.mark[i] == 2 && v.lvl[i] == lstar;
            r = block_sum(r, red);
            const int32_t j0 = pos + cumc + r + incl;
            jstar = j0 < lo ? lo : (j0 > hi ? hi : j0);
            if (jstar == j0) { d_lstar = lstar; d_istar = istar; d_incl = incl; }
          } else {
            jstar = INT_MAX;          // fixed by the rule below, inside this component
            d_lstar = lstar; d_istar = istar; d_incl = incl;
          }
        } else if (hi <= pos + cs) {
          jstar = hi;       // the crossing comes later, the cut stops at hi
        }
      }
      if (d_lstar >= 0) {
        for (int32_t i = threadIdx.x; i < m; i += blockDim.x)
          if (v.mark[i] == 2) {
            const int32_t lv = v.lvl[i];
            const int32_t sd = (lv < d_lstar || (lv == d_lstar && (i < d_istar || (d_incl && i == d_istar)))) ? 0 : 1;
            a.side[v.L[i]] = sd;
            if (v.sd) v.sd[i] = (int8_t)sd;
            v.mark[i] = 1;
          }
        if (jstar == INT_MAX) jstar = pos;  // every later component goes right
      } else if (jstar < 0 || pos + cs <= jstar || pos >= jstar) {
        const int32_t sd = (jstar >= 0 && pos >= jstar) ? 1 : 0;
        for (int32_t i = threadIdx.x; i < m; i += blockDim.x)
          if (v.mark[i] == 2) {
            a.side[v.L[i]] = sd;
            if (v.sd) v.sd[i] = (int8_t)sd;
            v.mark[i] = 1;
          }
      } else {
        // the cut falls inside the component: its first `need` patches in
        // (level, id) order go left; levels histogram in the frontier buffer
        // qa (free after the sweeps)
        const int32_t need = jstar - pos;
        int32_t* hist2 = v.qa;
        for (int32_t i = threadIdx.x; i < m; i += blockDim.x) hist2[i] = 0;
        __syncthreads();
        for (int32_t i = threadIdx.x; i < m; i += blockDim.x)
          if (v.mark[i] == 2) atomicAdd(&hist2[v.lvl[i]], 1);
        __syncthreads();
        if (threadIdx.x == 0) {
          int32_t cum = 0, l = 0;
          while (cum + hist2[l] < need) { cum += hist2[l]; ++l; }
          s_lstar = l;
          s_rem = need - cum;
        }
        __syncthreads();
        const int32_t lstar = s_lstar, rem = s_rem;
        int32_t before = 0;
        for (int32_t i0 = 0; i0 < m; i0 += blockDim.x) {
          const int32_t i = i0 + threadIdx.x;
          int32_t lv = -2, mk = 0;
          if (i < m) { mk = v.mark[i]; lv = v.lvl[i]; }
          const int32_t f = (mk == 2 && lv == lstar) ? 1 : 0;
          int32_t tot;
          const int32_t ex = block_excl_scan_i32(f, &tot, red) + before;
          if (mk == 2) {
            const int32_t sd = (lv < lstar || (lv == lstar && ex < rem)) ? 0 : 1;
            a.side[v.L[i]] = sd;
            if (v.sd) v.sd[i] = (int8_t)sd;
            v.mark[i] = 1;
          }
          before += tot;
        }
      }
      pos += cs;
      posw += cw;
      __syncthreads();
    }
    // crossing patches: a neighbour of positive weight in this node on the
    // other side (only their vertices can be superset vertices)
    if (v.sd) __syncthreads();     // the shared sides are complete
    for (int32_t i = threadIdx.x; i < m; i += blockDim.x) {
      int8_t c = 0;
      const int32_t rb = v.rbeg[i], re = rb + v.rlen[i];
      if (v.sd) {
        const int8_t si = v.sd[i];
        for (int32_t e = rb; e < re; ++e) c |= (int8_t)(v.sd[v.adj[e]] != si);
      } else {
        const int32_t si = a.side[v.L[i]];
        for (int32_t e = rb; e < re; ++e) c |= (int8_t)(a.side[v.L[v.adj[e]]] != si);
      }
      a.cross[v.L[i]] = c;
    }
    __syncthreads();
  }
}

// ---- a4 steps 2-4 on the vertices -----------------------------------------------------------------

struct LevelArgs {
  int32_t n, t0, T;
  const int32_t* rowptr;
  const int32_t* col;
  const int32_t* gmap;
  int32_t* node_of;
  int8_t* final_;
  const int32_t* side;
  const int32_t* split;
  int32_t* cdeg;
  int8_t* vstate;
  int32_t* cand;
  int2* cand_x;                // per candidate: start of its crossing list, cdeg
  int32_t* xcol;               // [nnz] crossing neighbours of v at rowptr[v]..
  int32_t* ctr;                // [0] candidates, [1..3] MIS round flags
  int32_t* w;
  const int32_t* q_rowptr;
  const int32_t* q_col;
  int32_t* q_w;
  int32_t* patch_node;
  int32_t k;
  const int8_t* cross;         // [k] crossing patches of this level (k_nd_bisect)
  const int8_t* bnd;           // [n] the vertex has a neighbour in another patch
  SegView sv;                  // fused batch: tie hashes of mesh-local vertex numbers
};

// SuperSeparator (Algorithm 2 step 3): remaining vertices of a split node with
// a neighbour on the other side. Vertices of nodes that are leaves at this
// depth become final.
__global__ void k_nd_superset(LevelArgs a) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += gridDim.x * blockDim.x) {
    if (a.final_[v]) continue;
    const int32_t t = a.node_of[v];
    if ((uint32_t)(t - a.t0) >= (uint32_t)a.T) continue;     // a subtree that starts deeper
    if (!a.split[t - a.t0]) { a.final_[v] = 1; continue; }
    const int32_t pv = a.gmap[v];
    // no neighbour across in its patch's quotient row, or none of its own
    // neighbours in another patch (those of its own patch are on its side):
    // not a candidate (its cdeg and state are not read this level)
    if (!a.cross[pv] || !a.bnd[v]) continue;
    const int32_t sv = a.side[pv];
    int32_t c = 0;
    // neighbours in batches of ND_BATCH: col, then node and patch, then side;
    // the crossing ones are listed in v's own row range of xcol, so that the
    // refinement rounds read only them
    const int32_t eb = a.rowptr[v], e1 = a.rowptr[v + 1];
    for (int32_t e0 = eb; e0 < e1; e0 += ND_BATCH) {
      int32_t u[ND_BATCH], nt[ND_BATCH], sd[ND_BATCH];
#pragma unroll
      for (int k = 0; k < ND_BATCH; ++k) u[k] = e0 + k < e1 ? a.col[e0 + k] : -1;
#pragma unroll
      for (int k = 0; k < ND_BATCH; ++k) {
        nt[k] = u[k] >= 0 ? a.node_of[u[k]] : -1;
        sd[k] = u[k] >= 0 ? a.gmap[u[k]] : 0;
      }
#pragma unroll
      for (int k = 0; k < ND_BATCH; ++k) sd[k] = nt[k] == t ? a.side[sd[k]] : sv;
#pragma unroll
      for (int k = 0; k < ND_BATCH; ++k)
        if (nt[k] == t && sd[k] != sv) a.xcol[eb + c++] = u[k];
    }
    a.cdeg[v] = c;
    a.vstate[v] = c ? VS_UND : VS_NONE;
    if (c) {
      const unsigned act = __activemask();
      const int lane = threadIdx.x & 31, leader = __ffs(act) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(&a.ctr[0], __popc(act));
      base = __shfl_sync(act, base, leader);
      const int32_t slot = base + __popc(act & lanemask_lt());
      a.cand[slot] = v;
      a.cand_x[slot] = make_int2(eb, c);
    }
  }
}

__device__ __forceinline__ bool key_less(int32_t cu, int32_t u, int32_t cv, int32_t v, const SegView& sv) {
  if (cu != cv) return cu < cv;
  const uint32_t hu = tie_hash(seg_local(sv, u)), hv = tie_hash(seg_local(sv, v));
  if (hu != hv) return hu < hv;
  return u < v;
}

constexpr int MIS_CACHE = 2, MIS_NB = 8;

// RefineSeparator (Algorithm 2 step 4): lexicographically-first maximal
// independent set of the crossing graph in increasing (cdeg, tie_hash, id).
// A candidate joins (IN = released to its side) when no crossing neighbour is IN
// and every undecided crossing neighbour has a larger key; it leaves (OUT =
// separator) once a crossing neighbour is IN. Monotone, so concurrent updates
// within a round only delay decisions; at most #candidates rounds.
__global__ void __launch_bounds__(ND_THREADS) k_nd_mis(LevelArgs a) {
  FP_PDL_WAIT();
  cg::grid_group grid = cg::this_grid();
  const int32_t nc = __ldcg(&a.ctr[0]);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 == 0) { a.ctr[1] = 0; a.ctr[2] = 0; a.ctr[3] = 0; }
  // The thread's first MIS_CACHE candidates with at most MIS_NB crossing
  // neighbours keep, for every round, their neighbours and which of them
  // precede them in the key order in registers (a candidate's own state is
  // written by its thread only): a round then reads just the neighbours'
  // states. The others re-read everything each round.
  int32_t cv[MIS_CACHE], nb[MIS_CACHE][MIS_NB];
  uint32_t before[MIS_CACHE];
  bool cached[MIS_CACHE], und[MIS_CACHE];
#pragma unroll
  for (int c = 0; c < MIS_CACHE; ++c) {
    const int64_t i = t0 + c * stride;
    cv[c] = i < nc ? __ldcg(&a.cand[i]) : -1;
    const int2 x = i < nc ? __ldcg(&a.cand_x[i]) : make_int2(0, MIS_NB + 1);
    cached[c] = x.y <= MIS_NB;
    und[c] = cached[c];
#pragma unroll
    for (int k = 0; k < MIS_NB; ++k) nb[c][k] = cached[c] && k < x.y ? __ldcg(&a.xcol[x.x + k]) : -1;
    int32_t cd[MIS_NB];
#pragma unroll
    for (int k = 0; k < MIS_NB; ++k) cd[k] = nb[c][k] >= 0 ? a.cdeg[nb[c][k]] : 0;
    before[c] = 0;
#pragma unroll
    for (int k = 0; k < MIS_NB; ++k)
      if (nb[c][k] >= 0 && key_less(cd[k], nb[c][k], x.y, cv[c], a.sv)) before[c] |= 1u << k;
  }
  grid.sync();
  for (int32_t round = 0; round <= nc; ++round) {
    if (t0 == 0) a.ctr[1 + (round + 1) % 3] = 0;
    int32_t undecided = 0;
#pragma unroll
    for (int c = 0; c < MIS_CACHE; ++c) {
      if (!und[c]) continue;
      int8_t st[MIS_NB];
#pragma unroll
      for (int k = 0; k < MIS_NB; ++k)
        st[k] = nb[c][k] >= 0 ? *(volatile int8_t*)&a.vstate[nb[c][k]] : (int8_t)VS_NONE;
      bool any_in = false, is_min = true;
#pragma unroll
      for (int k = 0; k < MIS_NB; ++k) {
        if (st[k] == VS_IN) any_in = true;
        else if (st[k] == VS_UND && (before[c] >> k & 1u)) is_min = false;
      }
      if (any_in) { a.vstate[cv[c]] = VS_OUT; und[c] = false; }
      else if (is_min) { a.vstate[cv[c]] = VS_IN; und[c] = false; }
      else ++undecided;
    }
    int32_t c = 0;
    for (int64_t i = t0; i < nc; i += stride, ++c) {
      if (c < MIS_CACHE && cached[c]) continue;
      const int32_t v = __ldcg(&a.cand[i]);
      const int2 x = __ldcg(&a.cand_x[i]);
      if (*(volatile int8_t*)&a.vstate[v] != VS_UND) continue;
      const int32_t cdv = x.y;
      bool any_in = false, is_min = true;
      // the crossing neighbours listed by k_nd_superset, ND_BATCH at a time
      for (int32_t j = 0; j < cdv && !any_in; j += ND_BATCH) {
        int32_t u[ND_BATCH];
#pragma unroll
        for (int k = 0; k < ND_BATCH; ++k) u[k] = j + k < cdv ? __ldcg(&a.xcol[x.x + j + k]) : -1;
        int8_t st[ND_BATCH];
        int32_t cd[ND_BATCH];
#pragma unroll
        for (int k = 0; k < ND_BATCH; ++k) {
          st[k] = u[k] >= 0 ? *(volatile int8_t*)&a.vstate[u[k]] : (int8_t)VS_NONE;
          cd[k] = u[k] >= 0 ? a.cdeg[u[k]] : 0;
        }
#pragma unroll
        for (int k = 0; k < ND_BATCH; ++k) {
          if (st[k] == VS_IN) any_in = true;
          else if (st[k] == VS_UND && key_less(cd[k], u[k], cdv, v, a.sv)) is_min = false;
        }
      }
      if (any_in) a.vstate[v] = VS_OUT;
      else if (is_min) a.vstate[v] = VS_IN;
      else ++undecided;
    }
    if (undecided) atomicAdd(&a.ctr[1 + round % 3], undecided);
    grid.sync();
    if (__ldcg(&a.ctr[1 + round % 3]) == 0) break;
  }
}

// Separator bookkeeping (Section 5): the OUT vertices stay in node t as its
// separator; patch weights and quotient edge weights lose them.
__global__ void k_nd_apply(LevelArgs a) {
  FP_PDL_WAIT();
  const int32_t nc = a.ctr[0];
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const int32_t v = a.cand[i];
    if (a.vstate[v] != VS_OUT) continue;
    a.final_[v] = 1;
    const int32_t pv = a.gmap[v], t = a.node_of[v];
    atomicSub(&a.w[pv], 1);
    const int32_t pb = a.q_rowptr[pv], pe = a.q_rowptr[pv + 1];
    // ND_BATCH edges per round: their ends, then the ends' node, patch and
    // state, then both quotient entries of every qualifying edge by binary
    // searches run in lockstep (independent loads per step)
    const int32_t e1 = a.rowptr[v + 1];
    for (int32_t e0 = a.rowptr[v]; e0 < e1; e0 += ND_BATCH) {
      int32_t u[ND_BATCH], pu[ND_BATCH], nt[ND_BATCH];
      int8_t st[ND_BATCH];
#pragma unroll
      for (int k = 0; k < ND_BATCH; ++k) u[k] = e0 + k < e1 ? a.col[e0 + k] : -1;
#pragma unroll
      for (int k = 0; k < ND_BATCH; ++k) {
        pu[k] = u[k] >= 0 ? a.gmap[u[k]] : -1;
        nt[k] = u[k] >= 0 ? a.node_of[u[k]] : -1;
        st[k] = u[k] >= 0 ? a.vstate[u[k]] : (int8_t)VS_NONE;
      }
      int32_t lo1[ND_BATCH], hi1[ND_BATCH], lo2[ND_BATCH], hi2[ND_BATCH];
      bool any = false;
#pragma unroll
      for (int k = 0; k < ND_BATCH; ++k) {
        // an edge to another patch of the same node; one between two
        // separator vertices is counted from its smaller-id end only
        const bool q = u[k] >= 0 && nt[k] == t && pu[k] != pv && !(st[k] == VS_OUT && u[k] < v);
        if (!q) u[k] = -1;
        any |= q;
        lo1[k] = pb;
        hi1[k] = q ? pe : pb;
        lo2[k] = q ? a.q_rowptr[pu[k]] : 0;
        hi2[k] = q ? a.q_rowptr[pu[k] + 1] : 0;
      }
      if (!any) continue;
      for (;;) {
        bool more = false;
        int32_t m1[ND_BATCH], m2[ND_BATCH], c1[ND_BATCH], c2[ND_BATCH];
#pragma unroll
        for (int k = 0; k < ND_BATCH; ++k) {
          m1[k] = (lo1[k] + hi1[k]) >> 1;
          m2[k] = (lo2[k] + hi2[k]) >> 1;
          c1[k] = lo1[k] < hi1[k] ? a.q_col[m1[k]] : 0;
          c2[k] = lo2[k] < hi2[k] ? a.q_col[m2[k]] : 0;
        }
#pragma unroll
        for (int k = 0; k < ND_BATCH; ++k) {
          if (lo1[k] < hi1[k]) {
            if (c1[k] < pu[k]) lo1[k] = m1[k] + 1; else hi1[k] = m1[k];
          }
          if (lo2[k] < hi2[k]) {
            if (c2[k] < pv) lo2[k] = m2[k] + 1; else hi2[k] = m2[k];
          }
          more |= lo1[k] < hi1[k] || lo2[k] < hi2[k];
        }
        if (!more) break;
      }
#pragma unroll
      for (int k = 0; k < ND_BATCH; ++k)
        if (u[k] >= 0) {
          atomicSub(&a.q_w[lo1[k]], 1);
          atomicSub(&a.q_w[lo2[k]], 1);
        }
    }
  }
}

// LeftRight (Algorithm 2 step 5): the remaining vertices of a split node move to
// child 2t+1 (left) or 2t+2 (right) with their patch.
// The patches follow: a split node's patch moves with its side, others drop out
// (one launch, threads cover both ranges).
__global__ void k_nd_move_patches(LevelArgs a) {
  FP_PDL_WAIT();
  const int32_t span = a.n > a.k ? a.n : a.k;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < span; i += gridDim.x * blockDim.x) {
    if (i < a.n && !a.final_[i]) {
      const int32_t t = a.node_of[i];
      if ((uint32_t)(t - a.t0) < (uint32_t)a.T) a.node_of[i] = 2 * t + 1 + a.side[a.gmap[i]];
    }
    if (i < a.k) {
      const int32_t t = a.patch_node[i];
      if ((uint32_t)(t - a.t0) < (uint32_t)a.T)
        a.patch_node[i] = (a.split[t - a.t0] && a.w[i] > 0) ? 2 * t + 1 + a.side[i] : -1;
    }
  }
}


// Bisection of nodes of at most 32 K patches (the deep levels, where the
// subtree capacity bounds every node by 2^(Dsplit-d) patches): one warp a
// node, the node's patches in id order as local indices j * 32 + lane (lane
// holds K of them), each one's local quotient neighbours as a K-word mask,
// BFS levels by OR-reductions of the frontier's masks. The same rule as
// k_nd_bisect (R8: components by smallest id, r0 and r1 by (degree, id),
// order by (level from r1, id), the weighted cut clamped to the subtree
// capacity), decided with warp votes and reductions instead of CTA barriers.
constexpr int BW_WARPS = 8;

// (degree << 8 | local index) keys: the least among `in`, as a local index
// (-1 if none)
template <int K>
__device__ __forceinline__ int32_t warp_argmin_key(const bool (&in)[K], const uint32_t (&key)[K]) {
  uint32_t best = 0xffffffffu;
#pragma unroll
  for (int j = 0; j < K; ++j) best = in[j] && key[j] < best ? key[j] : best;
  const uint32_t k = __reduce_min_sync(0xffffffffu, best);
  return k == 0xffffffffu ? -1 : (int32_t)(k & 0xffu);
}

// Level-synchronous BFS from local index src over the patches with lvl == -1
// (src among them); sets their levels and returns the number of levels.
template <int K>
__device__ __forceinline__ int32_t warp_bfs(const uint32_t (&adj)[K][K], int32_t (&lvl)[K], int32_t src) {
  const int lane = threadIdx.x & 31;
  uint32_t unv[K], front[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    unv[j] = __ballot_sync(0xffffffffu, lvl[j] == -1);
    front[j] = j == (src >> 5) ? 1u << (src & 31) : 0u;
    if (j == (src >> 5) && lane == (src & 31)) lvl[j] = 0;
    unv[j] &= ~front[j];
  }
  int32_t level = 0;
  for (;;) {
    uint32_t any = 0u;
#pragma unroll
    for (int j = 0; j < K; ++j) any |= front[j];
    if (!any) break;
    uint32_t nxt[K];
#pragma unroll
    for (int w = 0; w < K; ++w) {
      uint32_t acc = 0u;
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (front[j] >> lane & 1u) acc |= adj[j][w];
      nxt[w] = __reduce_or_sync(0xffffffffu, acc) & unv[w];
    }
    ++level;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (nxt[j] >> lane & 1u) lvl[j] = level;
      unv[j] &= ~nxt[j];
      front[j] = nxt[j];
    }
  }
  return level;
}

template <int K>
__global__ void __launch_bounds__(BW_WARPS * 32) k_nd_bisect_warp(BisectArgs a) {
  FP_PDL_WAIT();
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int MAXM = 32 * K;
  __shared__ int32_t s_ids[BW_WARPS][MAXM];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned ltm = (1u << lane) - 1u;
  for (int32_t ni = blockIdx.x * BW_WARPS + wid; ni < a.T; ni += gridDim.x * BW_WARPS) {
    const int32_t t = a.t0 + ni;
    const int32_t base = a.npstart[ni];
    const int32_t m = a.npstart[ni + 1] - base;
    if (m < 2 || m > MAXM) {
      // (above MAXM patches the subtree capacity was not met: flagged, and
      // the ordering stage reports it before any result is used)
      if (lane == 0) {
        a.split[ni] = 0;
        if (m > MAXM) atomicOr(a.status, ST_NODE_TOO_BIG);
      }
      continue;
    }
    if (lane == 0) a.split[ni] = 1;
    int32_t* Lg = a.nplist + base;
    // id order: every id's rank among the node's ids, then local index r
    // takes rank r
    int32_t myid[K], rank[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      myid[j] = j * 32 + lane < m ? Lg[j * 32 + lane] : INT_MAX;
      rank[j] = 0;
    }
#pragma unroll
    for (int jj = 0; jj < K; ++jj)
      for (int src = 0; src < 32; ++src) {
        const int32_t o = __shfl_sync(FULL, myid[jj], src);
#pragma unroll
        for (int j = 0; j < K; ++j) rank[j] += o < myid[j];
      }
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j * 32 + lane < m) s_ids[wid][rank[j]] = myid[j];
    __syncwarp();
    int32_t p[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int32_t i = j * 32 + lane;
      p[j] = i < m ? s_ids[wid][i] : -1;
      if (i < m) {
        Lg[i] = p[j];
        a.loc[p[j]] = i;
      }
    }
    __syncwarp();
    // neighbours in this node with remaining edge weight, ND_BATCH a round
    uint32_t adj[K][K];
    int32_t w[K], lvl[K], mark[K], sd[K];
    uint32_t key[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
#pragma unroll
      for (int x = 0; x < K; ++x) adj[j][x] = 0u;
      const int32_t i = j * 32 + lane;
      if (i < m) {
        const int32_t e0 = a.q_rowptr[p[j]], e1 = a.q_rowptr[p[j] + 1];
        for (int32_t eb = e0; eb < e1; eb += ND_BATCH) {
          int32_t q[ND_BATCH], wq[ND_BATCH], nq[ND_BATCH], lq[ND_BATCH];
#pragma unroll
          for (int k = 0; k < ND_BATCH; ++k) {
            q[k] = eb + k < e1 ? a.q_col[eb + k] : -1;
            wq[k] = eb + k < e1 ? a.q_w[eb + k] : 0;
          }
#pragma unroll
          for (int k = 0; k < ND_BATCH; ++k) {
            const bool live = q[k] >= 0 && wq[k] > 0;
            nq[k] = live ? a.patch_node[q[k]] : -1;
            lq[k] = live ? a.loc[q[k]] : 0;
          }
#pragma unroll
          for (int k = 0; k < ND_BATCH; ++k)
            if (nq[k] == t) {
#pragma unroll
              for (int x = 0; x < K; ++x)
                if ((lq[k] >> 5) == x) adj[j][x] |= 1u << (lq[k] & 31);
            }
        }
      }
      int32_t dg = 0;
#pragma unroll
      for (int x = 0; x < K; ++x) dg += __popc(adj[j][x]);
      w[j] = i < m ? a.w[p[j]] : 0;
      key[j] = ((uint32_t)dg << 8) | (uint32_t)i;
      lvl[j] = i < m ? -1 : -2;
      mark[j] = i < m ? 0 : 1;           // 0 untouched, 2 this component, 1 done
      sd[j] = 0;
    }
    auto lvl_of = [&](int32_t i) -> int32_t {   // the level of local index i (all lanes)
      int32_t v = 0;
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (j == (i >> 5)) v = lvl[j];
      return __shfl_sync(FULL, v, i & 31);
    };
    int32_t lo = 1, hi = m - 1;
    if (a.cap_log < 30) {
      const int32_t c = 1 << a.cap_log;
      const int32_t l2 = m - c > 1 ? m - c : 1, h2 = m - 1 < c ? m - 1 : c;
      if (l2 <= h2) { lo = l2; hi = h2; }
    }
    int64_t W = -1;
    int32_t jstar = lo == hi ? lo : -1;
    int32_t pos = 0;
    int64_t posw = 0;
    for (;;) {
      int32_t c0 = -1;
#pragma unroll
      for (int j = K - 1; j >= 0; --j) {
        const uint32_t b = __ballot_sync(FULL, mark[j] == 0);
        if (b) c0 = j * 32 + __ffs(b) - 1;
      }
      if (c0 < 0) break;
      bool in[K];
#pragma unroll
      for (int j = 0; j < K; ++j) in[j] = mark[j] == 0;
      int32_t nl0 = warp_bfs<K>(adj, lvl, warp_argmin_key<K>(in, key));
      if (lvl_of(c0) >= 0) {
#pragma unroll
        for (int j = 0; j < K; ++j)
          if (mark[j] == 0 && lvl[j] >= 0) mark[j] = 2;
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j)
          if (mark[j] == 0 && lvl[j] >= 0) lvl[j] = -1;
        warp_bfs<K>(adj, lvl, c0);
#pragma unroll
        for (int j = 0; j < K; ++j) {
          in[j] = mark[j] == 0 && lvl[j] >= 0;
          if (in[j]) {
            mark[j] = 2;
            lvl[j] = -1;
          }
        }
        nl0 = warp_bfs<K>(adj, lvl, warp_argmin_key<K>(in, key));
      }
#pragma unroll
      for (int j = 0; j < K; ++j) in[j] = mark[j] == 2 && lvl[j] == nl0 - 1;
      const int32_t r1 = warp_argmin_key<K>(in, key);
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (mark[j] == 2) lvl[j] = -1;
      warp_bfs<K>(adj, lvl, r1);
      bool cur[K];
      int32_t cs = 0;
      uint32_t cwl = 0u;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        cur[j] = mark[j] == 2;
        cs += __popc(__ballot_sync(FULL, cur[j]));
        cwl += cur[j] ? (uint32_t)w[j] : 0u;
      }
      const int64_t cw = (int64_t)__reduce_add_sync(FULL, cwl);
      int32_t d_lstar = -1, d_istar = 0, d_incl = 0;
      if (jstar < 0) {
        if (W < 0) {
          uint32_t wl = 0u;
#pragma unroll
          for (int j = 0; j < K; ++j) wl += (uint32_t)w[j];
          W = (pos == 0 && cs == m) ? cw : (int64_t)__reduce_add_sync(FULL, wl);
        }
        if (2 * (posw + cw) >= W) {
          // the crossing lies in this component: levels by weight (and
          // count), then the patches of the crossing level in id order
          const int64_t T2 = W - 2 * posw;
          int64_t cumw = 0;
          int32_t cumc = 0, l = 0, nlev = 0;
          for (; l < MAXM; ++l) {                 // levels <= m
            uint32_t hwl = 0u;
            int32_t hc = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) {
              const bool at = cur[j] && lvl[j] == l;
              hwl += at ? (uint32_t)w[j] : 0u;
              hc += __popc(__ballot_sync(FULL, at));
            }
            const int64_t hw = (int64_t)__reduce_add_sync(FULL, hwl);
            if (2 * (cumw + hw) < T2) {
              cumw += hw;
              cumc += hc;
            } else {
              nlev = hc;
              break;
            }
          }
          const int32_t lstar = l;
          // the first patch of the level (in id order) whose prefix weight
          // reaches half; keep it on the left iff that cut is strictly closer
          // to the half
          int32_t istar = -1, incl = 0, carry = 0;
#pragma unroll
          for (int j = 0; j < K; ++j) {
            const bool at = cur[j] && lvl[j] == lstar;
            const int32_t wi = at ? w[j] : 0;
            int32_t inc = wi;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const int32_t y = __shfl_up_sync(FULL, inc, o);
              if (lane >= o) inc += y;
            }
            const int32_t exw = carry + inc - wi;
            const bool hit = at && 2 * (cumw + exw) < T2 && 2 * (cumw + exw + wi) >= T2;
            int32_t my_incl = 0;
            if (hit) {
              const int64_t p1 = posw + cumw + exw + wi;
              my_incl = (2 * p1 - W) < (W - 2 * (p1 - wi)) ? 1 : 0;
            }
            const uint32_t hb = __ballot_sync(FULL, hit);
            if (istar < 0 && hb) {
              const int src = __ffs(hb) - 1;
              istar = j * 32 + src;
              incl = __shfl_sync(FULL, my_incl, src);
            }
            carry += __shfl_sync(FULL, inc, 31);
          }
          if (istar < 0) istar = 0;
          const int32_t j0lo = pos + cumc, j0hi = pos + cumc + nlev;
          if (j0lo < lo || j0hi > hi) {
            int32_t r = 0;
#pragma unroll
            for (int j = 0; j < K; ++j)
              r += __popc(__ballot_sync(FULL, cur[j] && lvl[j] == lstar && j * 32 + lane < istar));
            const int32_t j0 = pos + cumc + r + incl;
            jstar = j0 < lo ? lo : (j0 > hi ? hi : j0);
            if (jstar == j0) { d_lstar = lstar; d_istar = istar; d_incl = incl; }
          } else {
            jstar = INT_MAX;          // fixed by the rule below, inside this component
            d_lstar = lstar; d_istar = istar; d_incl = incl;
          }
        } else if (hi <= pos + cs) {
          jstar = hi;                 // the crossing comes later, the cut stops at hi
        }
      }
      if (d_lstar >= 0) {
#pragma unroll
        for (int j = 0; j < K; ++j)
          if (cur[j]) {
            const int32_t i = j * 32 + lane;
            sd[j] = (lvl[j] < d_lstar || (lvl[j] == d_lstar && (i < d_istar || (d_incl && i == d_istar)))) ? 0 : 1;
            mark[j] = 1;
          }
        if (jstar == INT_MAX) jstar = pos;   // every later component goes right
      } else if (jstar < 0 || pos + cs <= jstar || pos >= jstar) {
#pragma unroll
        for (int j = 0; j < K; ++j)
          if (cur[j]) {
            sd[j] = (jstar >= 0 && pos >= jstar) ? 1 : 0;
            mark[j] = 1;
          }
      } else {
        // the cut falls inside the component: its first `need` patches in
        // (level, id) order go left
        const int32_t need = jstar - pos;
        int32_t cum = 0, l = 0;
        for (; l < MAXM; ++l) {
          int32_t hc = 0;
#pragma unroll
          for (int j = 0; j < K; ++j) hc += __popc(__ballot_sync(FULL, cur[j] && lvl[j] == l));
          if (cum + hc < need) cum += hc; else break;
        }
        int32_t before = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const uint32_t atm = __ballot_sync(FULL, cur[j] && lvl[j] == l);
          const int32_t ex = before + __popc(atm & ltm);
          if (cur[j]) {
            sd[j] = (lvl[j] < l || (lvl[j] == l && ex < need - cum)) ? 0 : 1;
            mark[j] = 1;
          }
          before += __popc(atm);
        }
      }
      pos += cs;
      posw += cw;
    }
    // sides, and the crossing patches (a local neighbour on the other side)
    uint32_t right[K];
#pragma unroll
    for (int j = 0; j < K; ++j) right[j] = __ballot_sync(FULL, j * 32 + lane < m && sd[j] == 1);
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j * 32 + lane < m) {
        uint32_t c = 0u;
#pragma unroll
        for (int x = 0; x < K; ++x) c |= adj[j][x] & (sd[j] ? ~right[x] : right[x]);
        a.side[p[j]] = sd[j];
        a.cross[p[j]] = (int8_t)(c != 0u);
      }
  }
}

// Stage record (debug_dump) of one level's bisection: the side of every patch
// of a split node at this depth, -1 for the others.
__global__ void k_stage_sides(const int32_t* __restrict__ patch_node, const int32_t* __restrict__ side,
                              const int32_t* __restrict__ split, int32_t t0, int32_t T, int32_t k,
                              int32_t* __restrict__ out) {
  FP_PDL_WAIT();
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x) {
    const int32_t t = patch_node[p];
    out[p] = (t >= t0 && t < t0 + T && split[t - t0]) ? side[p] : -1;
  }
}

__global__ void k_patch_node_init(const int32_t* __restrict__ psize, int32_t k, int32_t* __restrict__ patch_node) {
  FP_PDL_WAIT();
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x)
    patch_node[p] = psize[p] > 0 ? 0 : -1;
}

__global__ void k_zero_i8(int8_t* p, int64_t n) {
  FP_PDL_WAIT();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 0;
}

int ceil_log2(int64_t k) {
  int d = 0;
  while (((int64_t)1 << d) < k) ++d;
  return d;
}

// ---- fused batch: the meshes' subtrees -------------------------------------------------
// pmesh[p]: the mesh of patch p (every vertex of a patch lies in one mesh).
__global__ void k_patch_mesh(const int32_t* __restrict__ gmap, const int32_t* __restrict__ vmesh, int32_t n,
                             int32_t* __restrict__ pmesh) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) pmesh[gmap[v]] = vmesh[v];
}

__global__ void k_mesh_patch_count(const int32_t* __restrict__ pmesh, int32_t k, int32_t* __restrict__ kcount) {
  FP_PDL_WAIT();
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x)
    atomicAdd(&kcount[pmesh[p]], 1);
}

// Every vertex and every patch starts at the root of its mesh's subtree.
__global__ void k_seg_roots(const int32_t* __restrict__ vmesh, const int32_t* __restrict__ pmesh,
                            const int32_t* __restrict__ psize, const int32_t* __restrict__ mroot, int32_t n, int32_t k,
                            int32_t* __restrict__ node_of, int32_t* __restrict__ patch_node) {
  FP_PDL_WAIT();
  const int32_t span = n > k ? n : k;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < span; i += gridDim.x * blockDim.x) {
    if (i < n) node_of[i] = mroot[vmesh[i]];
    if (i < k) patch_node[i] = psize[i] > 0 ? mroot[pmesh[i]] : -1;
  }
}

// Places the meshes' subtrees of a fused batch (after patching): mesh m with
// k_m patches needs a subtree of height h_m = ceil(log2 k_m), the depth one
// mesh alone is dissected to. Its root goes to depth l_m = D - h_m, with D the
// smallest depth whose Kraft sum sum_m 2^(h_m - D) is at most 1, as the
// canonical prefix code of the lengths l_m (largest subtree first, then mesh
// index); every leaf then lies at depth D. Leaves pmesh [k] on the device
// for the root initialisation, sets h->D, the roots and the meshes' position
// ranges (their left-to-right order in the tree).
fp_status seg_plan(fp_handle* h, int32_t** pmesh_out) {
  Segments* sg = h->seg;
  const int32_t n = h->n, k = h->k, M = sg->M;
  int32_t* pmesh = (int32_t*)dev_alloc(h, sizeof(int32_t) * (size_t)(k > 0 ? k : 1));
  int32_t* kc = (int32_t*)dev_alloc(h, sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
  int32_t* hk = pinned_ints(M);
  if (!pmesh || !kc || !hk) return fail(h, FP_ERR_OUT_OF_MEMORY, "batch plan");
  fill_i32(h, kc, 0, M);
  fill_i32(h, pmesh, 0, k);          // (every patch has a vertex; kept in range regardless)
  FP_LAUNCH(h, k_patch_mesh, grid_for(n, 256), 256, 0, h->gmap, sg->v.vmesh, n, pmesh);
  FP_LAUNCH(h, k_mesh_patch_count, grid_for(k, 256), 256, 0, pmesh, k, kc);
  cudaMemcpyAsync(hk, kc, sizeof(int32_t) * (size_t)M, cudaMemcpyDeviceToHost, h->stream);
  FP_CHECK_LAUNCH(h, "batch plan");
  int32_t st = 0;
  FP_TRY(sync_status(h, &st));
  dev_free(h, kc);
  sg->h_k.assign(hk, hk + M);
  std::vector<int32_t> hm(M, -1), order;
  int64_t S = 0;
  for (int32_t m = 0; m < M; ++m)
    if (sg->h_k[m] > 0) {
      hm[m] = ceil_log2(sg->h_k[m]);
      S += (int64_t)1 << hm[m];
      order.push_back(m);
    }
  const int32_t D = ceil_log2(S > 0 ? S : 1);
  if (D > 24) return fail(h, FP_ERR_UNSUPPORTED, "fused batch tree deeper than 24 levels");
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return hm[a] > hm[b]; });
  sg->h_root.assign(M, -1);
  sg->h_posoff.assign(M, 0);
  int64_t code = -1;
  int32_t lprev = 0, pos = 0;
  sg->dmin = order.empty() ? D : D - hm[order[0]];
  for (int32_t m : order) {
    const int32_t l = D - hm[m];
    code = code < 0 ? 0 : (code + 1) << (l - lprev);
    lprev = l;
    sg->h_root[m] = (int32_t)(((int64_t)1 << l) - 1 + code);
    sg->h_posoff[m] = pos;
    pos += sg->h_voff[m + 1] - sg->h_voff[m];
  }
  h->D = D;
  int32_t* hr = pinned_ints(M);
  if (!hr) return fail(h, FP_ERR_OUT_OF_MEMORY, "batch plan");
  for (int32_t m = 0; m < M; ++m) hr[m] = sg->h_root[m] < 0 ? 0 : sg->h_root[m];
  cudaMemcpyAsync(sg->mroot, hr, sizeof(int32_t) * (size_t)M, cudaMemcpyHostToDevice, h->stream);
  // the pinned buffer is reused by the next call on this thread: wait here
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "batch roots");
  *pmesh_out = pmesh;
  return FP_OK;
}

}  // namespace

fp_status run_nested_dissection(fp_handle* h) {
  const int32_t n = h->n, k = h->k;
  const int64_t Q = h->nnz > 0 ? h->nnz : 1;
  Segments* sg = h->seg;
  if (sg && h->opt.nd_level > 0) return fail(h, FP_ERR_UNSUPPORTED, "a fused batch takes nd_level 0");
  int32_t D = h->opt.nd_level > 0 ? h->opt.nd_level : ceil_log2(k);
  if (D > 24) return fail(h, FP_ERR_UNSUPPORTED, "nd_level above 24");
  h->D = D;
  if (n == 0) return FP_OK;
  // a fused batch: every mesh's subtree has its leaves at depth D; the levels
  // above the shallowest root hold no vertex
  int32_t* pmesh = nullptr;
  int32_t dmin = 0;
  if (sg) {
    FP_TRY(seg_plan(h, &pmesh));
    D = h->D;
    dmin = sg->dmin;
  } else {
    fill_i32(h, h->node_of, 0, n);
  }
  const int32_t Dsplit = sg ? D : (D < ceil_log2(k) ? D : ceil_log2(k));   // deeper nodes hold <= 1 patch
  // the separators of the top levels are ordered while deeper levels are cut
  FP_TRY(early_md_begin(h, sg ? 0 : (Dsplit < EARLY_LEVELS ? Dsplit : EARLY_LEVELS)));
  if (Dsplit == 0 && !sg) { FP_CHECK_LAUNCH(h, "nd init"); return FP_OK; }
  // per-level arrays hold one entry per node of the deepest cut level
  const int64_t tl = std::max<int64_t>((int64_t)k + 64, Dsplit > 0 ? ((int64_t)1 << (Dsplit - 1)) + 64 : 64);

  const int64_t kk = (int64_t)k + 64;
  int32_t *psize, *pstart, *pfill, *pverts, *qdeg, *q_rowptr, *q_col, *q_w, *ladj, *tmp, *patch_node, *w, *side, *loc;
  int32_t *ldeg, *lvl, *lbeg, *qa, *qb, *mark, *hist, *sortbuf, *npcount, *npstart, *npfill, *nplist, *split, *cdeg;
  int32_t *cand, *ctr, *xcol;
  int2* cand_x;
  int8_t *final_, *vstate, *cross, *bnd;
  Arena ar;
  auto layout = [&]() {
    psize = ar.get<int32_t>(kk); pstart = ar.get<int32_t>(kk); pfill = ar.get<int32_t>(kk);
    pverts = ar.get<int32_t>(n); qdeg = ar.get<int32_t>(kk); q_rowptr = ar.get<int32_t>(kk);
    q_col = ar.get<int32_t>(Q); q_w = ar.get<int32_t>(Q); ladj = ar.get<int32_t>(Q);
    tmp = ar.get<int32_t>(scan_tmp_ints(kk) + 8); patch_node = ar.get<int32_t>(kk); w = ar.get<int32_t>(kk);
    side = ar.get<int32_t>(kk); loc = ar.get<int32_t>(kk); ldeg = ar.get<int32_t>(kk); lvl = ar.get<int32_t>(kk);
    lbeg = ar.get<int32_t>(kk); qa = ar.get<int32_t>(kk); qb = ar.get<int32_t>(kk); mark = ar.get<int32_t>(kk);
    hist = ar.get<int32_t>(kk); sortbuf = ar.get<int32_t>(2 * kk + 64); npcount = ar.get<int32_t>(tl);
    npstart = ar.get<int32_t>(tl + 1); npfill = ar.get<int32_t>(tl); nplist = ar.get<int32_t>(kk);
    split = ar.get<int32_t>(tl); cdeg = ar.get<int32_t>(n); cand = ar.get<int32_t>(n); ctr = ar.get<int32_t>(8);
    xcol = ar.get<int32_t>(Q); cand_x = ar.get<int2>(n); final_ = ar.get<int8_t>(n); vstate = ar.get<int8_t>(n);
    cross = ar.get<int8_t>(kk); bnd = ar.get<int8_t>(n);
  };
  layout();
  if (!ar.alloc(h)) return fail(h, FP_ERR_OUT_OF_MEMORY, "nested dissection workspace");
  layout();

  const int G = grid_for(n, 256), GK = grid_for(k, 256);
  ProfScope ps_q(FP_PROF_QUOTIENT, h->stream);
  // patch vertex lists
  fill_i32(h, psize, 0, k);
  FP_LAUNCH(h, k_count_by, G, 256, 0, h->gmap, n, 0, k, psize);
  scan_exclusive(h, psize, pstart, k, tmp);
  fill_i32(h, pfill, 0, k);
  FP_LAUNCH(h, k_scatter_by, G, 256, 0, h->gmap, n, 0, k, pstart, pfill, pverts);
  // quotient graph (a3)
  const int GQ = k < NUM_SMS_B300 * 8 ? k : NUM_SMS_B300 * 8;
  // (ladj, xcol and lbeg serve as scratch here; the dissection uses them later)
  fill_i32(h, ctr, 0, 8);
  FP_LAUNCH(h, k_quotient_rows, GQ, ND_THREADS, 0, pstart, pverts, h->rowptr, h->col, h->gmap, k, qdeg, lbeg,
            ladj, xcol, ctr + 7, h->d_status, bnd);
  scan_exclusive(h, qdeg, q_rowptr, k, tmp);
  FP_LAUNCH(h, k_quotient_pack, grid_for((int64_t)k * 32, 256), 256, 0, q_rowptr, qdeg, lbeg, ladj, xcol, k, q_col,
            q_w);
  // state: every patch with vertices starts in the root; an empty one (a
  // label of a supplied patch map that no vertex carries) takes no part
  if (sg) {
    FP_LAUNCH(h, k_seg_roots, G > GK ? G : GK, 256, 0, sg->v.vmesh, pmesh, psize, sg->mroot, n, k, h->node_of,
              patch_node);
    dev_free(h, pmesh);
  } else {
    FP_LAUNCH(h, k_patch_node_init, GK, 256, 0, psize, k, patch_node);
  }
  cudaMemcpyAsync(w, psize, sizeof(int32_t) * k, cudaMemcpyDeviceToDevice, h->stream);
  FP_LAUNCH(h, k_zero_i8, G, 256, 0, final_, (int64_t)n);
  FP_LAUNCH(h, k_zero_i8, G, 256, 0, vstate, (int64_t)n);
  FP_CHECK_LAUNCH(h, "quotient graph");
  ps_q.end();
  if (h->opt.debug_dump) {
    // stage record: the quotient graph (its entry count is read back here)
    int32_t* hb = pinned_scratch();
    if (!hb) return fail(h, FP_ERR_OUT_OF_MEMORY, "stage record");
    cudaMemcpyAsync(hb, q_rowptr + k, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return check_cuda(h, e, "stage record");
    stage_dump(h, FP_STAGE_QUOTIENT_WEIGHT, 0, psize, k);
    stage_dump(h, FP_STAGE_QUOTIENT_ROWPTR, 0, q_rowptr, (int64_t)k + 1);
    stage_dump(h, FP_STAGE_QUOTIENT_COL, 0, q_col, hb[0]);
    stage_dump(h, FP_STAGE_QUOTIENT_EDGE_WEIGHT, 0, q_w, hb[0]);
  }

  int per = 0, sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_nd_mis, ND_THREADS, 0);
  const int gmis_max = sms * (per > 0 ? per : 1);

  allow_max_dynamic_smem(k_group_small);
  // the subtree capacity 2^(Dsplit-d) bounds every node's patches when the
  // depth is the patches' own (not an explicit smaller nd_level)
  const bool cap_exact = sg || Dsplit == ceil_log2(k);
  for (int32_t d = dmin; d < Dsplit; ++d) {
    const int32_t t0 = (1 << d) - 1, T = 1 << d;
    ProfScope ps_b(FP_PROF_ND_BISECT, h->stream);
    const bool grouped_small = T <= GROUP_SMALL_MAX;
    if (grouped_small) {
      // also zeroes the level's candidate and refinement counters
      FP_LAUNCH(h, k_group_small, 1, 1024, sizeof(int32_t) * 2 * (size_t)T, patch_node, k, t0, T, npstart, nplist,
                ctr);
    } else {
      fill_i32(h, npcount, 0, T);
      FP_LAUNCH(h, k_count_by, GK, 256, 0, patch_node, k, t0, T, npcount);
      scan_exclusive(h, npcount, npstart, T, tmp);
      fill_i32(h, npfill, 0, T);
      FP_LAUNCH(h, k_scatter_by, GK, 256, 0, patch_node, k, t0, T, npstart, npfill, nplist);
    }
    // a node at depth d holds at most 2^(Dsplit - d) patches (the subtree
    // capacity that bounds every cut, R8): stage that many in shared memory
    // with 7 adjacency entries per patch (quotient graphs of meshes have
    // degree ~6), up to what fits in a CTA; larger nodes (only with an
    // explicit depth below ceil(log2 k)) work in global memory
    constexpr int32_t MCAP_MAX = (225 * 1024 - 64) / (4 * 12 + 2);
    int32_t mcap = Dsplit - d >= 31 ? k : (int32_t)std::min<int64_t>(k, (int64_t)1 << (Dsplit - d));
    mcap = mcap < 32 ? 32 : (mcap > MCAP_MAX ? MCAP_MAX : mcap);
    const int32_t ecap = 7 * mcap;
    const size_t bsmem = sizeof(int32_t) * (5 * (size_t)mcap + 1 + (size_t)ecap) + 2 * (size_t)mcap;
    BisectArgs ba{t0, T, npstart, nplist, sortbuf, q_rowptr, q_col, q_w, patch_node, loc, ldeg, lbeg, ladj,
                  lvl, qa, qb, (int8_t*)mark, hist, side, split, cross, mcap, ecap, k, (int32_t)(bsmem / 4),
                  w, Dsplit - d - 1, h->d_status};
    const int GB = T < NUM_SMS_B300 * 8 ? T : NUM_SMS_B300 * 8;
    if (cap_exact && Dsplit - d <= 7) {
      // every node holds at most 2^(Dsplit-d) <= 128 patches: one warp a
      // node, one, two or four of them a lane
      const int gw = (int)std::min<int64_t>(((int64_t)T + BW_WARPS - 1) / BW_WARPS, NUM_SMS_B300 * 16);
      if (Dsplit - d <= 5) FP_LAUNCH(h, k_nd_bisect_warp<1>, gw, BW_WARPS * 32, 0, ba);
      else if (Dsplit - d == 6) FP_LAUNCH(h, k_nd_bisect_warp<2>, gw, BW_WARPS * 32, 0, ba);
      else FP_LAUNCH(h, k_nd_bisect_warp<4>, gw, BW_WARPS * 32, 0, ba);
    } else {
      // the top levels have a few large nodes, one CTA each: 1024 threads
      // make their gathers of the quotient rows (dependent L2 loads, one
      // round per blockDim patches) four times shorter
      const int bt = T <= 16 ? 1024 : ND_THREADS;
      allow_max_dynamic_smem(k_nd_bisect);
      FP_LAUNCH(h, k_nd_bisect, GB, bt, bsmem, ba);
    }
    ps_b.end();
    if (int32_t* sb = stage_buffer(h, FP_STAGE_SIDE, d, k))
      FP_LAUNCH(h, k_stage_sides, GK, 256, 0, patch_node, side, split, t0, T, k, sb);
    ProfScope ps_s(FP_PROF_ND_SEPARATOR, h->stream);
    LevelArgs la{n, t0, T, h->rowptr, h->col, h->gmap, h->node_of, final_, side, split, cdeg, vstate, cand, cand_x, xcol,
                 ctr, w, q_rowptr, q_col, q_w, patch_node, k, cross, bnd, sg ? sg->v : SegView{}};
    if (!grouped_small) fill_i32(h, ctr, 0, 4);
    FP_LAUNCH(h, k_nd_superset, G, 256, 0, la);
    {
      // at most one CTA per SM (few candidates per level, cheaper grid
      // barriers), leaving room beside the early separator ordering, whose
      // CTAs hold most of an SM's shared memory, so that the cooperative grid
      // is always co-resident
      int g = G < gmis_max ? G : gmis_max;
      if (g > NUM_SMS_B300 - 2 * EARLY_CTAS) g = NUM_SMS_B300 - 2 * EARLY_CTAS;
      void* args[] = {(void*)&la};
      cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_nd_mis, g, ND_THREADS, args, 0, h->stream);
      h->launches++;
      if (e != cudaSuccess) return check_cuda(h, e, "mis launch");
    }
    FP_LAUNCH(h, k_nd_apply, G, 256, 0, la);
    FP_LAUNCH(h, k_nd_move_patches, G > GK ? G : GK, 256, 0, la);
    FP_CHECK_LAUNCH(h, "nd level");
    stage_dump(h, FP_STAGE_CHILD, d, patch_node, k);
    // the nodes of depth d are final now
    FP_TRY(launch_early_md(h, d));
  }
  // no host sync here: a quotient overflow (ST_QUOTIENT_TOO_BIG, the patch
  // keeps no quotient edges, every node index stays in range) is reported by
  // the ordering stage's first sync, before any ordering kernel runs
  dev_free(h, ar.base);
  return FP_OK;
}

}  // namespace fp
