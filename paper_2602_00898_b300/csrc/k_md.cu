// a5 local ordering and a6 permutation assembly (Algorithm 3; Section 5
// "Concatenation and schedules"), a8 DOF expansion (Section 6.5).
//
// Layout: node sizes -> subtree sizes -> first position of every node in the
// chosen schedule (post-order: left subtree, right subtree, node; level order:
// deepest level first, node index ascending), one CTA.
//
// LocalOrder: exact minimum degree on the node's induced subgraph (the paper
// uses AMD; ties go to the smallest original vertex id, i.e. the smallest local
// index, local indices being assigned in id order). Each step takes the vertex
// of minimum (degree, local index), makes its neighbourhood a clique and
// updates the neighbours' degrees. Three kernels by node size:
//   * leaf (m <= 512, the patch leaves and small separators): the elimination
//     graph is a bit matrix in shared memory stored word-major (word w of row u
//     at R[w*S + u], S = m|1 odd so that a row's words fall in distinct banks);
//     each warp orders its own node. The arg-min reads all degrees (at most
//     eight 32-bit words a lane) and reduces across the warp; every lane holds
//     the pivot row's (at most 16) words and updates one neighbour;
//   * sparse (separators up to ~4300 vertices): separators' elimination graphs
//     stay very sparse, so each vertex keeps an adjacency list of at most
//     SP_CAP entries in shared memory; the CTA builds the lists, one warp
//     eliminates, one neighbour per lane. A list that would outgrow SP_CAP
//     flags the node, which is then redone by the global kernel;
//   * global (anything larger, or a flagged sparse node): bit rows in global
//     memory, a CTA per node.
// The leaf and sparse kernels keep the degrees packed two to a 32-bit word
// (dead vertices 0xffff). The leaf kernel finds the arg-min by a scan of all of
// them by one warp; the sparse kernel keeps the least key (degree, local
// index) of every 64 vertices and scans those (at most 70), rescanning only
// the groups whose minimum may have risen; the global kernel scans with its
// whole CTA.
// The separator kernels run on a second stream so that their long serial
// orderings overlap the leaves; the leaf kernel leaves them free SMs.
#include <algorithm>

#include "fp_device.cuh"

namespace fp {
namespace {

constexpr int MD_LEAF = 512;
constexpr int MD_MAX = 32768;
constexpr int MD_THREADS = 256;
constexpr int SP_CAP = 24;
constexpr int SP_GROUPS = 96;   // group minima the sparse kernel's arg-min reads (m <= 6144)
constexpr uint16_t DEG_DEAD = 0xffff;
constexpr size_t SMEM_MAX = 225 * 1024;

int pow2_host(int x) {
  int p = 32;
  while (p < x) p <<= 1;
  return p;
}

__global__ void k_node_sizes(const int32_t* __restrict__ node_of, int32_t n, int32_t* __restrict__ size) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) atomicAdd(&size[node_of[v]], 1);
}

__global__ void k_scatter_nodes(const int32_t* __restrict__ node_of, int32_t n, const int32_t* __restrict__ start,
                                int32_t* __restrict__ fill, int32_t* __restrict__ list) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int32_t t = node_of[v];
    list[start[t] + atomicAdd(&fill[t], 1)] = v;
  }
}

// Schedule layout (one CTA). sub: scratch [nnodes].
__global__ void k_tree_layout(int32_t D, int64_t nnodes, const int32_t* __restrict__ size, int32_t* __restrict__ sub,
                              int32_t* __restrict__ begin, int32_t schedule) {
  FP_PDL_WAIT();
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
  uint32_t* grows;            // global kernel: row storage base
  const int64_t* grow_off;    // global kernel: per launched node, word offset into grows
  int32_t* gsort;             // global kernel: sort scratch base
  const int64_t* gsort_off;   // global kernel: per launched node, int offset into gsort
  int64_t slice_bytes;        // leaf kernel: shared bytes per warp
  int32_t* overflow;          // sparse kernel: per launched node flag; global kernel: only flagged nodes
  const uint32_t* key;        // leaf kernel: per-vertex tie-break key (NULL: ties by id alone)
  int32_t* queue;             // leaf kernel: node counter the warps draw from (zeroed before launch)
  // early mode of the sparse kernel (nodes = NULL): node node_base + block,
  // size msize[t], rank inside the node written to rank_out[v] instead of
  // perm, nodes needing more than smem_avail bytes skipped, overflow[t]
  int32_t node_base;
  const int32_t* msize;
  int32_t* rank_out;
  int64_t smem_avail;
};

__host__ __device__ size_t sparse_smem(int m);

// ---- leaf kernel ---------------------------------------------------------------------

// Set bits of every 4-bit value v: their count (NIB_COUNT, 4 bits at 4v) and
// their positions in increasing order (2 bits each, 8 bits at 8(v & 7) of
// NIB_POS_LO for v < 8, of NIB_POS_HI otherwise).
__host__ __device__ constexpr uint64_t nib_positions(int v0) {
  uint64_t r = 0;
  for (int v = v0; v < v0 + 8; ++v) {
    uint64_t e = 0;
    int j = 0;
    for (int b = 0; b < 4; ++b)
      if ((v >> b) & 1) e |= (uint64_t)b << (2 * j++);
    r |= e << (8 * (v - v0));
  }
  return r;
}
__host__ __device__ constexpr uint64_t nib_counts() {
  uint64_t r = 0;
  for (int v = 0; v < 16; ++v) r |= (uint64_t)(((v >> 0) & 1) + ((v >> 1) & 1) + ((v >> 2) & 1) + ((v >> 3) & 1)) << (4 * v);
  return r;
}
constexpr uint64_t NIB_POS_LO = nib_positions(0), NIB_POS_HI = nib_positions(8), NIB_COUNT = nib_counts();
static_assert(NIB_COUNT == 0x4332322132212110ull, "nibble counts");

// e / d for 0 <= e < 2^13 and 1 <= d <= 16 as (e * ceil(2^31 / d)) >> 31: the
// rounding of the multiplier adds less than e / 2^31 < 2^-18, below the
// 1/16 that separates e / d from the next integer, so the quotient is exact.
#define FP_INV31(d) (uint32_t)((0x80000000ull + (d) - 1) / (d))
__constant__ uint32_t c_inv31[17] = {0u,          FP_INV31(1),  FP_INV31(2),  FP_INV31(3),  FP_INV31(4),
                                     FP_INV31(5),  FP_INV31(6),  FP_INV31(7),  FP_INV31(8),  FP_INV31(9),
                                     FP_INV31(10), FP_INV31(11), FP_INV31(12), FP_INV31(13), FP_INV31(14),
                                     FP_INV31(15), FP_INV31(16)};
#undef FP_INV31
__device__ __forceinline__ int div_small(int e, uint32_t inv) {
  return (int)(((unsigned long long)(uint32_t)e * inv) >> 31);
}

// Bitonic sort (Batcher, AFIPS 1968) of N <= 512 keys in shared memory by one
// warp, ascending. Each stage's compare-exchanges (at most 8 a lane) load all
// their pairs before storing any, so that their shared-memory round trips
// overlap; the code is one short loop whatever N is.
__device__ __forceinline__ void warp_sort_smem(unsigned long long* buf, int N, int lane) {
  const int half = N >> 1;
  for (int k = 2; k <= N; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int jj = __ffs(j) - 1;
      unsigned long long x[MD_LEAF / 64], y[MD_LEAF / 64];
      int ix[MD_LEAF / 64];
#pragma unroll
      for (int q = 0; q < MD_LEAF / 64; ++q) {
        const int c = lane + 32 * q;
        ix[q] = ((c >> jj) << (jj + 1)) | (c & (j - 1));
        if (c < half) {
          x[q] = buf[ix[q]];
          y[q] = buf[ix[q] + j];
        }
      }
#pragma unroll
      for (int q = 0; q < MD_LEAF / 64; ++q) {
        const int c = lane + 32 * q;
        if (c < half && ((y[q] < x[q]) == ((ix[q] & k) == 0))) {
          buf[ix[q]] = y[q];
          buf[ix[q] + j] = x[q];
        }
      }
      __syncwarp();
    }
}

// Sorts a node's m <= 512 vertices by (key, original id), writes the sorted
// list (to verts and to lv in shared memory) and every vertex's local index,
// then builds the induced graph's bit rows (R, word-major, zeroed here) and
// degrees. Each lane gathers two vertices at a time, eight neighbours each,
// so that their dependent loads (row bounds, neighbours, their node and local
// index) overlap.
template <int LEAF_GV>
__device__ __noinline__ void leaf_setup(const MdArgs& a, int32_t t, int m, int S, int W, int32_t* verts,
                                        unsigned char* mine, uint32_t* R, uint16_t* deg, int32_t* lv,
                                        int lane) {
  unsigned long long* sb = (unsigned long long*)mine;   // overlaps R
  const int N = pow2_at_least(m, 32);
  for (int i = lane; i < N; i += 32) {
    unsigned long long e = ~0ull;
    if (i < m) {
      const int32_t v = verts[i];
      e = ((unsigned long long)(a.key ? a.key[v] : 0u) << 32) | (uint32_t)v;
    }
    sb[i] = e;
  }
  __syncwarp();
  warp_sort_smem(sb, N, lane);
  // sorted by id alone (no keys): a neighbour's local index and whether it
  // lies in the node come from a binary search of the sorted list in shared
  // memory; with keys, from the global local-index and node arrays
  const bool by_id = a.key == nullptr;
  for (int i = lane; i < m; i += 32) {
    const int32_t v = (int32_t)(uint32_t)sb[i];
    lv[i] = v;
    verts[i] = v;
    if (!by_id) a.loc[v] = i;
  }
  __syncwarp();
  {
    const int nw = W * S, n4 = nw >> 2;
    uint4* R4 = (uint4*)R;
    for (int i = lane; i < n4; i += 32) R4[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = 4 * n4 + lane; i < nw; i += 32) R[i] = 0u;
  }
  const int M64 = (m + 63) & ~63;
  for (int i = m + lane; i < M64; i += 32) deg[i] = DEG_DEAD;
  __syncwarp();
  if (by_id) {
    // LEAF_GV vertices a lane per round: their edge ranges, their neighbours
    // (LEAF_GE at a time), then the searches, all independent
    constexpr int LEAF_GE = 8;
    for (int i0 = lane; i0 < m; i0 += 32 * LEAF_GV) {
      int32_t b[LEAF_GV], e[LEAF_GV], c[LEAF_GV];
#pragma unroll
      for (int s = 0; s < LEAF_GV; ++s) {
        const int i = i0 + 32 * s;
        const int32_t v = i < m ? lv[i] : 0;
        b[s] = i < m ? a.rowptr[v] : 0;
        e[s] = i < m ? a.rowptr[v + 1] : 0;
        c[s] = 0;
      }
      for (;;) {
        bool more = false;
#pragma unroll
        for (int s = 0; s < LEAF_GV; ++s) more |= b[s] < e[s];
        if (!more) break;
        int32_t u[LEAF_GV][LEAF_GE], lo[LEAF_GV][LEAF_GE];
#pragma unroll
        for (int s = 0; s < LEAF_GV; ++s)
#pragma unroll
          for (int k = 0; k < LEAF_GE; ++k) {
            u[s][k] = b[s] + k < e[s] ? a.col[b[s] + k] : -1;
            lo[s][k] = 0;
          }
        // lower bound: lo = number of list entries below u
#pragma unroll
        for (int st = MD_LEAF / 2; st > 0; st >>= 1)
#pragma unroll
          for (int s = 0; s < LEAF_GV; ++s)
#pragma unroll
            for (int k = 0; k < LEAF_GE; ++k) {
              const int j = lo[s][k] + st;
              if (j <= m && lv[j - 1] < u[s][k]) lo[s][k] = j;
            }
#pragma unroll
        for (int s = 0; s < LEAF_GV; ++s) {
          const int i = i0 + 32 * s;
#pragma unroll
          for (int k = 0; k < LEAF_GE; ++k) {
            const int j = lo[s][k];
            if (u[s][k] >= 0 && j < m && lv[j] == u[s][k]) {
              R[(j >> 5) * S + i] |= 1u << (j & 31);
              ++c[s];
            }
          }
          b[s] += LEAF_GE;
        }
      }
#pragma unroll
      for (int s = 0; s < LEAF_GV; ++s)
        if (i0 + 32 * s < m) deg[i0 + 32 * s] = (uint16_t)c[s];
    }
    return;
  }
  for (int i0 = lane; i0 < m; i0 += 64) {
    int32_t b[2], e[2], c[2] = {0, 0};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int i = i0 + 32 * s;
      const int32_t v = i < m ? lv[i] : 0;
      b[s] = i < m ? a.rowptr[v] : 0;
      e[s] = i < m ? a.rowptr[v + 1] : 0;
    }
    while (b[0] < e[0] || b[1] < e[1]) {
      int32_t u[2][8], nt[2][8], j[2][8];
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int k = 0; k < 8; ++k) u[s][k] = b[s] + k < e[s] ? a.col[b[s] + k] : -1;
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          nt[s][k] = u[s][k] >= 0 ? a.node_of[u[s][k]] : -1;
          j[s][k] = u[s][k] >= 0 ? a.loc[u[s][k]] : 0;
        }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int i = i0 + 32 * s;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (nt[s][k] == t) {
            R[(j[s][k] >> 5) * S + i] |= 1u << (j[s][k] & 31);
            ++c[s];
          }
        b[s] += 8;
      }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s)
      if (i0 + 32 * s < m) deg[i0 + 32 * s] = (uint16_t)c[s];
  }
}

// up to kWarps warps a CTA, one leaf each. Two builds: 10 warps at full
// registers for launches of about one wave, whose time is the largest leaf's
// latency, and 20 warps under the register cap that imposes (96 a thread,
// a few bytes of spill in the setup, slower steps) for launches of many
// waves, which gain the warps to hide the steps' latency. (The bound names
// no minimum of CTAs per SM: with an explicit 1 the 10-warp build ran its
// steps about 25% slower at the same register count.)
constexpr int LEAF_WARPS = 10, LEAF_WARPS_WIDE = 20;
template <int kWarps>
__global__ void __launch_bounds__(kWarps * 32) k_md_leaf(MdArgs a) {
  FP_PDL_WAIT();
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char* mine = smem + (size_t)wid * a.slice_bytes;
  // nodes are listed largest first and each warp takes the next one when it is
  // done (greedy largest-first balancing of the serial eliminations)
  for (;;) {
    int32_t li = 0;
    if (lane == 0) li = atomicAdd(a.queue, 1);
    li = __shfl_sync(0xffffffffu, li, 0);
    if (li >= a.nnodes_launch) break;
    const int32_t t = a.nodes[li];
    const int32_t m = a.node_size[t];
    const int32_t pbeg = a.node_begin[t];
    int32_t* verts = a.nvlist + a.nvstart[t];
    const int W = (m + 31) >> 5;                       // <= MD_LEAF / 32
    const int S = m | 1;
    const int M64 = (m + 63) & ~63;                    // degrees padded to whole warp reads
    uint32_t* R = (uint32_t*)mine;
    uint16_t* deg = (uint16_t*)(R + (size_t)W * S);
    uint16_t* order = deg + M64;                       // pivot of each step
    uint16_t* nb = order + ((m + 1) & ~1);             // pivot's neighbours, this step
    uint32_t* nzv = (uint32_t*)(nb + ((m + 1) & ~1));  // pivot row's non-zero words
    uint16_t* nzw = (uint16_t*)(nzv + MD_LEAF / 32);   //   and their indices
    // the sorted vertex list, during the setup only (overlaps order and nb)
    leaf_setup<kWarps == LEAF_WARPS ? 4 : 2>(a, t, m, S, W, verts, mine, R, deg, (int32_t*)order, lane);
    __syncwarp();
    const uint32_t* deg2 = (const uint32_t*)deg;
    uint32_t* degw = (uint32_t*)deg;
    const int H = M64 >> 1;
    // lanes 2w and 2w+1 (w < W) hold the alive bits of word w: dead vertices
    // are masked out of pivot rows instead of being cleared from their
    // neighbours' rows
    uint32_t alive = 0xffffffffu;
    const unsigned lt = lanemask_lt();
    for (int step = 0; step < m; ++step) {
      // arg-min of (degree, local index) over the alive vertices: every lane
      // takes the minimum of its packed degree pairs, then one warp reduction
      // (a dead vertex has degree 0xffff, above any alive one)
      uint32_t best = 0xffffffffu;
#pragma unroll
      for (int r = 0; r < MD_LEAF / 64; ++r) {
        const int j = lane + 32 * r;
        if (j < H) {
          const uint32_t d2 = deg2[j];
          const uint32_t k0 = (d2 << 16) | (uint32_t)(2 * j);
          const uint32_t k1 = (d2 & 0xffff0000u) | (uint32_t)(2 * j + 1);
          best = min(best, min(k0, k1));
        }
      }
      const int p = (int)(__reduce_min_sync(0xffffffffu, best) & 0xffffu);
      // pivot row, half a word per lane (lane 2w + h holds bits 16h.. of word
      // w): the neighbour list and the list of the non-zero words (nz of
      // them). The neighbour list offsets are an exclusive prefix sum of the
      // halves' bit counts (at most 16, five bits), taken bit plane by bit
      // plane with independent ballots.
      const int hw = lane >> 1, hh = lane & 1;
      const uint32_t word = hw < W ? (R[hw * S + p] & alive) : 0u;
      const uint32_t half = (word >> (16 * hh)) & 0xffffu;
      const int c = __popc(half);
      int ex = 0, nnb = 0;
#pragma unroll
      for (int bp = 0; bp < 5; ++bp) {
        const unsigned bb = __ballot_sync(0xffffffffu, (c >> bp) & 1);
        ex += __popc(bb & lt) << bp;
        nnb += __popc(bb) << bp;
      }
      const unsigned nzm = __ballot_sync(0xffffffffu, hh == 0 && word != 0u);
      const int nz = __popc(nzm);
      if (hh == 0 && word != 0u) {
        const int kk = __popc(nzm & lt);
        nzv[kk] = word;
        nzw[kk] = (uint16_t)hw;
      }
      {
        // the half's set bits, a nibble at a time, from the tables of the set
        // bit positions and counts of every 4-bit value (no serial bit scan)
        int off = ex;
        const int base = 32 * hw + 16 * hh;
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          const uint32_t v = (half >> (4 * n)) & 15u;
          const uint32_t pos = (uint32_t)(((v & 8u) ? NIB_POS_HI : NIB_POS_LO) >> (8 * (v & 7u))) & 0xffu;
          const int cn = (int)((NIB_COUNT >> (4 * v)) & 15u);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (j < cn) nb[off + j] = (uint16_t)(base + 4 * n + ((pos >> (2 * j)) & 3u));
          off += cn;
        }
      }
      if (hw == (p >> 5)) alive &= ~(1u << (p & 31));
      if (lane == 0) {
        order[step] = (uint16_t)p;
        deg[p] = DEG_DEAD;
      }
      const uint32_t inv = c_inv31[nz];
      __syncwarp();
      // clique, one (neighbour u, non-zero pivot word w) pair per lane, two
      // pairs a lane per round: row[u] |= row[p] \ {u} in word w, and
      // degree(u) grows by the bits added (less one, for p, in u's first
      // pair). Distinct pairs are distinct row words, so both loads go first.
      const int total = nnb * nz;
      for (int e0 = lane; e0 < total; e0 += 64) {
        const int e1 = e0 + 32;
        const bool two = e1 < total;
        const int i0 = div_small(e0, inv), k0 = e0 - i0 * nz;
        const int i1 = two ? div_small(e1, inv) : i0, k1 = two ? e1 - i1 * nz : k0;
        const int u0 = nb[i0], u1 = nb[i1];
        const int w0 = nzw[k0], w1 = nzw[k1];
        const uint32_t pv0 = nzv[k0], pv1 = nzv[k1];
        uint32_t* rp0 = R + w0 * S + u0;
        uint32_t* rp1 = R + w1 * S + u1;
        const uint32_t r0 = *rp0, r1 = two ? *rp1 : 0u;
        uint32_t n0 = pv0 & ~r0, n1 = pv1 & ~r1;
        if (w0 == (u0 >> 5)) n0 &= ~(1u << (u0 & 31));
        if (w1 == (u1 >> 5)) n1 &= ~(1u << (u1 & 31));
        if (n0) *rp0 = r0 | n0;
        const int d0 = __popc(n0) - (k0 == 0 ? 1 : 0);
        if (d0) atomicAdd(&degw[u0 >> 1], (uint32_t)d0 << ((u0 & 1) * 16));
        if (two) {
          if (n1) *rp1 = r1 | n1;
          const int d1 = __popc(n1) - (k1 == 0 ? 1 : 0);
          if (d1) atomicAdd(&degw[u1 >> 1], (uint32_t)d1 << ((u1 & 1) * 16));
        }
      }
      __syncwarp();
    }
    // positions of the node's vertices in elimination order
    for (int i = lane; i < m; i += 32) a.perm[pbeg + i] = verts[order[i]];
    __syncwarp();
  }
}

// Least key (degree << 16 | local index) of the 64 vertices of group g, by one
// warp (lane l reads the packed degree pair 32g + l).
__device__ __forceinline__ uint32_t group_min_key(const uint32_t* deg2, int g, int lane) {
  const int j = 32 * g + lane;
  const uint32_t d2 = deg2[j];
  const uint32_t k0 = (d2 << 16) | (uint32_t)(2 * j), k1 = (d2 & 0xffff0000u) | (uint32_t)(2 * j + 1);
  return __reduce_min_sync(0xffffffffu, min(k0, k1));
}

// ---- sparse kernel (separators) --------------------------------------------------------

// kGlobal: a node too large for the lists in shared memory (above about 4.5k
// vertices) keeps them in its stretch of the global row storage (L2
// resident, 48 B a vertex) and sorts in its global sort scratch; the
// degrees, pivots and group minima stay in shared memory. The same single
// warp runs the elimination; a list overflow leaves the node to the dense
// global kernel, as in shared memory.
template <bool kGlobal>
__global__ void __launch_bounds__(MD_THREADS) k_md_sparse(MdArgs a) {
  FP_PDL_WAIT();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int32_t s_ovf;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int32_t li = blockIdx.x; li < a.nnodes_launch; li += gridDim.x) {
    const int32_t t = a.nodes ? a.nodes[li] : a.node_base + li;
    const int32_t m = a.msize ? a.msize[t] : a.node_size[t];
    if (a.rank_out && (m == 0 || (int64_t)sparse_smem(m) > a.smem_avail)) continue;   // left to the regular path
    const int32_t oi = a.nodes ? li : t;                   // index of this node's overflow flag
    const int32_t pbeg = a.rank_out ? 0 : a.node_begin[t];
    int32_t* verts = a.nvlist + a.nvstart[t];
    const int M64 = (m + 63) & ~63, NG = M64 >> 6;
    // m x SP_CAP local ids (48 B rows), then [M64] degrees padded with dead
    // entries, the pivot of each step and [NG] least keys of each 64 vertices
    uint16_t* adj = kGlobal ? (uint16_t*)(a.grows + a.grow_off[li]) : (uint16_t*)smem;
    uint16_t* deg = kGlobal ? (uint16_t*)smem : adj + (size_t)m * SP_CAP;
    uint16_t* order = deg + M64;
    uint32_t* gmin = (uint32_t*)(order + ((m + 1) & ~1));
    // sort the node's vertices by original id (in shared memory the buffer
    // overlaps the lists)
    int32_t* sb = kGlobal ? a.gsort + a.gsort_off[li] : (int32_t*)smem;
    const int NS = pow2_at_least(m, 32);
    for (int i = tid; i < NS; i += blockDim.x) sb[i] = i < m ? verts[i] : INT_MAX;
    if (tid == 0) s_ovf = 0;
    __syncthreads();
    bitonic_sort<true>(sb, NS, tid, blockDim.x);
    for (int i = tid; i < m; i += blockDim.x) {
      const int32_t v = sb[i];
      verts[i] = v;
      a.loc[v] = i;
    }
    __syncthreads();
    for (int i = tid; i < m; i += blockDim.x) {
      const int32_t v = verts[i];
      int c = 0;
      // eight neighbours per round: their ids, then their node and local index
      const int32_t e1 = a.rowptr[v + 1];
      for (int32_t e0 = a.rowptr[v]; e0 < e1; e0 += 8) {
        int32_t u[8], nt[8], j[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) u[k] = e0 + k < e1 ? a.col[e0 + k] : -1;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          nt[k] = u[k] >= 0 ? a.node_of[u[k]] : -1;
          j[k] = u[k] >= 0 ? a.loc[u[k]] : 0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (nt[k] == t) {
            if (c < SP_CAP) adj[(size_t)i * SP_CAP + c] = (uint16_t)j[k];
            ++c;
          }
      }
      if (c > SP_CAP) s_ovf = 1;
      deg[i] = (uint16_t)(c < SP_CAP ? c : SP_CAP);
    }
    for (int i = m + tid; i < M64; i += blockDim.x) deg[i] = DEG_DEAD;
    __syncthreads();
    if (s_ovf) {
      if (tid == 0) a.overflow[oi] = 1;
      __syncthreads();
      continue;
    }
    const uint32_t* deg2 = (const uint32_t*)deg;
    for (int g = tid >> 5; g < NG; g += blockDim.x >> 5) {
      const uint32_t r = group_min_key(deg2, g, lane);
      if (lane == 0) gmin[g] = r;
    }
    __syncthreads();
    if (tid < 32) {
      bool ovf = false;
      for (int step = 0; step < m && !ovf; ++step) {
        // arg-min of the keys (degree << 16 | local index) over the group
        // minima; the key also gives the pivot's degree
        uint32_t best = 0xffffffffu;
        if (kGlobal) {
          for (int g = lane; g < NG; g += 32) best = min(best, gmin[g]);
        } else {
#pragma unroll
          for (int r = 0; r < SP_GROUPS / 32; ++r) {
            const int g = lane + 32 * r;
            if (g < NG) best = min(best, gmin[g]);
          }
        }
        const uint32_t pkey = __reduce_min_sync(0xffffffffu, best);
        const int p = (int)(pkey & 0xffffu);
        const int dp = (int)(pkey >> 16);
        // lane j holds the j-th neighbour of p
        // (p's row is not written during the step, and the previous step's
        // writes were ordered by its closing warp sync)
        const int mine_nb = lane < dp ? (int)adj[(size_t)p * SP_CAP + lane] : -1;
        if (lane == 0) {
          order[step] = (uint16_t)p;
          deg[p] = DEG_DEAD;
        }
        bool my_ovf = false;
        int u = -1, pos = 0, du = 0;
        union L24 { uint4 q[3]; uint16_t e[SP_CAP]; };
        L24 lu;
        uint16_t* nu = nullptr;
        // u's group minimum is read as soon as u is known: the neighbours'
        // lowerings in this step can only make a rescan it asks for
        // unnecessary, never a needed one missing (rescans are exact)
        uint32_t gmin_u = 0xffffffffu;
        if (lane < dp) {
          u = mine_nb;
          nu = adj + (size_t)u * SP_CAP;
          const uint4* su = (const uint4*)nu;
          lu.q[0] = su[0]; lu.q[1] = su[1]; lu.q[2] = su[2];
          du = deg[u];
          gmin_u = gmin[u >> 6];
        }
        // the loops run to the warp's longest list (a uniform exit, no
        // divergent branch per lane) with each lane's own entries predicated
        const int dmax = (int)__reduce_max_sync(0xffffffffu, (uint32_t)du);
        // new list: the old entries except p ...
#pragma unroll
        for (int k = 0; k < SP_CAP; ++k) {
          if (k >= dmax) break;
          if (k < du && lu.e[k] != p) nu[pos++] = lu.e[k];
        }
        // ... then p's other neighbours not yet present (broadcast one by one)
        for (int j = 0; j < dp; ++j) {
          const int y = __shfl_sync(0xffffffffu, mine_nb, j);
          bool found = !(lane < dp && y != u);
#pragma unroll
          for (int k = 0; k < SP_CAP; ++k) {
            if (k >= dmax) break;
            found |= k < du && lu.e[k] == y;
          }
          if (!found) {
            if (pos < SP_CAP) nu[pos++] = (uint16_t)y;
            else my_ovf = true;
          }
        }
        // group minima: a neighbour whose key fell lowers its group's
        // minimum; one that was its group's minimum and rose has the group
        // rescanned, as is always the pivot's group
        bool resc = false;
        int gu = 0;
        if (lane < dp) {
          deg[u] = (uint16_t)pos;
          const uint32_t kold = ((uint32_t)du << 16) | (uint32_t)u, knew = ((uint32_t)pos << 16) | (uint32_t)u;
          gu = u >> 6;
          if (knew < kold) atomicMin(&gmin[gu], knew);
          else if (knew > kold && gmin_u == kold) resc = true;
        }
        __syncwarp();
        ovf = __any_sync(0xffffffffu, my_ovf);
        unsigned rm = __ballot_sync(0xffffffffu, resc);
        const int gp = p >> 6;
        int g = gp;
        for (;;) {
          const uint32_t r = group_min_key(deg2, g, lane);
          if (lane == 0) gmin[g] = r;
          int gn = -1;
          while (rm && gn < 0) {
            const int l = __ffs(rm) - 1;
            rm &= rm - 1;
            const int c = __shfl_sync(0xffffffffu, gu, l);
            gn = c != gp ? c : -1;
          }
          if (gn < 0) break;
          g = gn;
        }
        __syncwarp();
      }
      if (ovf && lane == 0) {
        a.overflow[oi] = 1;
        s_ovf = 1;
      }
    }
    __syncthreads();
    // the elimination order, unless the node is left to the global kernel
    if (!s_ovf) {
      for (int i = tid; i < m; i += blockDim.x) {
        const int32_t v = verts[order[i]];
        if (a.rank_out) a.rank_out[v] = i;
        else a.perm[pbeg + i] = v;
      }
    }
    __syncthreads();
  }
}

// ---- global kernel -------------------------------------------------------------------

__global__ void __launch_bounds__(MD_THREADS) k_md_global(MdArgs a) {
  FP_PDL_WAIT();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t red32[40];
  __shared__ int32_t s_nnb;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int NT = blockDim.x, nw = NT >> 5;
  for (int32_t li = blockIdx.x; li < a.nnodes_launch; li += gridDim.x) {
    const int32_t t = a.nodes[li];
    if (a.overflow && !a.overflow[a.node_base < 0 ? t : li]) continue;
    const int32_t m = a.node_size[t];
    const int32_t pbeg = a.node_begin[t];
    int32_t* verts = a.nvlist + a.nvstart[t];
    const int W = (m + 31) >> 5;
    uint16_t* deg = (uint16_t*)smem;
    uint16_t* nb = deg + MD_MAX;
    uint32_t* rows = a.grows + a.grow_off[li];
    int32_t* sortbuf = a.gsort + a.gsort_off[li];
    const int NS = pow2_at_least(m, 32);
    for (int i = tid; i < NS; i += NT) sortbuf[i] = i < m ? verts[i] : INT_MAX;
    __syncthreads();
    bitonic_sort<true>(sortbuf, NS, tid, NT);
    for (int i = tid; i < m; i += NT) {
      const int32_t v = sortbuf[i];
      verts[i] = v;
      a.loc[v] = i;
    }
    __syncthreads();
    for (int64_t i = tid; i < (int64_t)m * W; i += NT) rows[i] = 0u;
    __syncthreads();
    for (int i = tid; i < m; i += NT) {
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
    __syncthreads();
    for (int step = 0; step < m; ++step) {
      uint32_t best = 0xffffffffu;
      for (int i = tid; i < m; i += NT) {
        const uint16_t dg = deg[i];
        if (dg != DEG_DEAD) {
          const uint32_t key = ((uint32_t)dg << 16) | (uint32_t)i;
          best = key < best ? key : best;
        }
      }
      const uint32_t kmin = block_min(best, red32);
      const int p = (int)(kmin & 0xffffu);
      const uint32_t* rp = rows + (size_t)p * W;
      if (wid == 0) {
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
      __syncthreads();
      const int nnb = s_nnb;
      for (int q = wid; q < nnb; q += nw) {
        const int u = nb[q];
        uint32_t* ru = rows + (size_t)u * W;
        uint32_t c = 0;
        for (int w = lane; w < W; w += 32) {
          uint32_t x = ru[w] | rp[w];
          if (w == (u >> 5)) x &= ~(1u << (u & 31));
          if (w == (p >> 5)) x &= ~(1u << (p & 31));
          ru[w] = x;
          c += __popc(x);
        }
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0) deg[u] = (uint16_t)c;
      }
      __syncthreads();
    }
    __syncthreads();
  }
}

__global__ void k_iperm(const int32_t* __restrict__ perm, int32_t n, int32_t* __restrict__ iperm) {
  FP_PDL_WAIT();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) iperm[perm[i]] = i;
}

__global__ void k_dof_perm(const int32_t* __restrict__ perm, int32_t n, int32_t b, int32_t* __restrict__ perm_d,
                           int32_t* __restrict__ iperm_d) {
  FP_PDL_WAIT();
  const int64_t N = (int64_t)n * b;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = (int32_t)(i / b), c = (int32_t)(i % b);
    const int32_t v = b * perm[k] + c;
    if (perm_d) perm_d[i] = v;
    if (iperm_d) iperm_d[v] = (int32_t)i;
  }
}

// Expands the columns [v0, v1) (vertex positions) to their DOF columns.
__global__ void k_dof_symbolic(const int32_t* __restrict__ parent, const int32_t* __restrict__ cc, int32_t v0,
                               int32_t v1, int32_t b, int32_t* __restrict__ parent_d, int32_t* __restrict__ cc_d) {
  FP_PDL_WAIT();
  const int64_t N = (int64_t)v1 * b;
  for (int64_t i = (int64_t)v0 * b + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = (int32_t)(i / b), c = (int32_t)(i % b);
    if (parent_d) parent_d[i] = c < b - 1 ? (int32_t)(i + 1) : (parent[j] < 0 ? -1 : b * parent[j]);
    if (cc_d) cc_d[i] = b * cc[j] - c;
  }
}

// ---- early separator ordering ------------------------------------------------------------

__global__ void k_early_count(const int32_t* __restrict__ node_of, int32_t n, int32_t t0, int32_t T,
                              int32_t* __restrict__ cnt) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int32_t t = node_of[v];
    if (t >= t0 && t < t0 + T) atomicAdd(&cnt[t], 1);
  }
}

// List offsets of the level's nodes after the lists of earlier levels (*base).
__global__ void k_early_starts(const int32_t* __restrict__ cnt, int32_t t0, int32_t T, int32_t* base,
                               int32_t* __restrict__ start, int32_t* __restrict__ fill) {
  FP_PDL_WAIT();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int32_t b = *base;
    for (int32_t i = 0; i < T; ++i) {
      start[t0 + i] = b;
      fill[t0 + i] = 0;
      b += cnt[t0 + i];
    }
    *base = b;
  }
}

__global__ void k_early_scatter(const int32_t* __restrict__ node_of, int32_t n, int32_t t0, int32_t T,
                                const int32_t* __restrict__ start, int32_t* __restrict__ fill,
                                int32_t* __restrict__ list) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int32_t t = node_of[v];
    if (t >= t0 && t < t0 + T) list[start[t] + atomicAdd(&fill[t], 1)] = v;
  }
}

// Places the early orders: every vertex of an early node that the sparse
// kernel finished goes to its node's first position plus its rank.
__global__ void k_early_place(const int32_t* __restrict__ node_of, int32_t n, int32_t NE,
                              const int32_t* __restrict__ node_size, const int32_t* __restrict__ node_begin,
                              const int32_t* __restrict__ rank, const int32_t* __restrict__ ovf,
                              int32_t* __restrict__ perm, int64_t smem_max) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int32_t t = node_of[v];
    if (t < NE && (int64_t)sparse_smem(node_size[t]) <= smem_max && !ovf[t]) perm[node_begin[t] + rank[v]] = v;
  }
}

// Warps of a leaf CTA (one CTA per SM): as many as the slices fit in 220 KB
// of shared memory, up to wmax.
int leaf_warps(size_t slice, int wmax) {
  int64_t nw = (int64_t)(220 * 1024 / slice);
  if (nw > wmax) nw = wmax;
  return nw < 1 ? 1 : (int)nw;
}

// Launches a leaf ordering of `nodes` nodes with slices of `slice` bytes on
// at most `sms` CTAs: the wide build when `allow_wide`, the nodes fill more
// than four waves of the 10-warp build and the slices leave room for more
// warps.
void launch_leaf(fp_handle* h, cudaStream_t s, const MdArgs& a0, size_t slice, int64_t nodes, int64_t sms,
                 bool allow_wide) {
  MdArgs a = a0;
  int nw = leaf_warps(slice, LEAF_WARPS);
  const bool wide = allow_wide && nodes > 4 * sms * nw && leaf_warps(slice, LEAF_WARPS_WIDE) > LEAF_WARPS;
  if (wide) nw = leaf_warps(slice, LEAF_WARPS_WIDE);
  size_t sm = slice * nw;
  if (sm < 116 * 1024) sm = 116 * 1024;       // one CTA per SM
  a.slice_bytes = (int64_t)slice;
  int64_t grid = (nodes + nw - 1) / nw;
  if (grid > sms) grid = sms;
  auto k = wide ? k_md_leaf<LEAF_WARPS_WIDE> : k_md_leaf<LEAF_WARPS>;
  allow_max_dynamic_smem(k);
  launch_pdl(s, k, (unsigned)grid, 32 * nw, sm, a);
  h->launches++;
}

size_t leaf_slice(int m);

// The leaf orderings run in two launches when the leaves span both size
// classes and are many more than one launch's warps (several waves): those
// above LEAF_SPLIT vertices with slices for the largest, then the others with
// slices for at most LEAF_SPLIT, so that more warps fit on an SM. With few
// leaves one wave holds them all and a second launch would only add its own
// largest leaf to the time. sz: the sizes, largest first; returns the number
// of leaves in the first launch (all of them for one launch).
int64_t leaf_class_cut(const int32_t* sz, int64_t nleaf, int32_t mmax, int64_t sms) {
  constexpr int LEAF_SPLIT = 256;
  const int64_t warps1 = sms * std::max(1, std::min<int>(LEAF_WARPS, (int)(220 * 1024 / leaf_slice(mmax))));
  int64_t cut = 0;
  while (cut < nleaf && sz[cut] > LEAF_SPLIT) ++cut;
  if (cut == 0 || cut == nleaf || nleaf <= 2 * warps1) cut = nleaf;
  return cut;
}

size_t leaf_slice(int m) {
  const size_t W = (m + 31) >> 5, S = m | 1, m2 = (size_t)((m + 1) & ~1), m64 = (size_t)((m + 63) & ~63);
  const size_t need = W * S * 4 + m64 * 2 + 2 * m2 * 2 + (MD_LEAF / 32) * 6;
  const size_t sortb = (size_t)pow2_host(m) * 8;
  return ((need > sortb ? need : sortb) + 15) & ~(size_t)15;
}

__host__ __device__ size_t sparse_smem(int m) {
  const size_t m2 = (size_t)((m + 1) & ~1), m64 = (size_t)((m + 63) & ~63);
  const size_t need = (size_t)m * SP_CAP * 2 + m64 * 2 + m2 * 2 + (m64 / 64) * 4;
  size_t p2 = 32;
  while (p2 < (size_t)m) p2 <<= 1;
  const size_t sortb = p2 * 4;
  return need > sortb ? need : sortb;
}

}  // namespace

fp_status early_md_begin(fp_handle* h, int32_t levels) {
  h->early_nodes = 0;
  if (levels <= 0 || h->n == 0) return FP_OK;
  const int32_t NE = (1 << levels) - 1, n = h->n;
  Arena ar;
  auto layout = [&]() {
    h->early_rank = ar.get<int32_t>(n);
    h->early_list = ar.get<int32_t>(n);
    h->early_loc = ar.get<int32_t>(n);
    h->early_start = ar.get<int32_t>(NE + 1);
    h->early_cnt = ar.get<int32_t>(NE);
    h->early_fill = ar.get<int32_t>(NE);
    h->early_ovf = ar.get<int32_t>(NE);
    h->early_base = ar.get<int32_t>(1);
  };
  layout();
  if (!ar.alloc(h)) return fail(h, FP_ERR_OUT_OF_MEMORY, "early ordering workspace");
  layout();      // early_rank is the block's base: early_md_release frees it
  fill_i32(h, h->early_cnt, 0, NE);
  fill_i32(h, h->early_ovf, 0, NE);
  fill_i32(h, h->early_base, 0, 1);
  h->early_nodes = NE;
  return FP_OK;
}

fp_status launch_early_md(fp_handle* h, int32_t d) {
  const int32_t t0 = (1 << d) - 1, T = 1 << d, n = h->n;
  if (t0 + T > h->early_nodes) return FP_OK;
  AuxStream* ax = aux_stream(h->device);
  if (!ax) return fail(h, FP_ERR_CUDA, "auxiliary stream");
  cudaStream_t s2 = ax->s;
  cudaEventRecord(ax->fork, h->stream);
  cudaStreamWaitEvent(s2, ax->fork, 0);
  const int G = grid_for(n, 256);
  ProfScope ps(FP_PROF_MD_MID, s2);
  launch_pdl(s2, k_early_count, G, 256, 0, h->node_of, n, t0, T, h->early_cnt);
  launch_pdl(s2, k_early_starts, 1, 32, 0, h->early_cnt, t0, T, h->early_base, h->early_start, h->early_fill);
  launch_pdl(s2, k_early_scatter, G, 256, 0, h->node_of, n, t0, T, h->early_start, h->early_fill, h->early_list);
  MdArgs a{h->rowptr, h->col, h->node_of, h->node_begin, h->node_size, h->early_start, h->early_list, h->early_loc,
           nullptr, nullptr, T, nullptr, nullptr, nullptr, nullptr, 0, h->early_ovf, nullptr, nullptr,
           t0, h->early_cnt, h->early_rank, (int64_t)SMEM_MAX};
  allow_max_dynamic_smem(k_md_sparse<false>);
  launch_pdl(s2, k_md_sparse<false>, T, MD_THREADS, SMEM_MAX, a);
  h->launches += 4;
  return check_cuda(h, cudaGetLastError(), "early ordering launch");
}

void early_md_release(fp_handle* h) {
  dev_free(h, h->early_rank);       // the base of the one block holding all eight arrays
  for (int32_t** p : {&h->early_rank, &h->early_list, &h->early_loc, &h->early_start, &h->early_cnt, &h->early_fill,
                      &h->early_ovf, &h->early_base})
    *p = nullptr;
  h->early_nodes = 0;
}

fp_status run_local_order(fp_handle* h) {
  const int32_t n = h->n;
  const int64_t nn = h->nnodes;
  const int G = grid_for(n, 256);
  auto I = [&](int64_t c) { return (int32_t*)dev_alloc(h, sizeof(int32_t) * (c > 0 ? c : 1)); };
  int32_t *sub = I(nn), *nvstart = I(nn + 1), *nvfill = I(nn), *nvlist = I(n), *loc = I(n), *tmp = I(scan_tmp_ints(nn) + 8);
  if (!sub || !nvstart || !nvfill || !nvlist || !loc || !tmp) return fail(h, FP_ERR_OUT_OF_MEMORY, "ordering workspace");
  // the node sizes (and the status word) go to the host as soon as they are
  // known; the host waits for them while the layout kernels still run
  int32_t* hsp = pinned_ints(nn);
  cudaEvent_t ev = mark_event(h->device);
  if (!hsp || !ev) return fail(h, FP_ERR_OUT_OF_MEMORY, "node size transfer");
  {
    ProfScope ps(FP_PROF_LAYOUT, h->stream);
    fill_i32(h, h->node_size, 0, nn);
    if (n > 0) FP_LAUNCH(h, k_node_sizes, G, 256, 0, h->node_of, n, h->node_size);
    cudaMemcpyAsync(hsp, h->node_size, sizeof(int32_t) * nn, cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    cudaEventRecord(ev, h->stream);
    FP_LAUNCH(h, k_tree_layout, 1, 1024, 0, h->D, nn, h->node_size, sub, h->node_begin, h->opt.schedule);
    scan_exclusive(h, h->node_size, nvstart, nn, tmp);
    fill_i32(h, nvfill, 0, nn);
    if (n > 0) FP_LAUNCH(h, k_scatter_nodes, G, 256, 0, h->node_of, n, nvstart, nvfill, nvlist);
  }
  FP_CHECK_LAUNCH(h, "tree layout");
  // plan the ordering launches from the node sizes
  cudaError_t e = cudaEventSynchronize(ev);
  if (e != cudaSuccess) return check_cuda(h, e, "node sizes");
  const int32_t st = *h->h_status;
  h->node_size_host.assign(hsp, hsp + nn);
  const std::vector<int32_t>& hs = h->node_size_host;
  if (st & ST_QUOTIENT_TOO_BIG) return fail(h, FP_ERR_UNSUPPORTED, "a patch has more than 4096 cross edges");
  if (st & ST_NODE_TOO_BIG) return fail(h, FP_ERR_UNSUPPORTED, "a dissection node above the warp bisection's 32 patches");
  // kinds: 0 leaf, 1 sparse, 2 global. Sparse nodes also get global rows, used
  // only if their adjacency lists overflow.
  std::vector<int32_t> ls[3], early;
  int mmax[3] = {0, 0, 0};
  for (int64_t t = 0; t < nn; ++t) {
    const int m = hs[t];
    if (m == 0) continue;
    if (m > MD_MAX) return fail(h, FP_ERR_UNSUPPORTED, "a tree node has more than 32768 vertices");
    if (t < h->early_nodes && sparse_smem(m) <= SMEM_MAX) {
      early.push_back((int32_t)t);     // ordered during the dissection
      continue;
    }
    const int kind = m <= MD_LEAF ? 0 : (sparse_smem(m) <= SMEM_MAX ? 1 : 2);
    ls[kind].push_back((int32_t)t);
    if (m > mmax[kind]) mmax[kind] = m;
  }
  // the leaf kernel's warps draw nodes largest first (ties by node index): a
  // counting sort over the sizes 1..MD_LEAF
  {
    std::vector<int32_t> cnt(MD_LEAF + 2, 0), sorted(ls[0].size());
    for (int32_t t : ls[0]) ++cnt[MD_LEAF - hs[t] + 1];
    for (int i = 1; i <= MD_LEAF + 1; ++i) cnt[i] += cnt[i - 1];
    for (int32_t t : ls[0]) sorted[cnt[MD_LEAF - hs[t]]++] = t;
    ls[0].swap(sorted);
  }
  // global rows and sort scratch for the sparse (fallback) and global nodes
  std::vector<int64_t> goff, soff;
  int64_t gwords = 0, gsort = 0;
  for (const std::vector<int32_t>* L : {&ls[1], &ls[2], &early})
    for (int32_t t : *L) {
      const int m = hs[t];
      goff.push_back(gwords);
      // dense bit rows, or the sparse lists (12 words a vertex), 16 B aligned
      gwords += (std::max<int64_t>((int64_t)m * ((m + 31) / 32), 12 * (int64_t)m) + 3) & ~(int64_t)3;
      soff.push_back(gsort);
      gsort += pow2_host(m);
    }
  const int64_t nlist = (int64_t)ls[0].size() + ls[1].size() + ls[2].size() + early.size();
  const int64_t nsg = (int64_t)goff.size();
  std::vector<int64_t> up((nlist + 1) / 2 + 2 * nsg + 1);
  int32_t* up32 = (int32_t*)up.data();
  int64_t o = 0;
  for (const std::vector<int32_t>* L : {&ls[0], &ls[1], &ls[2], &early})
    for (int32_t t : *L) up32[o++] = t;
  const int64_t off64 = (nlist + 1) / 2;
  for (int64_t i = 0; i < nsg; ++i) { up[off64 + i] = goff[i]; up[off64 + nsg + i] = soff[i]; }
  int64_t* dup;
  uint32_t* grows;
  int32_t *gs, *ovf;
  Arena ar;
  auto layout = [&]() {
    dup = ar.get<int64_t>((int64_t)up.size() + 1);
    grows = ar.get<uint32_t>(gwords);
    gs = ar.get<int32_t>(gsort);
    // flags of the sparse-list passes (ls[1], then ls[2] after the leaf
    // kernel's node queue)
    ovf = ar.get<int32_t>((int64_t)ls[1].size() + 2 + (int64_t)ls[2].size());
  };
  layout();
  if (!ar.alloc(h)) return fail(h, FP_ERR_OUT_OF_MEMORY, "ordering rows");
  layout();      // dup is the block's base
  e = cudaMemcpyAsync(dup, up.data(), sizeof(int64_t) * up.size(), cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "upload node lists");
  fill_i32(h, ovf, 0, (int64_t)ls[1].size() + 2 + (int64_t)ls[2].size());
  const int32_t* dnodes = (const int32_t*)dup;
  MdArgs base{h->rowptr, h->col, h->node_of, h->node_begin, h->node_size, nvstart, nvlist, loc, h->perm,
              nullptr, 0, grows, dup + off64, gs, dup + off64 + nsg, 0, nullptr, nullptr, ovf + ls[1].size()};
  // the separators ordered during the dissection are completed on the first
  // auxiliary stream, followed there by those too large for shared memory
  // (the longest orderings), the other separators run on the second one (so
  // that they need not wait for either), the leaves on the handle's stream
  // in CTAs that fill whole SMs, leaving `reserved` SMs for separator CTAs
  AuxStream* ax = aux_stream(h->device, 0);
  AuxStream* ax3 = aux_stream(h->device, 1);
  if (!ax || !ax3) return fail(h, FP_ERR_CUDA, "auxiliary stream");
  cudaStream_t s2 = ax->s, s3 = ax3->s;
  cudaEventRecord(ax->fork, h->stream);
  cudaStreamWaitEvent(s2, ax->fork, 0);
  cudaEventRecord(ax3->fork, h->stream);
  cudaStreamWaitEvent(s3, ax3->fork, 0);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  const int nbig = (int)(ls[1].size() + ls[2].size() + early.size());
  const int reserved = nbig < 24 ? nbig : 24;
  const int64_t lo1 = (int64_t)ls[0].size(), lo2 = lo1 + (int64_t)ls[1].size(), lo3 = lo2 + (int64_t)ls[2].size();
  // the leaves first: their launch is on the critical path, the separators'
  // on the auxiliary streams have time to spare
  if (!ls[0].empty()) {
    const int64_t nleaf = (int64_t)ls[0].size();
    const int64_t cap_sms = sms - reserved > 1 ? sms - reserved : 1;
    std::vector<int32_t> lsz(nleaf);
    for (int64_t i = 0; i < nleaf; ++i) lsz[i] = hs[ls[0][i]];
    const int64_t cut = leaf_class_cut(lsz.data(), nleaf, mmax[0], cap_sms);
    ProfScope ps(FP_PROF_MD_SMALL, h->stream);
    for (int part = 0; part < 2; ++part) {
      const int64_t lo = part == 0 ? 0 : cut, hi = part == 0 ? cut : (int64_t)ls[0].size();
      if (hi <= lo) continue;
      MdArgs a = base;
      a.nodes = dnodes + lo;
      a.nnodes_launch = (int32_t)(hi - lo);
      a.queue = base.queue + part;
      launch_leaf(h, h->stream, a, leaf_slice(hs[ls[0][lo]]), hi - lo, cap_sms, true);
    }
  }
  if (!early.empty()) {
    // separators ordered during the dissection: redo the ones whose adjacency
    // lists overflowed with global rows, then place every other one's ranks
    MdArgs a = base;
    a.nodes = dnodes + lo3;
    a.nnodes_launch = (int32_t)early.size();
    a.nvstart = h->early_start;
    a.nvlist = h->early_list;
    a.overflow = h->early_ovf;
    a.node_base = -1;                     // overflow flags indexed by node
    a.grow_off = dup + off64 + (int64_t)ls[1].size() + (int64_t)ls[2].size();
    a.gsort_off = dup + off64 + nsg + (int64_t)ls[1].size() + (int64_t)ls[2].size();
    const size_t smg = (size_t)2 * MD_MAX * sizeof(uint16_t);
    allow_max_dynamic_smem(k_md_global);
    ProfScope ps(FP_PROF_MD_LARGE, s2);
    launch_pdl(s2, k_md_global, (unsigned)early.size(), MD_THREADS, smg, a);
    launch_pdl(s2, k_early_place, G, 256, 0, h->node_of, n, h->early_nodes, h->node_size, h->node_begin, h->early_rank,
                                     h->early_ovf, h->perm, (int64_t)SMEM_MAX);
    h->launches += 2;
  }
  if (!ls[1].empty()) {
    MdArgs a = base;
    a.nodes = dnodes + lo1;
    a.nnodes_launch = (int32_t)ls[1].size();
    a.overflow = ovf;
    const size_t sm = sparse_smem(mmax[1]);
    allow_max_dynamic_smem(k_md_sparse<false>);
    {
      ProfScope ps(FP_PROF_MD_MID, s3);
      launch_pdl(s3, k_md_sparse<false>, (unsigned)ls[1].size(), MD_THREADS, sm, a);
      h->launches++;
    }
    // redo flagged nodes with global rows (grow_off/gsort_off index from 0 here)
    const size_t smg = (size_t)2 * MD_MAX * sizeof(uint16_t);
    allow_max_dynamic_smem(k_md_global);
    ProfScope ps(FP_PROF_MD_LARGE, s3);
    launch_pdl(s3, k_md_global, (unsigned)ls[1].size(), MD_THREADS, smg, a);
    h->launches++;
  }
  if (!ls[2].empty()) {
    MdArgs a = base;
    a.nodes = dnodes + lo2;
    a.nnodes_launch = (int32_t)ls[2].size();
    a.grow_off = dup + off64 + (int64_t)ls[1].size();
    a.gsort_off = dup + off64 + nsg + (int64_t)ls[1].size();
    a.overflow = ovf + ls[1].size() + 2;
    // first with sparse lists in global memory, then the dense kernel for the
    // nodes whose lists overflowed
    const size_t M64 = (size_t)((mmax[2] + 63) & ~63);
    const size_t smsp = M64 * 2 + (size_t)((mmax[2] + 1) & ~1) * 2 + (M64 / 64) * 4;
    allow_max_dynamic_smem(k_md_sparse<true>);
    ProfScope ps(FP_PROF_MD_LARGE, s2);
    launch_pdl(s2, k_md_sparse<true>, (unsigned)ls[2].size(), MD_THREADS, smsp, a);
    const size_t smg = (size_t)2 * MD_MAX * sizeof(uint16_t);
    allow_max_dynamic_smem(k_md_global);
    launch_pdl(s2, k_md_global, (unsigned)ls[2].size(), MD_THREADS, smg, a);
    h->launches += 2;
  }
  h->join_frees = {(void*)sub, (void*)nvstart, (void*)nvfill, (void*)nvlist, (void*)loc, (void*)tmp, (void*)dup};
  h->join_pending = true;
  if (h->qnet && n > 0) {
    // the learned pass needs only the leaves' orders (on this stream) and
    // some position inside each other node: it runs before the join
    FP_CHECK_LAUNCH(h, "minimum degree");
    h->pend_nvlist = nvlist;
    h->pend_nvstart = nvstart;
    return FP_OK;
  }
  FP_TRY(finish_orderings(h));
  if (n > 0) {
    ProfScope ps(FP_PROF_PERM, h->stream);
    FP_LAUNCH(h, k_iperm, G, 256, 0, h->perm, n, h->iperm);
  }
  FP_CHECK_LAUNCH(h, "iperm");
  return FP_OK;
}

fp_status finish_orderings(fp_handle* h) {
  if (!h->join_pending) return FP_OK;
  h->join_pending = false;
  AuxStream* ax = aux_stream(h->device, 0);
  AuxStream* ax3 = aux_stream(h->device, 1);
  if (!ax || !ax3) return fail(h, FP_ERR_CUDA, "auxiliary stream");
  {
    // the pair brackets only the wait: it starts when the handle's stream has
    // finished its own work and ends when both auxiliary streams have
    ProfScope ps(FP_PROF_JOIN_WAIT, h->stream);
    cudaEventRecord(ax->join, ax->s);
    cudaStreamWaitEvent(h->stream, ax->join, 0);
    cudaEventRecord(ax3->join, ax3->s);
    cudaStreamWaitEvent(h->stream, ax3->join, 0);
  }
  for (void* p : h->join_frees) dev_free(h, p);
  h->join_frees.clear();
  h->pend_nvlist = h->pend_nvstart = nullptr;
  FP_CHECK_LAUNCH(h, "minimum degree");
  early_md_release(h);
  return FP_OK;
}

fp_status run_leaf_md_keyed(fp_handle* h, const int32_t* d_nodes, int32_t count, int32_t mmax, int32_t* vlist,
                            int32_t* loc, const uint32_t* key, int32_t* perm_out, const std::vector<int32_t>* lsz) {
  if (count == 0) return FP_OK;
  if (mmax > MD_LEAF) return fail(h, FP_ERR_UNSUPPORTED, "keyed ordering of a node above 512 vertices");
  if (lsz && (int64_t)lsz->size() != count) return fail(h, FP_ERR_INVALID_ARG, "leaf sizes do not match the list");
  int32_t* queue = (int32_t*)dev_alloc(h, 2 * sizeof(int32_t));
  if (!queue) return fail(h, FP_ERR_OUT_OF_MEMORY, "node queue");
  fill_i32(h, queue, 0, 2);
  MdArgs base{h->rowptr, h->col, h->node_of, h->node_begin, h->node_size, h->node_begin, vlist, loc, perm_out,
              d_nodes, count, nullptr, nullptr, nullptr, nullptr, 0, nullptr, key, queue};
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  // the list is largest first: with the sizes, the same two size classes as
  // the plain leaf orderings
  const int64_t cut = lsz ? leaf_class_cut(lsz->data(), count, mmax, sms) : count;
  ProfScope ps(FP_PROF_LEARNED, h->stream);
  for (int part = 0; part < 2; ++part) {
    const int64_t lo = part == 0 ? 0 : cut, hi = part == 0 ? cut : count;
    if (hi <= lo) continue;
    MdArgs a = base;
    a.nodes = d_nodes + lo;
    a.nnodes_launch = (int32_t)(hi - lo);
    a.queue = queue + part;
    launch_leaf(h, h->stream, a, leaf_slice(part == 0 ? mmax : (*lsz)[lo]), hi - lo, sms, part == 1);
  }
  FP_CHECK_LAUNCH(h, "keyed minimum degree");
  dev_free(h, queue);
  return FP_OK;
}

void launch_dof_expand_perm(fp_handle* h, const int32_t* perm, int32_t* perm_d, int32_t* iperm_d) {
  const int64_t N = (int64_t)h->n * h->b;
  if (N == 0) return;
  ProfScope ps(FP_PROF_PERM, h->stream);
  FP_LAUNCH(h, k_dof_perm, grid_for(N, 256), 256, 0, perm, h->n, h->b, perm_d, iperm_d);
}

void launch_dof_expand_symbolic(fp_handle* h, const int32_t* parent, const int32_t* colcount, int32_t* parent_d,
                                int32_t* colcount_d, int32_t v0, int32_t v1, cudaStream_t s) {
  if (v1 < 0) v1 = h->n;
  const int64_t N = (int64_t)(v1 - v0) * h->b;
  if (N <= 0) return;
  if (!s) s = h->stream;
  ProfScope ps(FP_PROF_PERM, s);
  launch_pdl(s, k_dof_symbolic, grid_for(N, 256), 256, 0, parent, colcount, v0, v1, h->b, parent_d, colcount_d);
  h->launches++;
}

}  // namespace fp
