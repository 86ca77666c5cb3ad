// a7 symbolic Cholesky of B = P (G + I) P^T for a nested-dissection ordering:
// elimination-tree parent[j] = min{ i > j : L_ij != 0 } and colcount[j] =
// |{ i >= j : L_ij != 0 }| (textbook definitions; the paper hands the etree
// to cuDSS, Sections 4.2 and 6), nnz(L) = sum colcount, flops = sum colcount^2
// (Section 6.5).
//
// The nested-dissection tree makes the computation local. The structure of a
// column j of tree node t lives in U_t = V_t u A_t, where A_t are the ancestor
// vertices reachable from j through already-eliminated vertices: the ancestors
// adjacent to V_t, plus the entries of every "element" exported by a
// descendant -- the structure of a column whose etree parent lies above its own
// node (merged into that parent, as in the column-merge rule
//   struct(j) = adj(j)_{>j}  u  U_{c : parent(c) = j} struct(c) \ {j}).
// A node runs once all its descendants have (their elements are complete):
// every leaf (no non-empty descendant) in one launch, largest first, then the
// inner nodes depth by depth, deepest first. Per node:
//   1. stream the node's slab of B's pattern (rows in position order, built
//      once per call by k_perm_pairs): mark A_t in a bitmap over the
//      concatenated ancestor ranges and keep the (column, position) pairs
//      above the diagonal in shared memory; compact the bitmap (prefix
//      popcounts), so U_t gets dense local indices in position order;
//   2. seed one bit row per column from those pairs and the elements whose
//      smallest entry is in V_t;
//   3. one warp sweeps the columns in order: parent = first set bit, count =
//      popc; the row is merged into its parent's row, kept in registers when the
//      parent is the next column (the chains of separator blocks), or exported
//      as an element to the node holding its parent;
//   4. dense tail: once struct(i) holds every later column of the node, the
//      rest of the node is a chain (parent(j) = j+1) and struct(j) is
//      {j+1..m-1} plus the ancestor columns met in the rows i..j, counted per
//      row by a chunked prefix OR down the rows (rows in shared memory) or by
//      the first row of each ancestor column (an atomicMin per bit), then a
//      prefix sum. The top separators of a mesh reach this point within a
//      few columns.
// Launches of many small nodes run one node per small CTA (64 or 128
// threads, 30 KB of shared memory, the first warp sweeping); a node that does
// not fit is deferred to the block kernel, which also takes launches of at
// most 148 nodes (one 512-thread CTA per node, rows in shared memory when they
// fit, else in a global scratch pool).
// Positions of a node are contiguous in both schedules and ancestors always
// come later, so bit order equals position order.
#include <algorithm>
#include <vector>

#include "fp_device.cuh"

namespace fp {
namespace {

constexpr int SYM_MAX_ANC = 32;
constexpr int SW_SMEM_WORDS = 7680;        // small-node CTAs: 30 KB each
constexpr int SB_THREADS = 512;
constexpr int SB_SMEM_WORDS = 54 * 1024;   // block CTAs: 216 KB each
constexpr int DENSE_MIN = 16;              // shortest chain worth the parallel tail
constexpr int32_t NO_ROW = INT_MAX;

// Column i's bit row only holds words >= i/32 (its bits are all above i), so
// the rows are stored as a staircase: row i starts at tri_off(i, W).
__device__ __forceinline__ int64_t tri_off(int32_t i, int32_t W) {
  const int64_t q = i >> 5, r = i & 31;
  return (int64_t)i * W - (32 * q * (q - 1) / 2 + r * q);
}

struct SymArgs {
  const int32_t* prow;             // [n + 1] slab of row p: prow[p] .. prow[p+1]
  const int2* ppair;               // (p, q): position p adjacent to position q in B
  const int32_t* perm;
  const int32_t* node_of;
  const int32_t* node_begin;
  const int32_t* node_size;
  int32_t t0, T;
  int32_t* parent;
  int32_t* colcount;
  unsigned long long* sums;        // [0] nnz(L), [1] flops
  int32_t* elem_head;              // [nnodes]
  int32_t* elem_hdr;               // [3 * cap_hdr]: next, offset, length
  int32_t* elem_data;              // element entries (positions, ascending)
  int64_t cap_hdr, cap_data;
  unsigned long long* elem_ctr;    // [0] headers used, [1] entries used
  uint32_t* pool;                  // global scratch words for rows that do not fit
  int64_t pool_words;
  unsigned long long* pool_ctr;
  int32_t* big_list;               // nodes of this level deferred to the block kernel
  int32_t* big_count;
  int32_t* status;
  const int32_t* in_list;          // explicit node list (else the level t0 .. t0+T-1)
  int32_t in_count;
  int64_t* node_fill;              // fill mode: per node, the sum of its columns' counts; no exports
};

__device__ __forceinline__ int64_t r4(int64_t x) { return (x + 3) & ~3ll; }

// Local coordinate of an ancestor position in the concatenated ancestor
// ranges. Ancestor begins grow with the distance in both schedules, so the
// range is the last one that starts at or before pos.
__device__ __forceinline__ int32_t anc_coord(const int32_t* ab, const int32_t* ao, int32_t na, int32_t pos) {
  int32_t i = 0;
#pragma unroll
  for (int st = 16; st; st >>= 1)
    if (i + st < na && ab[i + st] <= pos) i += st;
  return ao[i] + pos - ab[i];
}

// Exports struct(i) (cnt entries; bit words given by word_of(w)) as an element
// to the node holding position pf. Called by one whole warp.
template <class WordOf>
__device__ __forceinline__ void export_element(const SymArgs& a, const int32_t* upos, int32_t W, uint32_t cnt,
                                               int32_t pf, WordOf word_of) {
  const int lane = threadIdx.x & 31;
  unsigned long long off = 0, hdr = 0;
  if (lane == 0) {
    off = atomicAdd(&a.elem_ctr[1], (unsigned long long)cnt);
    hdr = atomicAdd(&a.elem_ctr[0], 1ull);
  }
  off = __shfl_sync(0xffffffffu, off, 0);
  hdr = __shfl_sync(0xffffffffu, hdr, 0);
  if ((int64_t)(off + cnt) > a.cap_data || (int64_t)hdr >= a.cap_hdr) {
    if (lane == 0) atomicOr(a.status, ST_POOL_OVERFLOW);
    return;
  }
  int32_t base = 0;
  for (int w0 = 0; w0 < W; w0 += 32) {
    const int w = w0 + lane;
    uint32_t s = w < W ? word_of(w) : 0u;
    const int c = __popc(s);
    int32_t ex = warp_incl_scan_i32(c) - c;
    const int32_t tot = __shfl_sync(0xffffffffu, ex + c, 31);
    while (s) {
      const int bt = __ffs(s) - 1;
      s &= s - 1;
      a.elem_data[off + base + ex++] = upos[w * 32 + bt];
    }
    base += tot;
  }
  if (lane == 0) {
    const int32_t target = a.node_of[a.perm[pf]];
    a.elem_hdr[3 * hdr + 1] = (int32_t)off;
    a.elem_hdr[3 * hdr + 2] = (int32_t)cnt;
    __threadfence();
    a.elem_hdr[3 * hdr] = atomicExch(&a.elem_head[target], (int32_t)hdr);
  }
}

// export_element with the whole CTA, for the dense tail's last column (a
// structure of up to thousands of ancestor columns): a word of the structure
// a thread, offsets by a block scan of the words' popcounts, each thread's
// entries written eight at a time with their position loads issued first.
// Called by every thread of the CTA.
template <class WordOf>
__device__ void export_element_block(const SymArgs& a, const int32_t* upos, int32_t W, uint32_t cnt, int32_t pf,
                                     WordOf word_of, int32_t* red) {
  __shared__ unsigned long long s_eo[2];
  __shared__ int32_t s_bad;
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid == 0) {
    s_eo[0] = atomicAdd(&a.elem_ctr[1], (unsigned long long)cnt);
    s_eo[1] = atomicAdd(&a.elem_ctr[0], 1ull);
    s_bad = (int64_t)(s_eo[0] + cnt) > a.cap_data || (int64_t)s_eo[1] >= a.cap_hdr;
    if (s_bad) atomicOr(a.status, ST_POOL_OVERFLOW);
  }
  __syncthreads();
  if (s_bad) return;
  const unsigned long long off = s_eo[0], hdr = s_eo[1];
  int32_t carry = 0;
  for (int32_t w0 = 0; w0 < W; w0 += nthr) {
    const int32_t w = w0 + tid;
    uint32_t bits = w < W ? word_of(w) : 0u;
    int32_t tot;
    int32_t o = block_excl_scan_i32(__popc(bits), &tot, red) + carry;
    while (bits) {
      int32_t q[8];
      int n = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        q[k] = -1;
        if (bits) {
          q[k] = w * 32 + __ffs(bits) - 1;
          bits &= bits - 1;
          ++n;
        }
      }
      int32_t v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = q[k] >= 0 ? upos[q[k]] : 0;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < n) a.elem_data[off + o + k] = v[k];
      o += n;
    }
    carry += tot;
  }
  __syncthreads();
  if (tid == 0) {
    const int32_t target = a.node_of[a.perm[pf]];
    a.elem_hdr[3 * hdr + 1] = (int32_t)off;
    a.elem_hdr[3 * hdr + 2] = (int32_t)cnt;
    __threadfence();
    a.elem_hdr[3 * hdr] = atomicExch(&a.elem_head[target], (int32_t)hdr);
  }
}

constexpr int SLAB_ILP = 4;

// Step 1's gather, done once: the upper adjacency entries (column i, position
// pos > b + i) of the node's columns and the entries of its incoming elements
// (column r0 = the element's smallest entry, with each later entry) become
// (column, position) pairs of a list that grows down from `top` (pair s at
// top[-1 - s]); ancestor positions are marked in the bitmap. The loops run in
// step across each warp, so a round takes its list slots with one shared
// atomic per warp. *cnt ends as the number of pairs, which may exceed cap:
// then the pairs from cap on were not stored.
__device__ void gather_entries(const SymArgs& a, int32_t t, int32_t b, int32_t m, const int32_t* ab,
                               const int32_t* ao, int32_t na, uint32_t* bitmap, int2* top, int32_t cap,
                               int32_t* cnt) {
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
  const int32_t end = b + m;
  auto keep = [&](int32_t i, int32_t pos, int32_t slot) {
    if (pos >= end) {
      const int32_t c = anc_coord(ab, ao, na, pos);
      atomicOr(&bitmap[c >> 5], 1u << (c & 31));
    }
    if (slot < cap) top[-1 - slot] = make_int2(i, pos);
  };
  // the node's columns own one contiguous slab of B's pattern: stream it,
  // SLAB_ILP pairs a lane per round, all loads issued first
  const int32_t e0 = a.prow[b], e1 = a.prow[b + m];
  for (int32_t eb = e0 + SLAB_ILP * (tid - lane); eb < e1; eb += SLAB_ILP * nthr) {
    int2 pq[SLAB_ILP];
#pragma unroll
    for (int u = 0; u < SLAB_ILP; ++u) {
      const int32_t e = eb + 32 * u + lane;
      pq[u] = e < e1 ? a.ppair[e] : make_int2(0, -1);
    }
#pragma unroll
    for (int u = 0; u < SLAB_ILP; ++u) {
      const bool up = pq[u].y > pq[u].x;           // above the column (never the padding)
      const unsigned bal = __ballot_sync(0xffffffffu, up);
      int32_t base = 0;
      if (lane == 0 && bal) base = atomicAdd(cnt, __popc(bal));
      base = __shfl_sync(0xffffffffu, base, 0) + __popc(bal & lanemask_lt());
      if (up) keep(pq[u].x - b, pq[u].y, base);
    }
  }
  for (int32_t el = a.elem_head[t]; el >= 0; el = a.elem_hdr[3 * el]) {
    const int32_t off = a.elem_hdr[3 * el + 1], len = a.elem_hdr[3 * el + 2];
    const int32_t r0 = a.elem_data[off] - b;      // smallest entry: a column of this node
    for (int32_t j0 = 1 + tid - lane; j0 < len; j0 += nthr) {
      const int32_t j = j0 + lane;
      const int32_t pos = j < len ? a.elem_data[off + j] : -1;
      const unsigned bal = __ballot_sync(0xffffffffu, pos >= 0);
      int32_t base = 0;
      if (lane == 0) base = atomicAdd(cnt, __popc(bal));
      base = __shfl_sync(0xffffffffu, base, 0) + __popc(bal & lanemask_lt());
      if (pos >= 0) keep(r0, pos, base);
    }
  }
}

// Popcount of the bits of word w that fall in columns [lo, hi).
__device__ __forceinline__ uint32_t popc_range(uint32_t s, int w, int32_t lo, int32_t hi) {
  const int32_t l = max(lo - 32 * w, 0), h = min(hi - 32 * w, 32);
  if (l >= h) return 0u;
  const uint32_t mk = (h == 32 ? 0xffffffffu : ((1u << h) - 1u)) & ~((1u << l) - 1u);
  return __popc(s & mk);
}

// Column sweep of one node by one warp (step 3). Column i's parent is the first
// set bit of its row (struct(i)), its count the popcount; the row minus the
// parent bit is merged into the parent's row. Returns the column where the
// dense tail starts (its structure written back to its row), or m.
//
// Rows of at most 32*NCH words (NCH > 0): lane l holds words l, l+32, ...
// of the current row in registers. While the parent is the next column the
// merged structure stays in registers (carry); any other merge is an atomic OR
// into the parent's row. The next row is loaded one column ahead: a merge
// from column i never lands in row i+1 except through the carry, so the early
// load sees its final contents. The rare cases (an empty column, a parent
// above the node, the start of the dense tail) leave the common path in one
// branch.
template <int NCH>
__device__ int32_t sweep_columns(const SymArgs& a, uint32_t* rows, const int32_t* upos, int32_t m, int32_t W,
                                 int32_t b, bool tail_ok, unsigned long long& nnz, unsigned long long& fl) {
  const int lane = threadIdx.x & 31;
  uint32_t carry[NCH], nxt[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const int w = lane + 32 * c;
    carry[c] = 0u;
    nxt[c] = w < W ? rows[w] : 0u;
  }
  // column i's parent and count are held by lane i % 32 and stored 32 at a time
  int32_t my_par = -1, my_cc = 1;
  auto flush = [&](int32_t i_last) {
    const int32_t j = (i_last & ~31) + lane;
    if (j <= i_last) {
      a.parent[b + j] = my_par;
      a.colcount[b + j] = my_cc;
      nnz += (unsigned long long)my_cc;
      fl += (unsigned long long)my_cc * (unsigned long long)my_cc;
    }
  };
  int64_t off = 0;                                // tri_off(i, W)
  for (int32_t i = 0; i < m; ++i) {
    const int i0 = i >> 5;
    uint32_t* ri = rows + off - i0;               // word w of row i at ri[w], w >= i0
    off += W - i0;
    uint32_t cur[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) cur[c] = nxt[c] | carry[c];
    if (i + 1 < m) {
      const int i1 = (i + 1) >> 5;
      const uint32_t* rn = rows + off - i1;
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        const int w = lane + 32 * c;
        nxt[c] = (w < W && w >= i1) ? rn[w] : 0u;
      }
    }
    uint32_t f = 0xffffffffu, cnt = 0;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      const uint32_t s = cur[c];
      const uint32_t bt = s ? (uint32_t)((lane + 32 * c) * 32 + __ffs(s) - 1) : 0xffffffffu;
      f = bt < f ? bt : f;
      cnt += __popc(s);
    }
    f = __reduce_min_sync(0xffffffffu, f);
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    const bool inside = f < (uint32_t)m;          // false for an empty column too
    const bool chain = f == (uint32_t)i + 1;
    const int32_t rest = m - 1 - i;
    if (lane == (i & 31)) {
      my_par = inside ? b + (int32_t)f : -1;
      my_cc = (int32_t)cnt + 1;
    }
    if (!inside || (tail_ok && chain && rest >= DENSE_MIN && cnt >= (uint32_t)rest)) {
      if (!inside) {
        if (cnt != 0) {
          const int32_t pf = upos[f];
          if (lane == (i & 31)) my_par = pf;
          // fill mode: the structure goes nowhere
          if (!a.node_fill)
            export_element(a, upos, W, cnt, pf, [&](int w) -> uint32_t {
              uint32_t s = 0u;
#pragma unroll
              for (int c = 0; c < NCH; ++c) if (c == (w >> 5)) s = cur[c];
              return s;
            });
        }
        if ((i & 31) == 31) flush(i);
#pragma unroll
        for (int c = 0; c < NCH; ++c) carry[c] = 0u;
        continue;
      }
      // dense tail? struct(i) must hold every later column of the node (cnt
      // bounds that count from above, so most columns skip the exact test)
      uint32_t cn = 0;
#pragma unroll
      for (int c = 0; c < NCH; ++c) cn += popc_range(cur[c], lane + 32 * c, i + 1, m);
      cn = __reduce_add_sync(0xffffffffu, cn);
      if (cn == (uint32_t)rest) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          const int w = lane + 32 * c;
          if (w < W && w >= i0) ri[w] = cur[c];
        }
        flush(i);
        __syncwarp();
        return i;
      }
    }
    if ((i & 31) == 31) flush(i);
    // merge struct(i) \ {f} into column f
    const int f0 = (int)(f >> 5);
    const uint32_t fb = 1u << (f & 31);
#pragma unroll
    for (int c = 0; c < NCH; ++c)
      if (lane + 32 * c == f0) cur[c] &= ~fb;
    if (chain) {
#pragma unroll
      for (int c = 0; c < NCH; ++c) carry[c] = cur[c];
    } else {
#pragma unroll
      for (int c = 0; c < NCH; ++c) carry[c] = 0u;
      uint32_t* rf = rows + tri_off((int32_t)f, W) - f0;
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        const int w = lane + 32 * c;
        if (w < W && w >= f0 && cur[c]) atomicOr(&rf[w], cur[c]);
      }
    }
  }
  if (m & 31) flush(m - 1);
  return m;
}

// Rows of any width (NCH = 0): the same steps with every row in memory.
template <>
__device__ int32_t sweep_columns<0>(const SymArgs& a, uint32_t* rows, const int32_t* upos, int32_t m, int32_t W,
                                    int32_t b, bool tail_ok, unsigned long long& nnz, unsigned long long& fl) {
  const int lane = threadIdx.x & 31;
  int32_t my_par = -1, my_cc = 1;
  auto flush = [&](int32_t i_last) {
    const int32_t j = (i_last & ~31) + lane;
    if (j <= i_last) {
      a.parent[b + j] = my_par;
      a.colcount[b + j] = my_cc;
      nnz += (unsigned long long)my_cc;
      fl += (unsigned long long)my_cc * (unsigned long long)my_cc;
    }
  };
  int64_t off = 0;                                // tri_off(i, W)
  for (int32_t i = 0; i < m; ++i) {
    const int i0 = i >> 5;
    uint32_t* ri = rows + off - i0;               // word w of row i at ri[w], w >= i0
    off += W - i0;
    uint32_t f = 0xffffffffu, cnt = 0;
    for (int w = lane; w < W; w += 32) {
      const uint32_t s = w >= i0 ? ri[w] : 0u;
      if (s) { const uint32_t bt = w * 32 + __ffs(s) - 1; f = bt < f ? bt : f; cnt += __popc(s); }
    }
    f = __reduce_min_sync(0xffffffffu, f);
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    const bool inside = f < (uint32_t)m;
    const int32_t pf = cnt == 0 ? -1 : (inside ? b + (int32_t)f : upos[f]);
    if (lane == (i & 31)) {
      my_par = pf;
      my_cc = (int32_t)cnt + 1;
    }
    const bool flushed = (i & 31) == 31 || i + 1 == m;
    if (flushed) flush(i);
    if (cnt == 0) continue;
    if (!inside) {
      if (!a.node_fill)
        export_element(a, upos, W, cnt, pf, [&](int w) -> uint32_t { return w >= i0 ? ri[w] : 0u; });
      continue;
    }
    if (tail_ok && f == (uint32_t)i + 1 && m - 1 - i >= DENSE_MIN && cnt >= (uint32_t)(m - 1 - i)) {
      uint32_t cn = 0;
      for (int w = lane; w < W; w += 32) if (w >= i0) cn += popc_range(ri[w], w, i + 1, m);
      cn = __reduce_add_sync(0xffffffffu, cn);
      if (cn == (uint32_t)(m - 1 - i)) {
        if (!flushed) flush(i);
        __syncwarp();
        return i;
      }
    }
    // merge struct(i) \ {f} into column f
    const int f0 = (int)(f >> 5);
    uint32_t* rf = rows + tri_off((int32_t)f, W) - f0;
    for (int w = lane; w < W; w += 32) {
      if (w < f0) continue;           // struct(i) \ {f} lies above f
      uint32_t s = ri[w];
      if (w == f0) s &= ~(1u << (f & 31));
      if (s) rf[w] |= s;
    }
  }
  return m;
}

// Step 4 for columns is+1 .. m-1 (see the file comment). scratch holds
// U - m + (m - is) ints. All threads of the CTA call.
// The count of ancestor columns first met in each row comes from a prefix OR
// down the rows, word by word: the rows are cut into ch chunks, each (chunk,
// word) pair ORs its rows, an exclusive OR-scan over the chunks gives each
// pair the words met above it, and a second pass counts every row's new bits.
// When the rows are in shared memory and that scratch fits; else (rows in
// the global pool, or very few ancestor columns) each ancestor column takes
// the first row holding it by an atomicMin per bit.
__device__ void dense_tail(const SymArgs& a, const uint32_t* rows, const int32_t* upos, int32_t m, int32_t U,
                           int32_t W, int32_t b, int32_t is, int32_t* scratch, int32_t* red,
                           unsigned long long& nnz, unsigned long long& fl) {
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
  const int32_t nab = U - m, L = m - is;
  const int32_t wa = m >> 5, nwa = W - wa;
  const uint32_t amask0 = 0xffffffffu << (m & 31);
  // (rows in the global pool keep the atomicMin form: its single pass of
  // loads beats two passes there)
  int32_t ch = 0;
  if (nab > 0 && __isShared(rows)) {
    ch = nwa <= nthr ? nthr / nwa : 1;
    const int32_t chmax = (is + nab) / nwa - 1;
    if (ch > chmax) ch = chmax;
    if (ch > L) ch = L;
  }
  const bool por = ch >= 1;
  int32_t* hist;                     // [L]: ancestor columns first met in row is + l
  int32_t* first = nullptr;          // [nab]: first row holding each ancestor column (atomicMin form)
  uint32_t* part = nullptr;          // [ch * nwa]: OR of a chunk's rows, then of the rows above it
  uint32_t* tot = nullptr;           // [nwa]: OR of all rows
  if (por) {
    hist = scratch;
    part = reinterpret_cast<uint32_t*>(scratch + L);
    tot = part + (int64_t)ch * nwa;
  } else {
    first = scratch;
    hist = scratch + nab;
    for (int32_t u = tid; u < nab; u += nthr) first[u] = NO_ROW;
  }
  for (int32_t j = is + 1 + tid; j < m - 1; j += nthr) a.parent[b + j] = b + j + 1;
  for (int32_t l = tid; l < L; l += nthr) hist[l] = 0;
  __syncthreads();
  if (por) {
    const int32_t R = (L + ch - 1) / ch;
    auto word = [&](int32_t l, int32_t w) -> uint32_t {
      const uint32_t x = rows[tri_off(l, W) - (l >> 5) + wa + w];
      return w == 0 ? x & amask0 : x;
    };
    for (int32_t x = tid; x < ch * nwa; x += nthr) {
      const int32_t c = x / nwa, w = x - c * nwa;
      const int32_t l0 = is + c * R, l1 = min(l0 + R, m);
      uint32_t acc = 0u;
#pragma unroll 8
      for (int32_t l = l0; l < l1; ++l) acc |= word(l, w);
      part[x] = acc;
    }
    __syncthreads();
    for (int32_t w = tid; w < nwa; w += nthr) {
      uint32_t run = 0u;
      for (int32_t c = 0; c < ch; ++c) {
        const uint32_t t = part[c * nwa + w];
        part[c * nwa + w] = run;
        run |= t;
      }
      tot[w] = run;
    }
    __syncthreads();
    for (int32_t x = tid; x < ch * nwa; x += nthr) {
      const int32_t c = x / nwa, w = x - c * nwa;
      const int32_t l0 = is + c * R, l1 = min(l0 + R, m);
      uint32_t run = part[x];
#pragma unroll 8
      for (int32_t l = l0; l < l1; ++l) {
        const uint32_t v = word(l, w);
        const uint32_t nw = v & ~run;
        if (nw) atomicAdd(&hist[l - is], __popc(nw));
        run |= v;
      }
    }
  } else if (nab > 0) {
    // every (row, ancestor word) pair independently, TAIL_ILP pairs a thread
    // per round with all their loads issued first, so that many loads are in
    // flight; thread tid starts at pair tid and steps nthr pairs (dl rows and
    // dw words) at a time
    constexpr int TAIL_ILP = 8;
    const int64_t npair = (int64_t)L * nwa;
    const int32_t dl = nthr / nwa, dw = nthr % nwa;
    int32_t l = is + tid / nwa, w = wa + tid % nwa;
    for (int64_t x0 = tid; x0 < npair; x0 += (int64_t)TAIL_ILP * nthr) {
      uint32_t s[TAIL_ILP];
      int32_t ls[TAIL_ILP], ws[TAIL_ILP];
#pragma unroll
      for (int k = 0; k < TAIL_ILP; ++k) {
        ls[k] = l;
        ws[k] = w;
        s[k] = x0 + (int64_t)k * nthr < npair ? rows[tri_off(l, W) - (l >> 5) + w] : 0u;
        l += dl;
        w += dw;
        if (w >= W) {
          w -= nwa;
          ++l;
        }
      }
#pragma unroll
      for (int k = 0; k < TAIL_ILP; ++k) {
        uint32_t v = s[k];
        if (ws[k] == wa) v &= amask0;
        while (v) {
          const int bt = __ffs(v) - 1;
          v &= v - 1;
          atomicMin(&first[ws[k] * 32 + bt - m], ls[k]);
        }
      }
    }
    __syncthreads();
    for (int32_t u = tid; u < nab; u += nthr) {
      const int32_t f = first[u];
      if (f != NO_ROW) atomicAdd(&hist[f - is], 1);
    }
  }
  __syncthreads();
  int32_t run = 0;
  for (int32_t l0 = 0; l0 < L; l0 += nthr) {
    const int32_t l = l0 + tid;
    const int32_t hcount = l < L ? hist[l] : 0;
    int32_t total;
    const int32_t ex = block_excl_scan_i32(hcount, &total, red);
    if (l >= 1 && l < L) {
      const int32_t j = is + l;
      const int32_t cc = (m - 1 - j) + run + ex + hcount + 1;
      a.colcount[b + j] = cc;
      nnz += (unsigned long long)cc;
      fl += (unsigned long long)cc * (unsigned long long)cc;
    }
    run += total;
  }
  // the last column: its structure is every ancestor column met; its parent
  // is the first of them (warp 0), its element goes out with the whole CTA
  __shared__ int32_t s_pf;
  if (tid < 32) {
    int32_t pf = -1;
    if (run != 0 && por) {
      int32_t cmin = 0;
      for (int32_t w0 = 0; w0 < nwa; w0 += 32) {
        const int32_t w = w0 + lane;
        const uint32_t x = w < nwa ? tot[w] : 0u;
        const unsigned bal = __ballot_sync(0xffffffffu, x != 0u);
        if (bal) {
          const int src = __ffs(bal) - 1;
          const uint32_t xs = __shfl_sync(0xffffffffu, x, src);
          cmin = (wa + w0 + src) * 32 + __ffs(xs) - 1;
          break;
        }
      }
      pf = upos[cmin];
    } else if (run != 0) {
      int32_t umin = 0;
      for (int32_t u0 = 0; u0 < nab; u0 += 32) {
        const int32_t u = u0 + lane;
        const unsigned bal = __ballot_sync(0xffffffffu, u < nab && first[u] != NO_ROW);
        if (bal) {
          umin = u0 + __ffs(bal) - 1;
          break;
        }
      }
      pf = upos[m + umin];
    }
    if (lane == 0) {
      a.parent[b + m - 1] = pf;
      s_pf = pf;
    }
  }
  __syncthreads();
  const int32_t pf = s_pf;
  if (run != 0 && !a.node_fill) {
    if (por) {
      export_element_block(a, upos, W, (uint32_t)run, pf,
                           [&](int w) -> uint32_t { return w >= wa ? tot[w - wa] : 0u; }, red);
    } else {
      export_element_block(a, upos + m, (nab + 31) >> 5, (uint32_t)run, pf, [&](int w) -> uint32_t {
        const int32_t u = w * 32;
        uint32_t x = 0u;
        for (int k = 0; k < 32; ++k)
          if (u + k < nab && first[u + k] != NO_ROW) x |= 1u << k;
        return x;
      }, red);
    }
  }
}

// One node per CTA. Used with 64 or 128 threads for launches of many small
// nodes (the first warp sweeps, all gather; a node that does not fit in
// shared memory is deferred to a.big_list) and with SB_THREADS threads
// (launches of at most 148 nodes, or the deferred list; rows that do not fit
// go to the global pool).
__global__ void __launch_bounds__(SB_THREADS) k_symbolic_nodes(SymArgs a, int32_t smem_words, int32_t from_list,
                                                               int32_t may_defer) {
  FP_PDL_WAIT();
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ int32_t s_ab[32], s_ao[32];
  __shared__ int32_t s_na, s_atot, s_fail, s_is, s_cnt;
  __shared__ uint32_t* s_bitmap;
  __shared__ int32_t* s_wpre;
  __shared__ uint32_t* s_rows;
  __shared__ int32_t* s_upos;
  __shared__ int32_t* s_tail;
  __shared__ __align__(8) int32_t red[80];
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
  unsigned long long nnz = 0, fl = 0;
  const int32_t count = from_list ? *a.big_count : (a.in_list ? a.in_count : a.T);

  for (int32_t q = blockIdx.x; q < count; q += gridDim.x) {
    const int32_t t = from_list ? a.big_list[q] : (a.in_list ? a.in_list[q] : a.t0 + q);
    const int32_t m = a.node_size[t];
    if (m == 0) continue;
    const unsigned long long nnz0 = nnz;
    const int32_t b = a.node_begin[t];
    const int32_t end = b + m;
    if (tid < 32) {
      const int32_t na = 31 - __clz(t + 1);    // the ancestors of t, nearest first
      int32_t s = 0, bg = 0;
      if (lane < na) {
        const int32_t x = ((t + 1) >> (lane + 1)) - 1;
        bg = a.node_begin[x];
        s = a.node_size[x];
      }
      const int32_t inc = warp_incl_scan_i32(s);
      s_ab[lane] = bg;
      s_ao[lane] = inc - s;
      if (lane == 31) {
        s_na = na;
        s_atot = inc;
      }
    }
    __syncthreads();
    const int32_t na = s_na, atot = s_atot, bw = (atot + 31) >> 5;
    int32_t cur = 0;   // shared-memory words taken so far (every thread tracks it)
    int32_t lim = smem_words;   // below the gathered list while it is in use
    auto take = [&](int64_t words, bool& in_smem) -> int64_t {
      words = (words + 3) & ~3ll;     // keep every region 16-byte aligned
      if (cur + words <= lim) {
        in_smem = true;
        const int64_t o = cur;
        cur += (int32_t)words;
        return o;
      }
      in_smem = false;
      return -1;
    };
    // 1. bitmap of the reachable ancestor columns
    bool bm_smem = false;
    const int64_t bm_off = take(2 * (int64_t)bw, bm_smem);
    if (tid == 0) {
      s_fail = 0;
      s_cnt = 0;
      if (bm_smem) {
        s_bitmap = sm + bm_off;
      } else if (may_defer) {
        s_fail = 2;
      } else {
        const unsigned long long o = atomicAdd(a.pool_ctr, (unsigned long long)r4(2 * bw));
        if ((int64_t)(o + r4(2 * bw)) > a.pool_words) { s_fail = 1; atomicOr(a.status, ST_POOL_OVERFLOW); }
        s_bitmap = a.pool + o;
      }
      s_wpre = (int32_t*)(s_bitmap + bw);
    }
    __syncthreads();
    if (s_fail) {
      if (s_fail == 2 && tid == 0) a.big_list[atomicAdd(a.big_count, 1)] = t;
      continue;
    }
    uint32_t* bitmap = s_bitmap;
    int32_t* wpre = s_wpre;
    for (int32_t w = tid; w < bw; w += nthr) bitmap[w] = 0u;
    __syncthreads();
    // the list of (column, position) pairs fills shared memory down from the
    // top, above everything taken so far
    const int32_t cur_bm = cur;
    const int32_t cap = (smem_words - cur) / 2;
    int2* top = reinterpret_cast<int2*>(sm + smem_words);
    gather_entries(a, t, b, m, s_ab, s_ao, na, bitmap, top, cap, &s_cnt);
    __syncthreads();
    const int32_t npairs = s_cnt;
    int32_t acnt = 0;
    for (int32_t w0 = 0; w0 < bw; w0 += nthr) {
      const int32_t w = w0 + tid;
      const int32_t c = w < bw ? __popc(bitmap[w]) : 0;
      int32_t tot;
      const int32_t ex = block_excl_scan_i32(c, &tot, red);
      if (w < bw) wpre[w] = acnt + ex;
      acnt += tot;
    }
    const int32_t U = m + acnt;
    const int32_t W = (U + 31) >> 5;
    const int64_t row_words = tri_off(m, W);
    // 2. placement: the local->position map, the rows, the tail scratch --
    // below the list when it is complete and they fit there, else the list is
    // dropped and the seeding gathers again
    bool use_list = npairs <= cap;
    bool up_smem = false, rw_smem = false, tl_smem = false;
    int64_t up_off = -1, rw_off = -1, tl_off = -1;
    const bool tail_in_bitmap = 2 * (int64_t)bw >= U && bm_smem;
    for (int pass = use_list ? 0 : 1; pass < 2; ++pass) {
      cur = cur_bm;
      lim = pass == 0 ? (smem_words - 2 * npairs) & ~3 : smem_words;
      up_off = take(U, up_smem);
      rw_off = up_smem ? take(row_words, rw_smem) : (rw_smem = false, -1);
      tl_off = tail_in_bitmap ? -1 : take(U, tl_smem);
      if (pass == 0 && up_smem && rw_smem) break;
      use_list = false;
    }
    if (tid == 0) {
      if (may_defer && !(up_smem && rw_smem)) {
        s_fail = 2;
      } else {
        int64_t gwords = (up_smem ? 0 : r4(U)) + (rw_smem ? 0 : r4(row_words));
        uint32_t* g = nullptr;
        if (gwords > 0) {
          const unsigned long long o = atomicAdd(a.pool_ctr, (unsigned long long)gwords);
          if ((int64_t)(o + gwords) > a.pool_words) { s_fail = 1; atomicOr(a.status, ST_POOL_OVERFLOW); }
          g = a.pool + o;
        }
        s_upos = up_smem ? (int32_t*)(sm + up_off) : (int32_t*)g;
        s_rows = rw_smem ? sm + rw_off : (up_smem ? g : g + r4(U));
        if (tail_in_bitmap) {
          s_tail = (int32_t*)bitmap;
        } else if (tl_smem) {
          s_tail = (int32_t*)(sm + tl_off);
        } else if (!may_defer && !s_fail) {
          const unsigned long long o = atomicAdd(a.pool_ctr, (unsigned long long)r4(U));
          s_tail = (int64_t)(o + r4(U)) <= a.pool_words ? (int32_t*)(a.pool + o) : nullptr;
        } else {
          s_tail = nullptr;
        }
      }
    }
    __syncthreads();
    if (s_fail) {
      if (s_fail == 2 && tid == 0) a.big_list[atomicAdd(a.big_count, 1)] = t;
      continue;
    }
    uint32_t* rows = s_rows;
    int32_t* upos = s_upos;
    auto local_of = [&](int32_t pos) -> int32_t {
      if (pos < end) return pos - b;
      const int32_t c = anc_coord(s_ab, s_ao, na, pos);
      const int32_t w = c >> 5;
      return m + wpre[w] + __popc(bitmap[w] & ((1u << (c & 31)) - 1u));
    };
    for (int64_t i = tid; i < r4(row_words) / 4; i += nthr) reinterpret_cast<uint4*>(rows)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int32_t i = tid; i < m; i += nthr) upos[i] = b + i;
    for (int32_t w = tid; w < bw; w += nthr) {
      uint32_t x = bitmap[w];
      if (!x) continue;
      int32_t r = m + wpre[w];
      // the range of the word's first bit by binary search, later bits by
      // stepping forward (ranges grow with the coordinate)
      int32_t i = 0;
      {
        const int32_t c = w * 32 + __ffs(x) - 1;
#pragma unroll
        for (int st = 16; st; st >>= 1)
          if (i + st < na && s_ao[i + st] <= c) i += st;
      }
      int32_t base = s_ab[i] - s_ao[i];
      int32_t nb = i + 1 < na ? s_ao[i + 1] : INT_MAX;
      while (x) {
        const int bt = __ffs(x) - 1;
        x &= x - 1;
        const int32_t c = w * 32 + bt;
        while (c >= nb) {
          ++i;
          base = s_ab[i] - s_ao[i];
          nb = i + 1 < na ? s_ao[i + 1] : INT_MAX;
        }
        upos[r++] = base + c;
      }
    }
    __syncthreads();
    // seed the column rows: adjacency above the column, then the elements
    if (use_list) {
      for (int32_t q = tid; q < npairs; q += nthr) {
        const int2 e = top[-1 - q];
        const int32_t l = local_of(e.y);
        atomicOr(&rows[tri_off(e.x, W) - (e.x >> 5) + (l >> 5)], 1u << (l & 31));
      }
    } else {
      const int32_t e0 = a.prow[b], e1 = a.prow[b + m];
      for (int32_t e = e0 + tid; e < e1; e += nthr) {
        const int2 pq = a.ppair[e];
        if (pq.y > pq.x) {
          const int32_t i = pq.x - b, l = local_of(pq.y);
          atomicOr(&rows[tri_off(i, W) - (i >> 5) + (l >> 5)], 1u << (l & 31));
        }
      }
      for (int32_t el = a.elem_head[t]; el >= 0; el = a.elem_hdr[3 * el]) {
        const int32_t off = a.elem_hdr[3 * el + 1], len = a.elem_hdr[3 * el + 2];
        const int32_t r0 = a.elem_data[off] - b;      // smallest entry: a column of this node
        uint32_t* r = rows + tri_off(r0, W) - (r0 >> 5);
        for (int32_t j = 1 + tid; j < len; j += nthr) {
          const int32_t l = local_of(a.elem_data[off + j]);
          atomicOr(&r[l >> 5], 1u << (l & 31));
        }
      }
    }
    __syncthreads();
    // 3. column sweep by warp 0, unrolled for the row width
    const bool tail_ok = s_tail != nullptr;
    if (tid < 32) {
      const int nch = (W + 31) >> 5;
      int32_t is;
      if (nch <= 1) is = sweep_columns<1>(a, rows, upos, m, W, b, tail_ok, nnz, fl);
      else if (nch <= 2) is = sweep_columns<2>(a, rows, upos, m, W, b, tail_ok, nnz, fl);
      else if (nch <= 4) is = sweep_columns<4>(a, rows, upos, m, W, b, tail_ok, nnz, fl);
      else if (nch <= 8) is = sweep_columns<8>(a, rows, upos, m, W, b, tail_ok, nnz, fl);
      else is = sweep_columns<0>(a, rows, upos, m, W, b, tail_ok, nnz, fl);
      if (lane == 0) s_is = is;
    }
    __syncthreads();
    // 4. dense tail
    if (s_is < m) dense_tail(a, rows, upos, m, U, W, b, s_is, s_tail, red, nnz, fl);
    __syncthreads();
    if (a.node_fill) {
      const unsigned long long f = block_sum(nnz - nnz0, (unsigned long long*)red);
      if (tid == 0) a.node_fill[t] = (int64_t)f;
    }
  }
  nnz = warp_sum(nnz);
  fl = warp_sum(fl);
  if (lane == 0 && (nnz || fl)) {
    atomicAdd(&a.sums[0], nnz);
    atomicAdd(&a.sums[1], fl);
  }
}

__global__ void k_fill_u64(unsigned long long* p, unsigned long long v, int64_t n) {
  FP_PDL_WAIT();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

// B's pattern by rows in position order (row p = the neighbours of vertex
// perm[p], at their positions), so that the columns of a tree node, which
// hold consecutive positions, own one contiguous slab. deg[p] = |adj(perm[p])|
// for p < n and deg[n] = 0, for the exclusive scan that gives prow.
__global__ void k_perm_degrees(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ perm, int32_t n,
                               int32_t* __restrict__ deg) {
  FP_PDL_WAIT();
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p <= n; p += gridDim.x * blockDim.x) {
    int32_t d = 0;
    if (p < n) {
      const int32_t x = perm[p];
      d = rowptr[x + 1] - rowptr[x];
    }
    deg[p] = d;
  }
}

// One thread per row: its neighbours' positions, PP_ILP at a time.
constexpr int PP_ILP = 8;
__global__ void k_perm_pairs(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const int32_t* __restrict__ perm, const int32_t* __restrict__ iperm,
                             const int32_t* __restrict__ prow, int32_t n, int2* __restrict__ ppair) {
  FP_PDL_WAIT();
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int32_t x = perm[p];
    const int32_t e0 = rowptr[x], d = rowptr[x + 1] - e0, o = prow[p];
    for (int32_t k0 = 0; k0 < d; k0 += PP_ILP) {
      int32_t u[PP_ILP];
#pragma unroll
      for (int k = 0; k < PP_ILP; ++k) u[k] = k0 + k < d ? col[e0 + k0 + k] : -1;
#pragma unroll
      for (int k = 0; k < PP_ILP; ++k) u[k] = u[k] >= 0 ? iperm[u[k]] : -1;
#pragma unroll
      for (int k = 0; k < PP_ILP; ++k)
        if (k0 + k < d) ppair[o + k0 + k] = make_int2(p, u[k]);
    }
  }
}

}  // namespace

// Builds the position-ordered slab of B = P G P^T for perm/iperm; the caller
// frees *prow and *ppair.
static fp_status build_perm_pairs(fp_handle* h, const int32_t* perm, const int32_t* iperm, int32_t** prow,
                                  int2** ppair) {
  const int32_t n = h->n;
  int32_t* deg = (int32_t*)dev_alloc(h, sizeof(int32_t) * ((int64_t)n + 1));
  int32_t* tmp = (int32_t*)dev_alloc(h, sizeof(int32_t) * (scan_tmp_ints((int64_t)n + 1) + 8));
  *prow = (int32_t*)dev_alloc(h, sizeof(int32_t) * ((int64_t)n + 1));
  *ppair = (int2*)dev_alloc(h, sizeof(int2) * (h->nnz > 0 ? h->nnz : 1));
  if (!deg || !tmp || !*prow || !*ppair) return fail(h, FP_ERR_OUT_OF_MEMORY, "symbolic pattern");
  const int G = grid_for((int64_t)n + 1, 256);
  FP_LAUNCH(h, k_perm_degrees, G, 256, 0, h->rowptr, perm, n, deg);
  scan_exclusive(h, deg, *prow, (int64_t)n + 1, tmp);
  FP_LAUNCH(h, k_perm_pairs, G, 256, 0, h->rowptr, h->col, perm, iperm, *prow, n, *ppair);
  dev_free(h, deg);
  dev_free(h, tmp);
  return FP_OK;
}

fp_status run_symbolic(fp_handle* h, int32_t* d_parent, int32_t* d_colcount, int64_t* nnzL, int64_t* flops) {
  const int32_t n = h->n;
  const int64_t nn = h->nnodes;
  *nnzL = 0;
  *flops = 0;
  if (n == 0) return FP_OK;
  if (h->D + 1 > SYM_MAX_ANC) return fail(h, FP_ERR_UNSUPPORTED, "tree deeper than 31 levels");
  int64_t cap_hdr = (int64_t)n + 1024, cap_data = 8 * (int64_t)n + (1 << 20), pool_words = 4 * (int64_t)n + (1 << 22);
  int32_t* prow = nullptr;
  int2* ppair = nullptr;
  FP_TRY(build_perm_pairs(h, h->perm, h->iperm, &prow, &ppair));
  // launch lists: every leaf (no non-empty child; they need no other node's
  // result), largest first, in one launch; then the inner nodes depth by
  // depth, deepest first (a node's elements come from its descendants)
  if ((int64_t)h->node_size_host.size() != nn) {
    h->node_size_host.assign(nn, 0);
    cudaError_t e = cudaMemcpyAsync(h->node_size_host.data(), h->node_size, sizeof(int32_t) * nn,
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return check_cuda(h, e, "node sizes");
    int32_t st0 = 0;
    FP_TRY(sync_status(h, &st0));
  }
  const std::vector<int32_t>& hsz = h->node_size_host;
  // below[t]: some descendant of t holds vertices. A node with empty children
  // can still have them (a child split with an empty separator), and such a
  // node must wait for its descendants' elements.
  std::vector<int32_t> flat, leaves;
  std::vector<std::vector<int32_t>> inner(h->D + 1);
  std::vector<uint8_t> below(nn, 0);
  for (int64_t t = nn - 1; t >= 0; --t) {
    const int64_t c = 2 * t + 1;
    if (c < nn) below[t] = hsz[c] > 0 || hsz[c + 1] > 0 || below[c] || below[c + 1];
  }
  for (int64_t t = 0; t < nn; ++t) {
    if (hsz[t] == 0) continue;
    if (!below[t]) leaves.push_back((int32_t)t);
    else inner[63 - __builtin_clzll((unsigned long long)t + 1)].push_back((int32_t)t);
  }
  {
    // largest first, ties in node order: a counting sort by size
    int32_t smax = 0;
    for (int32_t t : leaves) smax = std::max(smax, hsz[t]);
    std::vector<int32_t> cnt((size_t)smax + 2, 0), sorted(leaves.size());
    for (int32_t t : leaves) ++cnt[(size_t)(smax - hsz[t]) + 1];
    for (size_t i = 1; i < cnt.size(); ++i) cnt[i] += cnt[i - 1];
    for (int32_t t : leaves) sorted[(size_t)cnt[(size_t)(smax - hsz[t])]++] = t;
    leaves.swap(sorted);
  }
  std::vector<std::pair<int64_t, int32_t>> launches;     // (offset in flat, count)
  std::vector<int32_t> ldepth;                            // depth of each launch's nodes (leaves: past the tree)
  launches.push_back({0, (int32_t)leaves.size()});
  ldepth.push_back(h->D + 1);
  flat = leaves;
  for (int32_t d = h->D; d >= 0; --d) {
    if (inner[d].empty()) continue;
    launches.push_back({(int64_t)flat.size(), (int32_t)inner[d].size()});
    ldepth.push_back(d);
    flat.insert(flat.end(), inner[d].begin(), inner[d].end());
  }
  h->sym_early_fired = false;
  int32_t* lst = (int32_t*)dev_alloc(h, sizeof(int32_t) * (flat.size() + 1));
  if (!lst) return fail(h, FP_ERR_OUT_OF_MEMORY, "symbolic node lists");
  if (!flat.empty()) {
    cudaError_t e = cudaMemcpyAsync(lst, flat.data(), sizeof(int32_t) * flat.size(), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return check_cuda(h, e, "symbolic node lists");
  }
  for (int attempt = 0; attempt < 4; ++attempt) {
    int32_t* head = (int32_t*)dev_alloc(h, sizeof(int32_t) * nn);
    int32_t* big = (int32_t*)dev_alloc(h, sizeof(int32_t) * (nn + 64));
    int32_t* hdr = (int32_t*)dev_alloc(h, sizeof(int32_t) * 3 * cap_hdr);
    int32_t* data = (int32_t*)dev_alloc(h, sizeof(int32_t) * cap_data);
    uint32_t* pool = (uint32_t*)dev_alloc(h, sizeof(uint32_t) * pool_words);
    // [0..1] sums, [2..3] element counters, [4 + j] the scratch-pool counter of launch j
    unsigned long long* ctr = (unsigned long long*)dev_alloc(h, sizeof(unsigned long long) * (8 + 32));
    if (!head || !big || !hdr || !data || !pool || !ctr) return fail(h, FP_ERR_OUT_OF_MEMORY, "symbolic workspace");
    fill_i32(h, head, -1, nn);
    fill_i32(h, big + nn, 0, 64);                 // per-launch deferred-node counts
    FP_LAUNCH(h, k_fill_u64, 1, 64, 0, ctr, 0ull, (int64_t)(8 + 32));
    allow_max_dynamic_smem(k_symbolic_nodes);
    bool early = false;
    auto fire_early = [&]() {
      if (early || attempt > 0 || !h->sym_early) return;
      cudaEvent_t ev = mark_event(h->device);
      if (ev && cudaEventRecord(ev, h->stream) == cudaSuccess) {
        h->sym_early(ev);
        early = true;
      }
    };
    for (size_t j = 0; j < launches.size(); ++j) {
      const int64_t off = launches[j].first;
      const int32_t c = launches[j].second;
      if (c == 0) continue;
      if (ldepth[j] < h->sym_early_depth) fire_early();
      // deferred nodes of launch j reuse its own stretch of `big`
      SymArgs sa{prow, ppair, h->perm, h->node_of, h->node_begin, h->node_size, 0, 0,
                 d_parent, d_colcount, ctr, head, hdr, data, cap_hdr, cap_data, ctr + 2, pool, pool_words,
                 ctr + 4 + j, big + off, big + nn + j, h->d_status, lst + off, c, nullptr};
      ProfScope ps(FP_PROF_SYMBOLIC, h->stream);
      if (c <= NUM_SMS_B300) {
        // few nodes: one large CTA each
        FP_LAUNCH(h, k_symbolic_nodes, c, SB_THREADS, (size_t)SB_SMEM_WORDS * 4, sa, SB_SMEM_WORDS, 0, 0);
      } else {
        // many small nodes: one small CTA each (its first warp sweeps the
        // columns, all of them gather); the ones that do not fit go to the
        // large CTAs afterwards. Four warps a node while every node of the
        // launch is resident at once (four such CTAs per SM), else two.
        const int thr = c <= NUM_SMS_B300 * 4 ? 128 : 64;
        FP_LAUNCH(h, k_symbolic_nodes, c, thr, (size_t)SW_SMEM_WORDS * 4, sa, SW_SMEM_WORDS, 0, 1);
        sa.in_list = nullptr;
        FP_LAUNCH(h, k_symbolic_nodes, NUM_SMS_B300, SB_THREADS, (size_t)SB_SMEM_WORDS * 4, sa, SB_SMEM_WORDS, 1,
                  0);
      }
    }
    FP_CHECK_LAUNCH(h, "symbolic");
    fire_early();          // no launch of the top levels: every column is final here
    unsigned long long hs[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(hs, ctr, sizeof(hs), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return check_cuda(h, e, "read sums");
    int32_t st = 0;
    FP_TRY(sync_status(h, &st));
    for (void* p : {(void*)head, (void*)big, (void*)hdr, (void*)data, (void*)pool, (void*)ctr}) dev_free(h, p);
    if (st & ST_POOL_OVERFLOW) {
      // clear the flag and retry with larger pools
      int32_t zero = 0;
      cudaMemcpyAsync(h->d_status, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream);
      cap_hdr *= 4; cap_data *= 4; pool_words *= 4;
      continue;
    }
    h->sym_early_fired = early;
    *nnzL = (int64_t)hs[0];
    *flops = (int64_t)hs[1];
    dev_free(h, prow);
    dev_free(h, ppair);
    dev_free(h, lst);
    return FP_OK;
  }
  return fail(h, FP_ERR_OUT_OF_MEMORY, "symbolic pools exhausted");
}

}  // namespace fp

namespace fp {

fp_status run_leaf_fill(fp_handle* h, const int32_t* perm, const int32_t* iperm, const int32_t* d_nodes,
                        int32_t count, int64_t* d_fill) {
  if (count == 0) return FP_OK;
  const int32_t n = h->n;
  const int64_t nn = h->nnodes;
  if (h->D + 1 > SYM_MAX_ANC) return fail(h, FP_ERR_UNSUPPORTED, "tree deeper than 31 levels");
  int64_t pool_words = 4 * (int64_t)n + (1 << 22);
  int32_t* prow = nullptr;
  int2* ppair = nullptr;
  FP_TRY(build_perm_pairs(h, perm, iperm, &prow, &ppair));
  for (int attempt = 0; attempt < 4; ++attempt) {
    int32_t* head = (int32_t*)dev_alloc(h, sizeof(int32_t) * nn);
    int32_t* big = (int32_t*)dev_alloc(h, sizeof(int32_t) * ((int64_t)count + 64));
    int32_t* scr = (int32_t*)dev_alloc(h, sizeof(int32_t) * 2 * (int64_t)(n > 0 ? n : 1));
    uint32_t* pool = (uint32_t*)dev_alloc(h, sizeof(uint32_t) * pool_words);
    unsigned long long* ctr = (unsigned long long*)dev_alloc(h, sizeof(unsigned long long) * 8);
    if (!head || !big || !scr || !pool || !ctr) return fail(h, FP_ERR_OUT_OF_MEMORY, "leaf fill workspace");
    fill_i32(h, head, -1, nn);
    fill_i32(h, big + count, 0, 64);
    FP_LAUNCH(h, k_fill_u64, 1, 32, 0, ctr, 0ull, (int64_t)8);
    allow_max_dynamic_smem(k_symbolic_nodes);
    // leaves export nothing and receive nothing: no element lists are needed
    SymArgs sa{prow, ppair, perm, h->node_of, h->node_begin, h->node_size, 0, 0, scr, scr + n, ctr,
               head, nullptr, nullptr, 0, 0, ctr + 2, pool, pool_words, ctr + 4, big, big + count, h->d_status,
               d_nodes, count, d_fill};
    FP_LAUNCH(h, k_symbolic_nodes, count, 64, (size_t)SW_SMEM_WORDS * 4, sa, SW_SMEM_WORDS, 0, 1);
    sa.in_list = nullptr;
    FP_LAUNCH(h, k_symbolic_nodes, NUM_SMS_B300, SB_THREADS, (size_t)SB_SMEM_WORDS * 4, sa, SB_SMEM_WORDS, 1, 0);
    FP_CHECK_LAUNCH(h, "leaf fill");
    int32_t st = 0;
    FP_TRY(sync_status(h, &st));
    for (void* p : {(void*)head, (void*)big, (void*)scr, (void*)pool, (void*)ctr}) dev_free(h, p);
    if (st & ST_POOL_OVERFLOW) {
      int32_t zero = 0;
      cudaMemcpyAsync(h->d_status, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream);
      pool_words *= 4;
      continue;
    }
    dev_free(h, prow);
    dev_free(h, ppair);
    return FP_OK;
  }
  return fail(h, FP_ERR_OUT_OF_MEMORY, "leaf fill pools exhausted");
}

}  // namespace fp
