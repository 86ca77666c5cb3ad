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
// Nodes are processed level by level from the deepest, one CTA per node:
//   1. mark A_t in a bitmap over the concatenated ancestor ranges and compact
//      it (prefix popcounts), so U_t gets dense local indices in position order;
//   2. seed one bit row per column with its adjacency and the elements whose
//      smallest entry is in V_t;
//   3. one warp sweeps the columns in order: parent = first set bit, count =
//      popc; the row is merged into its parent's row, kept in registers when the
//      parent is the next column (the chains of separator blocks), or exported
//      as an element to the node holding its parent.
// Positions of a node are contiguous in both schedules and ancestors always
// come later, so bit order equals position order.
#include "fp_device.cuh"

namespace fp {
namespace {

constexpr int SYM_THREADS = 128;
constexpr int SYM_MAX_ANC = 32;
constexpr size_t SYM_SMEM_BITMAP = 8 * 1024;    // bitmap + prefix (<= 1024 words each)
constexpr size_t SYM_SMEM_ROWS_SMALL = 40 * 1024;   // rows + local->position map, deep levels
constexpr size_t SYM_SMEM_ROWS_BIG = 208 * 1024;    // same, shallow levels (few, large nodes)

// Column i's bit row only holds words >= i/32 (its bits are all above i), so
// the rows are stored as a staircase: row i starts at tri_off(i, W).
__device__ __forceinline__ int64_t tri_off(int32_t i, int32_t W) {
  const int64_t q = i >> 5, r = i & 31;
  return (int64_t)i * W - (32 * q * (q - 1) / 2 + r * q);
}

struct SymArgs {
  const int32_t* rowptr;
  const int32_t* col;
  const int32_t* perm;
  const int32_t* iperm;
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
  uint32_t* pool;                  // per-launch scratch words
  int64_t pool_words;
  unsigned long long* pool_ctr;
  int32_t* status;
  int64_t smem_rows;               // shared bytes available for rows + map in this launch
};

// Column sweep of one node by one warp (see step 3 below). NCH > 0: rows of at
// most 32*NCH words, the current column's row is kept in registers (carry)
// while the etree parent is the next column; NCH = 0: rows of any width,
// merged through memory.
template <int NCH>
__device__ __forceinline__ void sweep_columns(const SymArgs& a, uint32_t* rows, const int32_t* upos, int32_t m,
                                              int32_t W, int32_t b, unsigned long long& nnz,
                                              unsigned long long& fl) {
  const int lane = threadIdx.x & 31;
  constexpr int NC = NCH > 0 ? NCH : 1;
  uint32_t carry[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) carry[c] = 0u;
  bool cv = false;
  for (int32_t i = 0; i < m; ++i) {
    const int i0 = i >> 5;
    const uint32_t* ri = rows + tri_off(i, W) - i0;     // word w of row i at ri[w], w >= i0
    uint32_t f = 0xffffffffu, cnt = 0;
    if constexpr (NCH > 0) {
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        const int w = lane + 32 * c;
        uint32_t s = (w < W && w >= i0) ? ri[w] : 0u;
        if (cv) s |= carry[c];
        carry[c] = s;
        if (s) { const uint32_t bt = w * 32 + __ffs(s) - 1; f = bt < f ? bt : f; cnt += __popc(s); }
      }
    } else {
      for (int w = lane; w < W; w += 32) {
        const uint32_t s = w >= i0 ? ri[w] : 0u;
        if (s) { const uint32_t bt = w * 32 + __ffs(s) - 1; f = bt < f ? bt : f; cnt += __popc(s); }
      }
    }
    f = __reduce_min_sync(0xffffffffu, f);
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    const int32_t pf = cnt ? upos[f] : -1;
    if (lane == 0) {
      a.parent[b + i] = pf;
      a.colcount[b + i] = (int32_t)cnt + 1;
      nnz += (unsigned long long)(cnt + 1);
      fl += (unsigned long long)(cnt + 1) * (unsigned long long)(cnt + 1);
    }
    if (cnt == 0) { cv = false; continue; }
    if (f >= (uint32_t)m) {
      // export struct(i) (f first) to the node holding position pf
      unsigned long long off = 0, hdr = 0;
      if (lane == 0) {
        off = atomicAdd(&a.elem_ctr[1], (unsigned long long)cnt);
        hdr = atomicAdd(&a.elem_ctr[0], 1ull);
      }
      off = __shfl_sync(0xffffffffu, off, 0);
      hdr = __shfl_sync(0xffffffffu, hdr, 0);
      const bool ok = (int64_t)(off + cnt) <= a.cap_data && (int64_t)hdr < a.cap_hdr;
      if (!ok) {
        if (lane == 0) atomicOr(a.status, ST_POOL_OVERFLOW);
      } else {
        int32_t base = 0;
        for (int w0 = 0; w0 < W; w0 += 32) {
          const int w = w0 + lane;
          uint32_t s = 0u;
          if (w < W) {
            if constexpr (NCH > 0) {
#pragma unroll
              for (int c = 0; c < NCH; ++c) if (c == (w0 >> 5)) s = carry[c];
            } else if (w >= i0) {
              s = ri[w];
            }
          }
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
      cv = false;
      continue;
    }
    // merge struct(i) \ {f} into column f
    const int f0 = (int)(f >> 5);
    if constexpr (NCH > 0) {
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        const int w = lane + 32 * c;
        if (w == f0) carry[c] &= ~(1u << (f & 31));
      }
      if (f == (uint32_t)i + 1) {
        cv = true;
      } else {
        cv = false;
        uint32_t* rf = rows + tri_off((int32_t)f, W) - f0;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          const int w = lane + 32 * c;
          if (w < W && w >= f0 && carry[c]) rf[w] |= carry[c];
        }
      }
    } else {
      uint32_t* rf = rows + tri_off((int32_t)f, W) - f0;
      for (int w = lane; w < W; w += 32) {
        if (w < f0) continue;           // struct(i) \ {f} lies above f
        uint32_t s = ri[w];
        if (w == f0) s &= ~(1u << (f & 31));
        if (s) rf[w] |= s;
      }
    }
  }
}

__global__ void __launch_bounds__(SYM_THREADS) k_symbolic_level(SymArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int32_t anc_b[SYM_MAX_ANC], anc_s[SYM_MAX_ANC], anc_o[SYM_MAX_ANC];
  __shared__ int32_t s_na, s_atot;
  __shared__ int32_t red[40];
  __shared__ uint32_t* s_bitmap;
  __shared__ int32_t* s_wpre;
  __shared__ uint32_t* s_rows;
  __shared__ int32_t* s_upos;
  __shared__ int32_t s_fail;
  const int tid = threadIdx.x, lane = tid & 31;

  for (int32_t ni = blockIdx.x; ni < a.T; ni += gridDim.x) {
    const int32_t t = a.t0 + ni;
    const int32_t m = a.node_size[t];
    if (m == 0) continue;
    const int32_t b = a.node_begin[t];
    if (tid == 0) {
      int32_t na = 0, off = 0, x = t;
      while (x > 0 && na < SYM_MAX_ANC) {
        x = (x - 1) / 2;
        anc_b[na] = a.node_begin[x];
        anc_s[na] = a.node_size[x];
        anc_o[na] = off;
        off += anc_s[na];
        ++na;
      }
      s_na = na;
      s_atot = off;
      s_fail = 0;
      const int32_t bw = (off + 31) >> 5;
      if ((size_t)bw * 8 <= SYM_SMEM_BITMAP) {
        s_bitmap = (uint32_t*)smem;
        s_wpre = (int32_t*)(smem + SYM_SMEM_BITMAP / 2);
      } else {
        unsigned long long o = atomicAdd(a.pool_ctr, (unsigned long long)(2 * bw + 2));
        if ((int64_t)(o + 2 * bw + 2) > a.pool_words) { s_fail = 1; atomicOr(a.status, ST_POOL_OVERFLOW); }
        s_bitmap = a.pool + o;
        s_wpre = (int32_t*)(a.pool + o + bw + 1);
      }
    }
    __syncthreads();
    if (s_fail) continue;
    const int32_t na = s_na, atot = s_atot, bw = (atot + 31) >> 5;
    uint32_t* bitmap = s_bitmap;
    int32_t* wpre = s_wpre;
    auto anc_coord = [&](int32_t pos) -> int32_t {
      for (int i = 0; i < na; ++i)
        if (pos >= anc_b[i] && pos < anc_b[i] + anc_s[i]) return anc_o[i] + pos - anc_b[i];
      return -1;
    };
    for (int32_t w = tid; w < bw; w += SYM_THREADS) bitmap[w] = 0u;
    __syncthreads();
    // 1. mark the ancestors reachable from this node
    const int32_t end = b + m;
    for (int32_t i = tid; i < m; i += SYM_THREADS) {
      const int32_t x = a.perm[b + i];
      for (int32_t e = a.rowptr[x]; e < a.rowptr[x + 1]; ++e) {
        const int32_t pos = a.iperm[a.col[e]];
        if (pos >= end) {
          const int32_t c = anc_coord(pos);
          atomicOr(&bitmap[c >> 5], 1u << (c & 31));
        }
      }
    }
    for (int32_t el = a.elem_head[t]; el >= 0; el = a.elem_hdr[3 * el]) {
      const int32_t off = a.elem_hdr[3 * el + 1], len = a.elem_hdr[3 * el + 2];
      for (int32_t j = tid; j < len; j += SYM_THREADS) {
        const int32_t pos = a.elem_data[off + j];
        if (pos >= end) {
          const int32_t c = anc_coord(pos);
          atomicOr(&bitmap[c >> 5], 1u << (c & 31));
        }
      }
    }
    __syncthreads();
    int32_t acnt = 0;
    for (int32_t w0 = 0; w0 < bw; w0 += SYM_THREADS) {
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
    if (tid == 0) {
      const int64_t need = (row_words + U) * 4;
      if (need <= a.smem_rows) {
        s_rows = (uint32_t*)(smem + SYM_SMEM_BITMAP);
      } else {
        const unsigned long long words = (unsigned long long)(row_words + U);
        unsigned long long o = atomicAdd(a.pool_ctr, words);
        if ((int64_t)(o + words) > a.pool_words) { s_fail = 1; atomicOr(a.status, ST_POOL_OVERFLOW); }
        s_rows = a.pool + o;
      }
      s_upos = (int32_t*)(s_rows + row_words);
    }
    __syncthreads();
    if (s_fail) continue;
    uint32_t* rows = s_rows;
    int32_t* upos = s_upos;
    auto local_of = [&](int32_t pos) -> int32_t {
      if (pos < end) return pos - b;
      const int32_t c = anc_coord(pos);
      const int32_t w = c >> 5;
      return m + wpre[w] + __popc(bitmap[w] & ((1u << (c & 31)) - 1u));
    };
    for (int64_t i = tid; i < row_words; i += SYM_THREADS) rows[i] = 0u;
    for (int32_t i = tid; i < m; i += SYM_THREADS) upos[i] = b + i;
    for (int32_t w = tid; w < bw; w += SYM_THREADS) {
      uint32_t x = bitmap[w];
      int32_t r = m + wpre[w];
      while (x) {
        const int bt = __ffs(x) - 1;
        x &= x - 1;
        const int32_t c = w * 32 + bt;
        int32_t pos = -1;
        for (int i = 0; i < na; ++i)
          if (c >= anc_o[i] && c < anc_o[i] + anc_s[i]) { pos = anc_b[i] + c - anc_o[i]; break; }
        upos[r++] = pos;
      }
    }
    __syncthreads();
    // 2. seed the column rows: adjacency above the column, then the elements
    for (int32_t i = tid; i < m; i += SYM_THREADS) {
      const int32_t x = a.perm[b + i];
      uint32_t* r = rows + tri_off(i, W) - (i >> 5);
      for (int32_t e = a.rowptr[x]; e < a.rowptr[x + 1]; ++e) {
        const int32_t pos = a.iperm[a.col[e]];
        if (pos > b + i) {
          const int32_t l = local_of(pos);
          atomicOr(&r[l >> 5], 1u << (l & 31));
        }
      }
    }
    for (int32_t el = a.elem_head[t]; el >= 0; el = a.elem_hdr[3 * el]) {
      const int32_t off = a.elem_hdr[3 * el + 1], len = a.elem_hdr[3 * el + 2];
      const int32_t r0 = a.elem_data[off] - b;      // smallest entry: a column of this node
      uint32_t* r = rows + tri_off(r0, W) - (r0 >> 5);
      for (int32_t j = 1 + tid; j < len; j += SYM_THREADS) {
        const int32_t l = local_of(a.elem_data[off + j]);
        atomicOr(&r[l >> 5], 1u << (l & 31));
      }
    }
    __syncthreads();
    // 3. column sweep by warp 0, unrolled for the row width
    if (tid < 32) {
      unsigned long long nnz = 0, fl = 0;
      const int nch = (W + 31) >> 5;
      if (nch <= 1) sweep_columns<1>(a, rows, upos, m, W, b, nnz, fl);
      else if (nch <= 2) sweep_columns<2>(a, rows, upos, m, W, b, nnz, fl);
      else if (nch <= 4) sweep_columns<4>(a, rows, upos, m, W, b, nnz, fl);
      else if (nch <= 8) sweep_columns<8>(a, rows, upos, m, W, b, nnz, fl);
      else sweep_columns<0>(a, rows, upos, m, W, b, nnz, fl);
      if (lane == 0) {
        atomicAdd(&a.sums[0], nnz);
        atomicAdd(&a.sums[1], fl);
      }
    }
    __syncthreads();
  }
}

__global__ void k_fill_u64(unsigned long long* p, unsigned long long v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

}  // namespace

fp_status run_symbolic(fp_handle* h, int32_t* d_parent, int32_t* d_colcount, int64_t* nnzL, int64_t* flops) {
  const int32_t n = h->n;
  const int64_t nn = h->nnodes;
  *nnzL = 0;
  *flops = 0;
  if (n == 0) return FP_OK;
  if (h->D + 1 > SYM_MAX_ANC) return fail(h, FP_ERR_UNSUPPORTED, "tree deeper than 31 levels");
  int64_t cap_hdr = (int64_t)n + 1024, cap_data = 8 * (int64_t)n + (1 << 20), pool_words = 4 * (int64_t)n + (1 << 22);
  for (int attempt = 0; attempt < 4; ++attempt) {
    int32_t* head = (int32_t*)dev_alloc(h, sizeof(int32_t) * nn);
    int32_t* hdr = (int32_t*)dev_alloc(h, sizeof(int32_t) * 3 * cap_hdr);
    int32_t* data = (int32_t*)dev_alloc(h, sizeof(int32_t) * cap_data);
    uint32_t* pool = (uint32_t*)dev_alloc(h, sizeof(uint32_t) * pool_words);
    unsigned long long* ctr = (unsigned long long*)dev_alloc(h, sizeof(unsigned long long) * 8);
    if (!head || !hdr || !data || !pool || !ctr) return fail(h, FP_ERR_OUT_OF_MEMORY, "symbolic workspace");
    fill_i32(h, head, -1, nn);
    FP_LAUNCH(h, k_fill_u64, 1, 32, 0, ctr, 0ull, (int64_t)8);
    allow_max_dynamic_smem(k_symbolic_level);
    for (int32_t d = h->D; d >= 0; --d) {
      const int32_t t0 = (1 << d) - 1, T = 1 << d;
      // shallow levels hold few, large nodes: one CTA per SM with most of its
      // shared memory; deep levels hold many small nodes: several CTAs per SM
      const size_t rows_smem = T <= 2 * NUM_SMS_B300 ? SYM_SMEM_ROWS_BIG : SYM_SMEM_ROWS_SMALL;
      SymArgs sa{h->rowptr, h->col, h->perm, h->iperm, h->node_of, h->node_begin, h->node_size, t0, T,
                 d_parent, d_colcount, ctr, head, hdr, data, cap_hdr, cap_data, ctr + 2, pool, pool_words,
                 ctr + 4, h->d_status, (int64_t)rows_smem};
      ProfScope ps(FP_PROF_SYMBOLIC, h->stream);
      FP_LAUNCH(h, k_fill_u64, 1, 32, 0, ctr + 4, 0ull, (int64_t)1);
      const int grid = T < NUM_SMS_B300 * 16 ? T : NUM_SMS_B300 * 16;
      FP_LAUNCH(h, k_symbolic_level, grid, SYM_THREADS, SYM_SMEM_BITMAP + rows_smem, sa);
    }
    FP_CHECK_LAUNCH(h, "symbolic");
    unsigned long long hs[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(hs, ctr, sizeof(hs), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return check_cuda(h, e, "read sums");
    int32_t st = 0;
    FP_TRY(sync_status(h, &st));
    for (void* p : {(void*)head, (void*)hdr, (void*)data, (void*)pool, (void*)ctr}) dev_free(h, p);
    if (st & ST_POOL_OVERFLOW) {
      // clear the flag and retry with larger pools
      int32_t zero = 0;
      cudaMemcpyAsync(h->d_status, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream);
      cap_hdr *= 4; cap_data *= 4; pool_words *= 4;
      continue;
    }
    *nnzL = (int64_t)hs[0];
    *flops = (int64_t)hs[1];
    return FP_OK;
  }
  return fail(h, FP_ERR_OUT_OF_MEMORY, "symbolic pools exhausted");
}

}  // namespace fp
