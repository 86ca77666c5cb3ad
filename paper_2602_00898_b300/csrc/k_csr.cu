// a1 CSR assembly (Section 2; Section 4.1 step 2): G = graph of A without its
// diagonal, as a symmetric CSR with sorted, duplicate-free rows.
//
// No global sort: each corner pair is counted and scattered into its row's
// raw segment (atomics), then every row is sorted and deduplicated on chip
// (one thread per row of at most 32 raw entries, sorted in registers; a warp
// per longer row in shared memory; a CTA per row above 256), and the unique
// entries are compacted. Three streaming passes over the faces and two over
// the raw rows: HBM-bound.
#include <climits>

#include "fp_device.cuh"

namespace fp {
namespace {

constexpr int WARP_ROW_CAP = 256;    // rows up to this many raw entries: one warp
constexpr int BLOCK_ROW_CAP = 8192;  // longer rows: one CTA; beyond: unsupported
constexpr int ROW_WARPS = 8;         // warps per CTA in the warp-per-row kernel

// ---- faces ------------------------------------------------------------------------

// Counts the raw entries of every row; the count each increment returns is the
// entry's slot in its row, kept (for every face edge, its slot in both end
// rows) so that the fill pass places entries without atomics. Each corner
// takes the slots of its two face edges (fewer where an edge is degenerate)
// with one atomic: three a face.
__global__ void k_face_count(const int32_t* __restrict__ faces, int64_t nf, int32_t n, int32_t* __restrict__ cnt,
                             int2* __restrict__ slots, int32_t* status) {
  FP_PDL_WAIT();
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    int32_t c[3] = {faces[3 * f], faces[3 * f + 1], faces[3 * f + 2]};
    if (c[0] < 0 || c[0] >= n || c[1] < 0 || c[1] >= n || c[2] < 0 || c[2] >= n) {
      atomicOr(status, ST_BAD_INDEX);
      continue;
    }
    // corner i owns edge i = (c[i], c[i+1]) first, then edge i-1 = (c[i-1], c[i])
    int32_t out[3], base[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) out[i] = c[i] != c[(i + 1) % 3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int32_t k = out[i] + out[(i + 2) % 3];
      base[i] = k ? atomicAdd(&cnt[c[i]], k) : 0;
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int j = (e + 1) % 3;
      slots[3 * f + e] = out[e] ? make_int2(base[e], base[j] + out[j]) : make_int2(0, 0);
    }
  }
}

__global__ void k_face_fill(const int32_t* __restrict__ faces, int64_t nf, int32_t n, const int32_t* __restrict__ off,
                            const int2* __restrict__ slots, int32_t* __restrict__ raw) {
  FP_PDL_WAIT();
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    int32_t c[3] = {faces[3 * f], faces[3 * f + 1], faces[3 * f + 2]};
    if (c[0] < 0 || c[0] >= n || c[1] < 0 || c[1] >= n || c[2] < 0 || c[2] >= n) continue;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int32_t a = c[e], b = c[(e + 1) % 3];
      if (a == b) continue;
      const int2 sl = slots[3 * f + e];
      raw[off[a] + sl.x] = b;
      raw[off[b] + sl.y] = a;
    }
  }
}

// ---- CSR pattern (scalar or b x b blocks) -------------------------------------------

__global__ void k_pat_count(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int32_t nrows, int32_t b,
                            int32_t* __restrict__ cnt, int32_t* status) {
  FP_PDL_WAIT();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += gridDim.x * blockDim.x) {
    int32_t u = i / b, c = 0;
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
      int32_t j = col[e];
      if (j < 0 || j >= nrows) { atomicOr(status, ST_BAD_INDEX); continue; }
      c += (j / b != u);
    }
    if (c) atomicAdd(&cnt[u], c);
  }
}

__global__ void k_pat_fill(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int32_t nrows, int32_t b,
                           const int32_t* __restrict__ off, int32_t* __restrict__ fill, int32_t* __restrict__ raw) {
  FP_PDL_WAIT();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += gridDim.x * blockDim.x) {
    int32_t u = i / b, c = 0;
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
      int32_t j = col[e];
      c += (j >= 0 && j < nrows && j / b != u);
    }
    if (!c) continue;
    int32_t slot = off[u] + atomicAdd(&fill[u], c);
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
      int32_t j = col[e];
      if (j >= 0 && j < nrows && j / b != u) raw[slot++] = j / b;
    }
  }
}

// ---- row sort + dedupe ----------------------------------------------------------------

__device__ __forceinline__ int next_pow2(int x) {
  int p = 32;
  while (p < x) p <<= 1;
  return p;
}

// Sorts a row of at most N raw entries in registers and writes its unique
// prefix back in place; returns its length.
template <int N>
__device__ __forceinline__ int32_t dedupe_row_regs(int32_t* __restrict__ raw, int32_t b, int32_t L) {
  int32_t x[N];
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = i < L ? raw[b + i] : INT_MAX;
  thread_sort_regs<N>(x);
  int32_t c = 0;
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < L && (i == 0 || x[i] != x[i - 1])) raw[b + c++] = x[i];
  return c;
}

// One thread per row of at most 32 raw entries (mesh rows hold about twelve):
// sort in registers, write the unique prefix back in place and its length to
// ucnt. Longer rows are listed for the warp kernel.
__global__ void k_rows_dedupe_thread(const int32_t* __restrict__ off, int32_t n, int32_t* __restrict__ raw,
                                     int32_t* __restrict__ ucnt, int32_t* __restrict__ mid_rows, int32_t* n_mid) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int32_t b = off[v], L = off[v + 1] - b;
    if (L > 32) {
      mid_rows[atomicAdd(n_mid, 1)] = v;
      continue;
    }
    ucnt[v] = L <= 16 ? dedupe_row_regs<16>(raw, b, L) : dedupe_row_regs<32>(raw, b, L);
  }
}

// One warp per listed row: sort the raw segment, write the unique prefix back
// in place and its length to ucnt. Rows longer than WARP_ROW_CAP are queued
// for the CTA kernel.
__global__ void __launch_bounds__(ROW_WARPS * 32) k_rows_dedupe_warp(const int32_t* __restrict__ off,
                                                                      const int32_t* __restrict__ mid_rows,
                                                                      const int32_t* n_mid, int32_t* __restrict__ raw,
                                                                      int32_t* __restrict__ ucnt,
                                                                      int32_t* __restrict__ long_rows, int32_t* n_long) {
  FP_PDL_WAIT();
  __shared__ int32_t sbuf[ROW_WARPS][WARP_ROW_CAP];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* buf = sbuf[wid];
  const int32_t nm = *n_mid;
  for (int32_t r = blockIdx.x * ROW_WARPS + wid; r < nm; r += gridDim.x * ROW_WARPS) {
    const int32_t v = mid_rows[r];
    int32_t b = off[v], L = off[v + 1] - b;
    if (L > WARP_ROW_CAP) {
      if (lane == 0) long_rows[atomicAdd(n_long, 1)] = v;
      continue;
    }
    int N = next_pow2(L);
    for (int i = lane; i < N; i += 32) buf[i] = i < L ? raw[b + i] : INT_MAX;
    __syncwarp();
    bitonic_sort<false>(buf, N, lane, 32);
    int32_t cnt = 0;
    for (int i0 = 0; i0 < L; i0 += 32) {
      int i = i0 + lane;
      bool keep = i < L && (i == 0 || buf[i] != buf[i - 1]);
      unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) raw[b + cnt + __popc(m & ((1u << lane) - 1))] = buf[i];
      cnt += __popc(m);
    }
    if (lane == 0) ucnt[v] = cnt;
    __syncwarp();
  }
}

__global__ void k_rows_dedupe_block(const int32_t* __restrict__ off, const int32_t* __restrict__ long_rows,
                                    const int32_t* n_long, int32_t* __restrict__ raw, int32_t* __restrict__ ucnt,
                                    int32_t* status) {
  FP_PDL_WAIT();
  extern __shared__ int32_t buf[];
  __shared__ int32_t warp_cnt[32];
  for (int32_t r = blockIdx.x; r < *n_long; r += gridDim.x) {
    int32_t v = long_rows[r];
    int32_t b = off[v], L = off[v + 1] - b;
    if (L > BLOCK_ROW_CAP) {
      if (threadIdx.x == 0) { atomicOr(status, ST_ROW_TOO_LONG); ucnt[v] = 0; }
      continue;
    }
    int N = next_pow2(L);
    for (int i = threadIdx.x; i < N; i += blockDim.x) buf[i] = i < L ? raw[b + i] : INT_MAX;
    __syncthreads();
    bitonic_sort<true>(buf, N, threadIdx.x, blockDim.x);
    // serial-order compaction in chunks of blockDim.x
    int32_t base = 0;
    for (int i0 = 0; i0 < L; i0 += blockDim.x) {
      int i = i0 + threadIdx.x;
      bool keep = i < L && (i == 0 || buf[i] != buf[i - 1]);
      unsigned m = __ballot_sync(0xffffffffu, keep);
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      if (lane == 0) warp_cnt[wid] = __popc(m);
      __syncthreads();
      int32_t before = 0, tot = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        if (w < wid) before += warp_cnt[w];
        tot += warp_cnt[w];
      }
      if (keep) raw[b + base + before + __popc(m & ((1u << lane) - 1))] = buf[i];
      base += tot;
      __syncthreads();
    }
    if (threadIdx.x == 0) ucnt[v] = base;
    __syncthreads();
  }
}

// Copy each row's unique prefix to its final place; thread per row (mesh rows
// hold about six entries).
__global__ void k_rows_compact(const int32_t* __restrict__ off, const int32_t* __restrict__ raw, int32_t n,
                               const int32_t* __restrict__ rowptr, int32_t* __restrict__ col) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int32_t s = off[v], d = rowptr[v], L = rowptr[v + 1] - d;
    for (int32_t i = 0; i < L; ++i) col[d + i] = raw[s + i];
  }
}

// Structural symmetry: every (u, v) must have (v, u). Warp per row, binary
// search in the sorted row of v.
__global__ void k_check_symmetric(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int32_t n,
                                  int32_t* status) {
  FP_PDL_WAIT();
  const int lane = threadIdx.x & 31;
  for (int32_t u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += (gridDim.x * blockDim.x) >> 5) {
    for (int32_t e = rowptr[u] + lane; e < rowptr[u + 1]; e += 32) {
      int32_t v = col[e];
      int32_t lo = rowptr[v], hi = rowptr[v + 1];
      while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (col[mid] < u) lo = mid + 1; else hi = mid;
      }
      if (lo >= rowptr[v + 1] || col[lo] != u) atomicOr(status, ST_NOT_SYMMETRIC);
    }
  }
}

// Shared tail: raw rows [off] -> sorted unique CSR in h->rowptr / h->col. The
// column array is sized for nraw entries (an upper bound of the unique ones);
// one host sync at the end reads the entry count and the status word
// (bad_index: the message for ST_BAD_INDEX).
fp_status finish_rows(fp_handle* h, int32_t* off, int32_t* raw, int64_t nraw, int32_t* tmp, const char* bad_index) {
  const int32_t n = h->n;
  int32_t* ucnt = (int32_t*)dev_alloc(h, sizeof(int32_t) * (n + 1));
  int32_t* long_rows = (int32_t*)dev_alloc(h, sizeof(int32_t) * (n + 1));
  int32_t* mid_rows = (int32_t*)dev_alloc(h, sizeof(int32_t) * (n + 1));
  int32_t* n_long = (int32_t*)dev_alloc(h, sizeof(int32_t) * 2);     // [0] long rows, [1] mid rows
  h->rowptr = (int32_t*)dev_alloc(h, sizeof(int32_t) * (n + 1));
  if (!ucnt || !long_rows || !mid_rows || !n_long || !h->rowptr) return fail(h, FP_ERR_OUT_OF_MEMORY, "graph workspace");
  {
  ProfScope ps(FP_PROF_GRAPH, h->stream);
  fill_i32(h, n_long, 0, 2);
  fill_i32(h, ucnt, 0, n + 1);
  if (n > 0) {
    FP_LAUNCH(h, k_rows_dedupe_thread, grid_for(n, 256), 256, 0, off, n, raw, ucnt, mid_rows, n_long + 1);
    FP_LAUNCH(h, k_rows_dedupe_warp, NUM_SMS_B300 * 8, ROW_WARPS * 32, 0, off, mid_rows, n_long + 1, raw, ucnt,
              long_rows, n_long);
    FP_LAUNCH(h, k_rows_dedupe_block, NUM_SMS_B300, 512, BLOCK_ROW_CAP * sizeof(int32_t), off, long_rows, n_long, raw,
              ucnt, h->d_status);
  }
  scan_exclusive(h, ucnt, h->rowptr, n, tmp);
  }
  FP_CHECK_LAUNCH(h, "graph rows");
  h->col = (int32_t*)dev_alloc(h, sizeof(int32_t) * (nraw > 0 ? nraw : 1));
  if (!h->col) return fail(h, FP_ERR_OUT_OF_MEMORY, "graph columns");
  if (n > 0) {
    ProfScope ps(FP_PROF_GRAPH, h->stream);
    FP_LAUNCH(h, k_rows_compact, grid_for(n, 256), 256, 0, off, raw, n, h->rowptr, h->col);
  }
  FP_CHECK_LAUNCH(h, "graph compact");
  int32_t* hb = pinned_scratch();
  if (!hb) return fail(h, FP_ERR_OUT_OF_MEMORY, "pinned scratch");
  cudaError_t e = cudaMemcpyAsync(hb, h->rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "read nnz");
  int32_t st = 0;
  FP_TRY(sync_status(h, &st));
  if (st & ST_BAD_INDEX) return fail(h, FP_ERR_INVALID_ARG, bad_index);
  if (st & ST_ROW_TOO_LONG) return fail(h, FP_ERR_UNSUPPORTED, "a vertex has more than 8192 raw adjacency entries");
  h->nnz = hb[0];
  dev_free(h, ucnt);
  dev_free(h, long_rows);
  dev_free(h, mid_rows);
  dev_free(h, n_long);
  return FP_OK;
}

}  // namespace

fp_status build_graph_from_faces(fp_handle* h, const int32_t* d_faces, int64_t nf) {
  const int32_t n = h->n;
  if (6 * nf > INT32_MAX) return fail(h, FP_ERR_UNSUPPORTED, "more than 2^31-1 adjacency entries");
  int32_t* cnt = (int32_t*)dev_alloc(h, sizeof(int32_t) * (n + 1));
  int32_t* off = (int32_t*)dev_alloc(h, sizeof(int32_t) * (n + 1));
  int32_t* tmp = (int32_t*)dev_alloc(h, sizeof(int32_t) * scan_tmp_ints(n + 1));
  int2* slots = (int2*)dev_alloc(h, sizeof(int2) * 3 * (nf > 0 ? nf : 1));
  if (!cnt || !off || !tmp || !slots) return fail(h, FP_ERR_OUT_OF_MEMORY, "graph workspace");
  {
    ProfScope ps(FP_PROF_GRAPH, h->stream);
    fill_i32(h, cnt, 0, n + 1);
    if (nf > 0) FP_LAUNCH(h, k_face_count, grid_for(nf, 256), 256, 0, d_faces, nf, n, cnt, slots, h->d_status);
    scan_exclusive(h, cnt, off, n, tmp);
  }
  FP_CHECK_LAUNCH(h, "face count");
  // no host round trip here: every face contributes at most 6 raw entries,
  // faces with a corner out of range are skipped by both kernels and
  // reported at the sync that ends the build
  const int64_t nraw = 6 * nf;
  int32_t* raw = (int32_t*)dev_alloc(h, sizeof(int32_t) * (nraw > 0 ? nraw : 1));
  if (!raw) return fail(h, FP_ERR_OUT_OF_MEMORY, "raw adjacency");
  if (nf > 0) {
    ProfScope ps(FP_PROF_GRAPH, h->stream);
    FP_LAUNCH(h, k_face_fill, grid_for(nf, 256), 256, 0, d_faces, nf, n, off, slots, raw);
  }
  dev_free(h, slots);
  FP_TRY(finish_rows(h, off, raw, nraw, tmp, "face corner out of range"));
  dev_free(h, cnt);
  dev_free(h, off);
  dev_free(h, tmp);
  dev_free(h, raw);
  return FP_OK;
}

// A caller's row pointers must start at 0 and never decrease (checked before
// any kernel reads a column index through them).
__global__ void k_check_rowptr(const int32_t* __restrict__ rowptr, int32_t nrows, int32_t* status) {
  FP_PDL_WAIT();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += gridDim.x * blockDim.x)
    if ((i == 0 && rowptr[0] != 0) || rowptr[i] > rowptr[i + 1]) atomicOr(status, ST_BAD_ROWPTR);
}

fp_status build_graph_from_csr(fp_handle* h, const int32_t* d_rowptr, const int32_t* d_col, int32_t nrows) {
  const int32_t n = h->n, b = h->b;
  if (nrows > 0) {
    FP_LAUNCH(h, k_check_rowptr, grid_for(nrows, 256), 256, 0, d_rowptr, nrows, h->d_status);
    FP_CHECK_LAUNCH(h, "row pointer check");
    int32_t st0 = 0;
    FP_TRY(sync_status(h, &st0));
    if (st0 & ST_BAD_ROWPTR) return fail(h, FP_ERR_INVALID_ARG, "row pointers must start at 0 and not decrease");
    if (!d_col) {
      int32_t last = 0;
      cudaError_t e0 = cudaMemcpy(&last, d_rowptr + nrows, sizeof(int32_t), cudaMemcpyDeviceToHost);
      if (e0 != cudaSuccess) return check_cuda(h, e0, "row pointers");
      if (last != 0) return fail(h, FP_ERR_INVALID_ARG, "NULL column array with entries");
    }
  }
  int32_t* cnt = (int32_t*)dev_alloc(h, sizeof(int32_t) * (n + 1));
  int32_t* off = (int32_t*)dev_alloc(h, sizeof(int32_t) * (n + 1));
  int32_t* tmp = (int32_t*)dev_alloc(h, sizeof(int32_t) * scan_tmp_ints(n + 1));
  if (!cnt || !off || !tmp) return fail(h, FP_ERR_OUT_OF_MEMORY, "graph workspace");
  fill_i32(h, cnt, 0, n + 1);
  if (nrows > 0) FP_LAUNCH(h, k_pat_count, grid_for(nrows, 256), 256, 0, d_rowptr, d_col, nrows, b, cnt, h->d_status);
  scan_exclusive(h, cnt, off, n, tmp);
  FP_CHECK_LAUNCH(h, "pattern count");
  int32_t st = 0;
  FP_TRY(sync_status(h, &st));
  if (st & ST_BAD_INDEX) return fail(h, FP_ERR_INVALID_ARG, "column index out of range");
  int32_t nraw = 0;
  cudaError_t e = cudaMemcpy(&nraw, off + n, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return check_cuda(h, e, "read raw size");
  int32_t* raw = (int32_t*)dev_alloc(h, sizeof(int32_t) * (nraw > 0 ? nraw : 1));
  if (!raw) return fail(h, FP_ERR_OUT_OF_MEMORY, "raw adjacency");
  fill_i32(h, cnt, 0, n + 1);
  if (nrows > 0) FP_LAUNCH(h, k_pat_fill, grid_for(nrows, 256), 256, 0, d_rowptr, d_col, nrows, b, off, cnt, raw);
  FP_TRY(finish_rows(h, off, raw, nraw, tmp, "column index out of range"));
  if (n > 0) FP_LAUNCH(h, k_check_symmetric, grid_for((int64_t)n * 32, 256), 256, 0, h->rowptr, h->col, n, h->d_status);
  FP_CHECK_LAUNCH(h, "symmetry check");
  FP_TRY(sync_status(h, &st));
  if (st & ST_NOT_SYMMETRIC) return fail(h, FP_ERR_NOT_SYMMETRIC, "pattern is not structurally symmetric");
  dev_free(h, cnt);
  dev_free(h, off);
  dev_free(h, tmp);
  dev_free(h, raw);
  return FP_OK;
}

}  // namespace fp
