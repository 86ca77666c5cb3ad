// Numeric sparse Cholesky driven by the permutation and its nested-dissection
// tree (Section 6: the ordering exists to feed a direct solver; the paper
// hands perm and the elimination tree to cuDSS / MKL). Multifrontal, one dense
// front per tree node:
//   front(t) = the node's own columns (positions node_begin .. + m) followed by
//   U_t, the ancestor positions that some column of t's subtree reaches in L.
// Levels are processed bottom-up. A level's fronts are zeroed, receive the
// entries of P A P^T in their columns, then the children's update matrices
// (extend-add, child slot by child slot, so every sum has a fixed order); the
// first m columns are factored by a tiled right-looking partial Cholesky whose
// tiles of all the level's fronts run in the same launches; what remains in
// the trailing r x r block is the front's update matrix for its parent. The
// factor stays in the fronts (column-major, leading dimension m + r): L's
// columns of node t are the front's first m columns.
// FP64 throughout. With the sparse orders of meshes every front is small
// except near the root, so the work is spread as tiles, not as fronts.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fp_device.cuh"

namespace fp {

struct NumericFactor {
  int64_t nn = 0;
  std::vector<int32_t> begin, size, r;     // per node
  std::vector<int64_t> uoff, foff;         // per node: U list offset (ints), front offset (doubles)
  std::vector<char> active;                // node or a descendant holds a vertex
  std::vector<std::vector<int32_t>> level; // active nodes by depth
  int32_t* d_level_nodes = nullptr;        // all levels' node lists, concatenated
  std::vector<int64_t> level_at;           // offset of each depth's list in d_level_nodes
  int32_t* d_rows = nullptr;               // U lists (positions, ascending)
  int32_t* d_r = nullptr;
  int64_t* d_uoff = nullptr;
  int64_t* d_foff = nullptr;
  char* d_active = nullptr;
  double* d_front = nullptr;
  int64_t front_doubles = 0;
  int64_t dense_flops = 0;                 // flops of the partial factorisations (the fronts' work)
  int64_t nnz_front = 0;                   // entries of L as stored (lower trapezoids of the fronts)
  std::vector<void*> owned;                // device blocks, freed by numeric_release
};

namespace {

constexpr int NT = 256;        // threads of the front kernels
constexpr int NB = 64;         // tile edge

__device__ __forceinline__ int32_t lower_bound_i32(const int32_t* a, int32_t len, int32_t x) {
  int32_t lo = 0, hi = len;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Index of position p in the sorted list U (len entries), or -1 if absent
// (which the structure rules out; the callers flag it instead of writing
// outside the front).
__device__ __forceinline__ int32_t find_row(const int32_t* U, int32_t len, int32_t p) {
  const int32_t i = lower_bound_i32(U, len, p);
  return (i < len && U[i] == p) ? i : -1;
}

// ---- U lists ------------------------------------------------------------------------------

struct RowsArgs {
  const int32_t* nodes;
  const int32_t* node_begin;
  const int32_t* node_size;
  const int32_t* perm;
  const int32_t* iperm;
  const int32_t* rowptr;
  const int32_t* col;
  const int64_t* uoff;
  int32_t* r;
  int32_t* rows;
  const char* active;
  int64_t nn;
};

// U_t for every node of one depth: the proper-ancestor positions met by the
// matrix entries of t's columns and by the children's U lists, marked in a
// bitmap over the ancestors' columns (parent first, so bit order is position
// order) and listed in ascending position.
__global__ void __launch_bounds__(NT) k_front_rows(RowsArgs a) {
  FP_PDL_WAIT();
  extern __shared__ uint32_t bm[];
  __shared__ int32_t s_ab[32], s_as[32], s_off[33];
  __shared__ int32_t s_na;
  __shared__ int32_t red[40];
  const int32_t t = a.nodes[blockIdx.x];
  if (threadIdx.x == 0) {
    int32_t na = 0;
    for (int64_t x = t; x > 0 && na < 32;) {
      x = (x - 1) / 2;
      s_ab[na] = a.node_begin[x];
      s_as[na] = a.node_size[x];
      ++na;
    }
    s_off[0] = 0;
    for (int32_t l = 0; l < na; ++l) s_off[l + 1] = s_off[l] + s_as[l];
    s_na = na;
  }
  __syncthreads();
  const int32_t na = s_na, nbits = s_off[na], words = (nbits + 31) >> 5;
  for (int32_t w = threadIdx.x; w < words; w += NT) bm[w] = 0u;
  __syncthreads();
  auto mark = [&](int32_t p) {
    for (int32_t l = 0; l < na; ++l) {
      const int32_t q = p - s_ab[l];
      if (q >= 0 && q < s_as[l]) {
        const int32_t bit = s_off[l] + q;
        atomicOr(&bm[bit >> 5], 1u << (bit & 31));
        return;
      }
    }
  };
  const int32_t b = a.node_begin[t], m = a.node_size[t];
  for (int32_t j = b + threadIdx.x; j < b + m; j += NT) {
    const int32_t v = a.perm[j];
    for (int32_t e = a.rowptr[v]; e < a.rowptr[v + 1]; ++e) mark(a.iperm[a.col[e]]);
  }
  for (int32_t s = 0; s < 2; ++s) {
    const int64_t c = 2 * (int64_t)t + 1 + s;
    if (c >= a.nn || !a.active[c]) continue;
    const int32_t* uc = a.rows + a.uoff[c];
    const int32_t rc = a.r[c];
    for (int32_t i = threadIdx.x; i < rc; i += NT) mark(uc[i]);
  }
  __syncthreads();
  int32_t* out = a.rows + a.uoff[t];
  int32_t carry = 0;
  for (int32_t w0 = 0; w0 < words; w0 += NT) {
    const int32_t w = w0 + threadIdx.x;
    const uint32_t x0 = w < words ? bm[w] : 0u;
    int32_t tot;
    int32_t o = block_excl_scan_i32(__popc(x0), &tot, red) + carry;
    uint32_t x = x0;
    while (x) {
      const int32_t bit = w * 32 + __ffs(x) - 1;
      x &= x - 1;
      int32_t l = 0;
      while (bit >= s_off[l + 1]) ++l;
      out[o++] = s_ab[l] + (bit - s_off[l]);
    }
    carry += tot;
  }
  if (threadIdx.x == 0) a.r[t] = carry;
}

// ---- assembly --------------------------------------------------------------------------------

struct FrontArgs {
  const int32_t* nodes;
  const int32_t* node_begin;
  const int32_t* node_size;
  const int32_t* r;
  const int64_t* uoff;
  const int32_t* rows;
  const int64_t* foff;
  double* front;
  const char* active;
  int64_t nn;
  const int32_t* perm;
  const int32_t* iperm;
  const int32_t* rowptr;
  const int32_t* col;
  const double* diag;      // by vertex
  const double* off;       // aligned with (rowptr, col)
  int32_t* status;
};

// Entries of P A P^T in the node's columns, on and below the diagonal.
__global__ void __launch_bounds__(NT) k_front_scatter(FrontArgs a) {
  FP_PDL_WAIT();
  const int32_t t = a.nodes[blockIdx.x];
  const int32_t b = a.node_begin[t], m = a.node_size[t], r = a.r[t];
  const int64_t f = (int64_t)m + r;
  double* F = a.front + a.foff[t];
  const int32_t* U = a.rows + a.uoff[t];
  for (int32_t j = b + threadIdx.x; j < b + m; j += NT) {
    const int32_t c = j - b, v = a.perm[j];
    F[c + c * f] = a.diag[v];
    for (int32_t e = a.rowptr[v]; e < a.rowptr[v + 1]; ++e) {
      const int32_t p = a.iperm[a.col[e]];
      if (p <= j) continue;
      const int32_t u = p < b + m ? p - b : find_row(U, r, p);
      if (u < 0) { atomicOr(a.status, ST_BAD_INDEX); continue; }
      F[(p < b + m ? u : m + u) + c * f] = a.off[e];
    }
  }
}

// Extend-add of one child slot's update matrix into the parents' fronts:
// F_t[map(i), map(k)] += U_c[i, k] for i >= k; blockIdx.y strides the
// child's columns.
__global__ void __launch_bounds__(NT) k_front_extend(FrontArgs a, int32_t slot) {
  FP_PDL_WAIT();
  extern __shared__ int32_t map[];
  const int32_t t = a.nodes[blockIdx.x];
  const int64_t c = 2 * (int64_t)t + 1 + slot;
  if (c >= a.nn || !a.active[c]) return;
  const int32_t rc = a.r[c];
  if (rc == 0) return;
  const int32_t b = a.node_begin[t], m = a.node_size[t], r = a.r[t];
  const int32_t* Ut = a.rows + a.uoff[t];
  const int32_t* Uc = a.rows + a.uoff[c];
  for (int32_t i = threadIdx.x; i < rc; i += NT) {
    const int32_t p = Uc[i];
    int32_t u = (p >= b && p < b + m) ? p - b : find_row(Ut, r, p);
    if (u < 0) atomicOr(a.status, ST_BAD_INDEX);
    else if (!(p >= b && p < b + m)) u += m;
    map[i] = u;
  }
  __syncthreads();
  const int32_t mc = a.node_size[c];
  const int64_t fc = (int64_t)mc + rc, ft = (int64_t)m + r;
  const double* Fc = a.front + a.foff[c] + mc + mc * fc;
  double* Ft = a.front + a.foff[t];
  for (int32_t k = blockIdx.y; k < rc; k += gridDim.y) {
    const double* src = Fc + k * fc;
    double* dst = Ft + (int64_t)(map[k] < 0 ? 0 : map[k]) * ft;
    if (map[k] < 0) continue;
    for (int32_t i = k + threadIdx.x; i < rc; i += NT)
      if (map[i] >= 0) dst[map[i]] += src[i];
  }
}

// ---- tiled partial Cholesky ------------------------------------------------------------------

struct TileArgs {
  const int32_t* nodes;
  int32_t count;
  const int32_t* node_size;
  const int32_t* r;
  const int64_t* foff;
  double* front;
  const int64_t* pre;      // [count + 1] tile-item prefix over the level's nodes (panel / update)
  int32_t k0;              // first column of this step's panel
  int32_t* status;
};

// Diagonal tile of every front with columns left: Cholesky in shared memory,
// written back.
__global__ void __launch_bounds__(NT) k_tile_potrf(TileArgs a) {
  FP_PDL_WAIT();
  __shared__ double A[NB][NB + 1];
  __shared__ double s_piv;
  const int32_t t = a.nodes[blockIdx.x];
  const int32_t m = a.node_size[t];
  if (a.k0 >= m) return;
  const int32_t nb = min(NB, m - a.k0);
  const int64_t f = (int64_t)m + a.r[t];
  double* F = a.front + a.foff[t] + a.k0 + a.k0 * f;
  for (int32_t x = threadIdx.x; x < nb * nb; x += NT) {
    const int32_t i = x % nb, j = x / nb;
    A[i][j] = i >= j ? F[i + j * f] : 0.0;
  }
  __syncthreads();
  for (int32_t k = 0; k < nb; ++k) {
    if (threadIdx.x == 0) {
      double d = A[k][k];
      if (!(d > 0.0)) {
        atomicOr(a.status, ST_NOT_SPD);
        d = 1.0;
      }
      d = sqrt(d);
      A[k][k] = d;
      s_piv = 1.0 / d;
    }
    __syncthreads();
    const double ip = s_piv;
    for (int32_t i = k + 1 + threadIdx.x; i < nb; i += NT) A[i][k] *= ip;
    __syncthreads();
    const int32_t w = nb - k - 1;
    for (int32_t x = threadIdx.x; x < w * w; x += NT) {
      const int32_t i = k + 1 + x % w, j = k + 1 + x / w;
      if (i >= j) A[i][j] -= A[i][k] * A[j][k];
    }
    __syncthreads();
  }
  for (int32_t x = threadIdx.x; x < nb * nb; x += NT) {
    const int32_t i = x % nb, j = x / nb;
    if (i >= j) F[i + j * f] = A[i][j];
  }
}

__device__ __forceinline__ int32_t item_owner(const int64_t* pre, int32_t count, int64_t b) {
  int32_t lo = 0, hi = count;            // last i with pre[i] <= b
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) >> 1;
    if (pre[mid] <= b) lo = mid; else hi = mid;
  }
  return lo;
}

// Panel below the diagonal tile: X L_kk^T = F[rows, k0:k0+nb], solved by
// substitution along the columns, one row a thread and PR rows a CTA. (A
// product with the tile's inverse would leave rounding residue where L is
// structurally zero; substitution keeps those entries exactly 0.)
constexpr int PR = NT;
__global__ void __launch_bounds__(NT) k_tile_panel(TileArgs a) {
  FP_PDL_WAIT();
  extern __shared__ double psm[];
  double (*P)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(psm);           // [PR][NB+1]
  double (*Lk)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(psm + PR * (NB + 1));
  const int32_t i = item_owner(a.pre, a.count, blockIdx.x);
  const int32_t t = a.nodes[i];
  const int32_t m = a.node_size[t];
  const int32_t nb = min(NB, m - a.k0);
  const int64_t f = (int64_t)m + a.r[t];
  const int64_t row0 = a.k0 + nb + (int64_t)(blockIdx.x - a.pre[i]) * PR;
  const int32_t nr = (int32_t)min((int64_t)PR, f - row0);
  double* F = a.front + a.foff[t];
  for (int32_t x = threadIdx.x; x < nb * nb; x += NT) {
    const int32_t rr = x % nb, q = x / nb;
    Lk[rr][q] = rr >= q ? F[a.k0 + rr + (a.k0 + q) * f] : 0.0;
  }
  for (int32_t q = 0; q < nb; ++q)
    for (int32_t rr = threadIdx.x; rr < PR; rr += NT) P[rr][q] = rr < nr ? F[row0 + rr + (a.k0 + q) * f] : 0.0;
  __syncthreads();
  const int32_t rr = threadIdx.x;
  if (rr < nr) {
    for (int32_t c = 0; c < nb; ++c) {
      double s = P[rr][c];
      for (int32_t q = 0; q < c; ++q) s -= P[rr][q] * Lk[c][q];
      P[rr][c] = s / Lk[c][c];
    }
  }
  __syncthreads();
  for (int32_t q = 0; q < nb; ++q)
    for (int32_t x = threadIdx.x; x < nr; x += NT) F[row0 + x + (a.k0 + q) * f] = P[x][q];
}

// Trailing update: F[I, J] -= X_I X_J^T for 64 x 64 tile pairs I >= J below
// the panel (the diagonal tiles are computed whole; their upper halves are
// never read).
__global__ void __launch_bounds__(NT) k_tile_update(TileArgs a) {
  FP_PDL_WAIT();
  __shared__ double XI[NB][NB + 1];
  __shared__ double XJ[NB][NB + 1];
  const int32_t i = item_owner(a.pre, a.count, blockIdx.x);
  const int32_t t = a.nodes[i];
  const int32_t m = a.node_size[t];
  const int32_t nb = min(NB, m - a.k0);
  const int64_t f = (int64_t)m + a.r[t];
  const int64_t li = blockIdx.x - a.pre[i];
  int64_t I = (int64_t)((sqrt(8.0 * (double)li + 1.0) - 1.0) / 2.0);
  while (I * (I + 1) / 2 > li) --I;
  while ((I + 1) * (I + 2) / 2 <= li) ++I;
  const int64_t J = li - I * (I + 1) / 2;
  const int64_t base = a.k0 + nb;
  const int64_t ri = base + I * NB, rj = base + J * NB;
  const int32_t ni = (int32_t)min((int64_t)NB, f - ri), nj = (int32_t)min((int64_t)NB, f - rj);
  double* F = a.front + a.foff[t];
  for (int32_t x = threadIdx.x; x < NB * NB; x += NT) {
    const int32_t rr = x % NB, q = x / NB;
    const double* col = F + (a.k0 + q) * f;
    XI[rr][q] = (rr < ni && q < nb) ? col[ri + rr] : 0.0;
    XJ[rr][q] = (rr < nj && q < nb) ? col[rj + rr] : 0.0;
  }
  __syncthreads();
  const int32_t r0 = (threadIdx.x & 15) * 4, c0 = (threadIdx.x >> 4) * 4;
  double acc[4][4];
#pragma unroll
  for (int32_t x = 0; x < 4; ++x)
#pragma unroll
    for (int32_t y = 0; y < 4; ++y) acc[x][y] = 0.0;
  for (int32_t q = 0; q < nb; ++q) {
    double u[4], w[4];
#pragma unroll
    for (int32_t x = 0; x < 4; ++x) { u[x] = XI[r0 + x][q]; w[x] = XJ[c0 + x][q]; }
#pragma unroll
    for (int32_t x = 0; x < 4; ++x)
#pragma unroll
      for (int32_t y = 0; y < 4; ++y) acc[x][y] += u[x] * w[y];
  }
#pragma unroll
  for (int32_t y = 0; y < 4; ++y) {
    if (c0 + y >= nj) continue;
    double* col = F + (rj + c0 + y) * f + ri;
#pragma unroll
    for (int32_t x = 0; x < 4; ++x)
      if (r0 + x < ni) col[r0 + x] -= acc[x][y];
  }
}

// ---- solve ------------------------------------------------------------------------------------

struct SolveArgs {
  const int32_t* nodes;
  const int32_t* node_begin;
  const int32_t* node_size;
  const int32_t* r;
  const int64_t* uoff;
  const int32_t* rows;
  const int64_t* foff;
  const double* front;
  const char* active;
  int64_t nn;
  double* y;               // [n] by position
  double* w;               // [sum r] update vectors, at uoff
};

__global__ void k_gather_perm(const double* __restrict__ b, const int32_t* __restrict__ perm, int32_t n,
                              double* __restrict__ y) {
  FP_PDL_WAIT();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = b[perm[i]];
}

__global__ void k_scatter_perm(const double* __restrict__ y, const int32_t* __restrict__ perm, int32_t n,
                               double* __restrict__ x) {
  FP_PDL_WAIT();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[perm[i]] = y[i];
}

// Forward substitution of one depth (L x = b, deepest nodes first): the
// children's update vectors are subtracted from this node's entries or passed
// on to its own update vector, the node's diagonal block is solved, and
// L[U_t, t] x_t joins the update vector.
__global__ void __launch_bounds__(NT) k_solve_forward(SolveArgs a) {
  FP_PDL_WAIT();
  const int32_t t = a.nodes[blockIdx.x];
  const int32_t b = a.node_begin[t], m = a.node_size[t], r = a.r[t];
  const int64_t f = (int64_t)m + r;
  const int32_t* Ut = a.rows + a.uoff[t];
  double* wt = a.w + a.uoff[t];
  double* y = a.y + b;
  const double* F = a.front + a.foff[t];
  for (int32_t i = threadIdx.x; i < r; i += NT) wt[i] = 0.0;
  __syncthreads();
  for (int32_t s = 0; s < 2; ++s) {
    const int64_t c = 2 * (int64_t)t + 1 + s;
    if (c >= a.nn || !a.active[c]) continue;
    const int32_t rc = a.r[c];
    const int32_t* Uc = a.rows + a.uoff[c];
    const double* wc = a.w + a.uoff[c];
    for (int32_t i = threadIdx.x; i < rc; i += NT) {
      const int32_t p = Uc[i];
      if (p >= b && p < b + m) {
        y[p - b] -= wc[i];
      } else {
        const int32_t u = find_row(Ut, r, p);
        if (u >= 0) wt[u] += wc[i];
      }
    }
    __syncthreads();
  }
  // blocks of 64 columns: warp 0 solves the diagonal block (lanes own rows
  // k0 + lane and k0 + 32 + lane, the solved entry passed by shuffle), then
  // every thread subtracts the block's contribution from one row below it
  const int32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int32_t k0 = 0; k0 < m; k0 += 64) {
    const int32_t nb = min(64, m - k0);
    if (warp == 0) {
      double y0 = lane < nb ? y[k0 + lane] : 0.0, y1 = 32 + lane < nb ? y[k0 + 32 + lane] : 0.0;
      for (int32_t k = 0; k < nb; ++k) {
        const double* colk = F + (int64_t)(k0 + k) * f + k0;
        const double yk = __shfl_sync(0xffffffffu, k < 32 ? y0 : y1, k & 31);
        const double xk = yk / colk[k];
        if (lane == (k & 31)) { if (k < 32) y0 = xk; else y1 = xk; }
        if (lane > k && lane < nb) y0 -= colk[lane] * xk;
        if (32 + lane > k && 32 + lane < nb) y1 -= colk[32 + lane] * xk;
      }
      if (lane < nb) y[k0 + lane] = y0;
      if (32 + lane < nb) y[k0 + 32 + lane] = y1;
    }
    __syncthreads();
    for (int32_t i = k0 + nb + threadIdx.x; i < m; i += NT) {
      double s = 0.0;
      for (int32_t k = 0; k < nb; ++k) s += F[i + (int64_t)(k0 + k) * f] * y[k0 + k];
      y[i] -= s;
    }
    __syncthreads();
  }
  for (int32_t i = threadIdx.x; i < r; i += NT) {
    double s = 0.0;
    for (int32_t k = 0; k < m; ++k) s += F[m + i + k * f] * y[k];
    wt[i] += s;
  }
}

// Back substitution of one depth (L^T x = y, root first): the ancestors'
// entries are final, so each node subtracts L[U_t, t]^T x[U_t] and solves its
// transposed diagonal block.
__global__ void __launch_bounds__(NT) k_solve_backward(SolveArgs a) {
  FP_PDL_WAIT();
  const int32_t t = a.nodes[blockIdx.x];
  const int32_t b = a.node_begin[t], m = a.node_size[t], r = a.r[t];
  const int64_t f = (int64_t)m + r;
  const int32_t* Ut = a.rows + a.uoff[t];
  double* y = a.y + b;
  const double* F = a.front + a.foff[t];
  for (int32_t k = threadIdx.x; k < m; k += NT) {
    double s = 0.0;
    const double* colk = F + k * f + m;
    for (int32_t i = 0; i < r; ++i) s += colk[i] * a.y[Ut[i]];
    y[k] -= s;
  }
  __syncthreads();
  // blocks of 64 columns from the last: warp 0 solves the transposed
  // diagonal block, then every thread subtracts the block's contribution
  // from one entry above it
  const int32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int32_t k1 = m; k1 > 0; k1 -= 64) {
    const int32_t k0 = k1 > 64 ? k1 - 64 : 0, nb = k1 - k0;
    if (warp == 0) {
      double y0 = lane < nb ? y[k0 + lane] : 0.0, y1 = 32 + lane < nb ? y[k0 + 32 + lane] : 0.0;
      for (int32_t k = nb - 1; k >= 0; --k) {
        // row k of the block: L[k0 + k][k0 + i] = F[(k0 + k) + (k0 + i) f]
        const double yk = __shfl_sync(0xffffffffu, k < 32 ? y0 : y1, k & 31);
        const double xk = yk / F[(k0 + k) + (int64_t)(k0 + k) * f];
        if (lane == (k & 31)) { if (k < 32) y0 = xk; else y1 = xk; }
        if (lane < k) y0 -= F[(k0 + k) + (int64_t)(k0 + lane) * f] * xk;
        if (32 + lane < k) y1 -= F[(k0 + k) + (int64_t)(k0 + 32 + lane) * f] * xk;
      }
      if (lane < nb) y[k0 + lane] = y0;
      if (32 + lane < nb) y[k0 + 32 + lane] = y1;
    }
    __syncthreads();
    for (int32_t i = threadIdx.x; i < k0; i += NT) {
      const double* coli = F + (int64_t)i * f + k0;
      double s = 0.0;
      for (int32_t k = 0; k < nb; ++k) s += coli[k] * y[k0 + k];
      y[i] -= s;
    }
    __syncthreads();
  }
}

// L in compressed columns: column j of node t holds the rows j .. end of the
// node's block (dense; exact zeros where L is structurally zero) and U_t.
__global__ void k_front_export(SolveArgs a, const int64_t* __restrict__ colptr, int32_t* __restrict__ ri,
                               double* __restrict__ rx) {
  FP_PDL_WAIT();
  const int32_t t = a.nodes[blockIdx.x];
  const int32_t b = a.node_begin[t], m = a.node_size[t], r = a.r[t];
  const int64_t f = (int64_t)m + r;
  const int32_t* Ut = a.rows + a.uoff[t];
  const double* F = a.front + a.foff[t];
  for (int32_t c = 0; c < m; ++c) {
    const int64_t o = colptr[b + c];
    const double* colc = F + c * f;
    for (int32_t i = c + threadIdx.x; i < m + r; i += blockDim.x) {
      ri[o + i - c] = i < m ? b + i : Ut[i - m];
      rx[o + i - c] = colc[i];
    }
  }
}

}  // namespace

void numeric_release(fp_handle* h) {
  if (!h->numeric) return;
  for (void* p : h->numeric->owned) dev_free(h, p);
  delete h->numeric;
  h->numeric = nullptr;
}

namespace {

int depth_of(int64_t t) {
  int d = 0;
  while (((int64_t)1 << (d + 1)) - 1 <= t) ++d;
  return d;
}

template <class T>
T* nalloc(fp_handle* h, NumericFactor* F, int64_t count) {
  T* p = (T*)dev_alloc(h, sizeof(T) * (size_t)(count > 0 ? count : 1));
  if (p) F->owned.push_back(p);
  return p;
}

}  // namespace

fp_status run_factor(fp_handle* h, const double* d_diag, const double* d_off) {
  numeric_release(h);
  const int64_t nn = h->nnodes;
  const int32_t n = h->n, D = h->D;
  NumericFactor* F = new NumericFactor();
  h->numeric = F;
  F->nn = nn;
  F->size = h->node_size_host;
  F->begin.resize(nn);
  cudaError_t e = cudaMemcpyAsync(F->begin.data(), h->node_begin, sizeof(int32_t) * nn, cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "node layout");
  // active nodes (a vertex in the subtree), ancestor column totals
  F->active.assign(nn, 0);
  for (int64_t t = nn - 1; t >= 0; --t) {
    bool act = F->size[t] > 0;
    for (int64_t c = 2 * t + 1; c <= 2 * t + 2; ++c)
      if (c < nn && F->active[c]) act = true;
    F->active[t] = act;
  }
  std::vector<int64_t> anc(nn, 0);
  for (int64_t t = 1; t < nn; ++t) anc[t] = anc[(t - 1) / 2] + F->size[(t - 1) / 2];
  F->level.assign(D + 1, {});
  F->uoff.assign(nn, 0);
  int64_t utot = 0;
  for (int64_t t = 0; t < nn; ++t) {
    if (!F->active[t]) continue;
    F->level[depth_of(t)].push_back((int32_t)t);
    F->uoff[t] = utot;
    utot += anc[t];
  }
  std::vector<int32_t> all;
  F->level_at.assign(D + 2, 0);
  for (int d = 0; d <= D; ++d) {
    F->level_at[d] = (int64_t)all.size();
    all.insert(all.end(), F->level[d].begin(), F->level[d].end());
  }
  F->level_at[D + 1] = (int64_t)all.size();
  F->d_level_nodes = nalloc<int32_t>(h, F, (int64_t)all.size());
  F->d_rows = nalloc<int32_t>(h, F, utot);
  F->d_r = nalloc<int32_t>(h, F, nn);
  F->d_uoff = nalloc<int64_t>(h, F, nn);
  F->d_foff = nalloc<int64_t>(h, F, nn);
  F->d_active = nalloc<char>(h, F, nn);
  if (!F->d_level_nodes || !F->d_rows || !F->d_r || !F->d_uoff || !F->d_foff || !F->d_active)
    return fail(h, FP_ERR_OUT_OF_MEMORY, "factor structure");
  cudaMemcpyAsync(F->d_level_nodes, all.data(), sizeof(int32_t) * all.size(), cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(F->d_uoff, F->uoff.data(), sizeof(int64_t) * nn, cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(F->d_active, F->active.data(), (size_t)nn, cudaMemcpyHostToDevice, h->stream);
  cudaMemsetAsync(F->d_r, 0, sizeof(int32_t) * nn, h->stream);
  // 1. U lists, deepest level first
  allow_max_dynamic_smem(k_front_rows);
  for (int d = D; d >= 0; --d) {
    const auto& L = F->level[d];
    if (L.empty()) continue;
    int64_t words = 0;
    for (int32_t t : L) words = std::max<int64_t>(words, (anc[t] + 31) / 32);
    if (words * 4 > 200 * 1024) return fail(h, FP_ERR_UNSUPPORTED, "a tree node with more than 1.6M ancestor columns");
    RowsArgs ra{F->d_level_nodes + F->level_at[d], h->node_begin, h->node_size, h->perm, h->iperm, h->rowptr, h->col,
                F->d_uoff, F->d_r, F->d_rows, F->d_active, nn};
    FP_LAUNCH(h, k_front_rows, (int)L.size(), NT, (size_t)(words > 0 ? words : 1) * 4, ra);
  }
  FP_CHECK_LAUNCH(h, "front rows");
  F->r.assign(nn, 0);
  e = cudaMemcpyAsync(F->r.data(), F->d_r, sizeof(int32_t) * nn, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "front sizes");
  // 2. fronts, deepest level first so that a level's fronts are contiguous
  F->foff.assign(nn, 0);
  int64_t ftot = 0;
  std::vector<int64_t> lvl_lo(D + 1), lvl_hi(D + 1);
  int64_t max_rc = 1;
  for (int d = D; d >= 0; --d) {
    lvl_lo[d] = ftot;
    for (int32_t t : F->level[d]) {
      const int64_t fsz = (int64_t)F->size[t] + F->r[t];
      F->foff[t] = ftot;
      ftot += fsz * fsz;
      max_rc = std::max<int64_t>(max_rc, F->r[t]);
      const int64_t m = F->size[t], r = F->r[t];
      // a pivot with x rows left costs about x^2 flops (the lower half of its
      // rank-1 update, a multiply and an add each): sum over x = r+1 .. f
      F->dense_flops += (fsz * fsz * fsz - r * r * r) / 3;
      F->nnz_front += m * (m + 1) / 2 + m * r;
    }
    lvl_hi[d] = ftot;
  }
  if (max_rc * 4 > 200 * 1024) return fail(h, FP_ERR_UNSUPPORTED, "an update matrix above 51,200 rows");
  F->front_doubles = ftot;
  F->d_front = nalloc<double>(h, F, ftot);
  if (!F->d_front) return fail(h, FP_ERR_OUT_OF_MEMORY, "fronts");
  cudaMemcpyAsync(F->d_foff, F->foff.data(), sizeof(int64_t) * nn, cudaMemcpyHostToDevice, h->stream);
  // item prefix arrays of every (level, step): panel tiles and update tiles per node
  std::vector<int64_t> pre;
  struct Step { int d, s; int64_t panel_at, update_at, panel_items, update_items; };
  std::vector<Step> steps;
  for (int d = D; d >= 0; --d) {
    const auto& L = F->level[d];
    int32_t mmax = 0;
    for (int32_t t : L) mmax = std::max(mmax, F->size[t]);
    for (int s = 0; s * NB < mmax; ++s) {
      Step st{d, s, (int64_t)pre.size(), 0, 0, 0};
      int64_t acc = 0;
      for (int32_t t : L) {
        pre.push_back(acc);
        const int64_t m = F->size[t], f = m + F->r[t], k0 = (int64_t)s * NB;
        if (k0 < m) acc += (f - k0 - std::min<int64_t>(NB, m - k0) + PR - 1) / PR;
      }
      pre.push_back(acc);
      st.panel_items = acc;
      st.update_at = (int64_t)pre.size();
      acc = 0;
      for (int32_t t : L) {
        pre.push_back(acc);
        const int64_t m = F->size[t], f = m + F->r[t], k0 = (int64_t)s * NB;
        if (k0 < m) {
          const int64_t rt = (f - k0 - std::min<int64_t>(NB, m - k0) + NB - 1) / NB;
          acc += rt * (rt + 1) / 2;
        }
      }
      pre.push_back(acc);
      st.update_items = acc;
      steps.push_back(st);
    }
  }
  int64_t* d_pre = nalloc<int64_t>(h, F, (int64_t)pre.size());
  if (!d_pre) return fail(h, FP_ERR_OUT_OF_MEMORY, "factor schedule");
  cudaMemcpyAsync(d_pre, pre.data(), sizeof(int64_t) * pre.size(), cudaMemcpyHostToDevice, h->stream);
  // 3. numeric, deepest level first
  allow_max_dynamic_smem(k_front_extend);
  allow_max_dynamic_smem(k_tile_panel);
  size_t si = 0;
  for (int d = D; d >= 0; --d) {
    const auto& L = F->level[d];
    if (L.empty()) continue;
    ProfScope ps(FP_PROF_NUMERIC, h->stream);
    const int32_t* nodes = F->d_level_nodes + F->level_at[d];
    cudaMemsetAsync(F->d_front + lvl_lo[d], 0, sizeof(double) * (size_t)(lvl_hi[d] - lvl_lo[d]), h->stream);
    FrontArgs fa{nodes, h->node_begin, h->node_size, F->d_r, F->d_uoff, F->d_rows, F->d_foff, F->d_front,
                 F->d_active, nn, h->perm, h->iperm, h->rowptr, h->col, d_diag, d_off, h->d_status};
    FP_LAUNCH(h, k_front_scatter, (int)L.size(), NT, 0, fa);
    if (d < D) {
      int64_t rcmax = 1;
      for (int32_t t : L)
        for (int64_t c = 2 * (int64_t)t + 1; c <= 2 * (int64_t)t + 2; ++c)
          if (c < nn && F->active[c]) rcmax = std::max<int64_t>(rcmax, F->r[c]);
      const int gy = (int)std::min<int64_t>(64, std::max<int64_t>(1, rcmax / 64));
      for (int32_t slot = 0; slot < 2; ++slot)
        FP_LAUNCH(h, k_front_extend, dim3((unsigned)L.size(), (unsigned)gy), NT, (size_t)rcmax * 4, fa, slot);
    }
    for (; si < steps.size() && steps[si].d == d; ++si) {
      const Step& st = steps[si];
      TileArgs ta{nodes, (int32_t)L.size(), h->node_size, F->d_r, F->d_foff, F->d_front, nullptr, st.s * NB,
                  h->d_status};
      FP_LAUNCH(h, k_tile_potrf, (int)L.size(), NT, 0, ta);
      if (st.panel_items > 0) {
        ta.pre = d_pre + st.panel_at;
        FP_LAUNCH(h, k_tile_panel, (unsigned)st.panel_items, NT, sizeof(double) * (PR + NB) * (NB + 1), ta);
      }
      if (st.update_items > 0) {
        ta.pre = d_pre + st.update_at;
        FP_LAUNCH(h, k_tile_update, (unsigned)st.update_items, NT, 0, ta);
      }
    }
    FP_CHECK_LAUNCH(h, "numeric level");
  }
  int32_t st = 0;
  FP_TRY(sync_status(h, &st));
  if (st & ST_BAD_INDEX) {
    cudaMemsetAsync(h->d_status, 0, sizeof(int32_t), h->stream);
    numeric_release(h);
    return fail(h, FP_ERR_CUDA, "factor structure: a matrix entry outside its front");
  }
  if (st & ST_NOT_SPD) {
    cudaMemsetAsync(h->d_status, 0, sizeof(int32_t), h->stream);
    numeric_release(h);
    return fail(h, FP_ERR_INVALID_ARG, "matrix not positive definite (a pivot was not positive)");
  }
  (void)n;
  return FP_OK;
}

fp_status run_solve(fp_handle* h, const double* d_b, double* d_x) {
  NumericFactor* F = h->numeric;
  const int32_t n = h->n, D = h->D;
  double* y = (double*)dev_alloc(h, sizeof(double) * (size_t)(n > 0 ? n : 1));
  int64_t utot = 0;
  for (int64_t t = 0; t < F->nn; ++t)
    if (F->active[t]) utot = std::max<int64_t>(utot, F->uoff[t] + F->r[t]);
  double* w = (double*)dev_alloc(h, sizeof(double) * (size_t)(utot > 0 ? utot : 1));
  if (!y || !w) return fail(h, FP_ERR_OUT_OF_MEMORY, "solve workspace");
  const int G = grid_for(n, 256);
  ProfScope ps(FP_PROF_NUMERIC, h->stream);
  FP_LAUNCH(h, k_gather_perm, G, 256, 0, d_b, h->perm, n, y);
  SolveArgs sa{nullptr, h->node_begin, h->node_size, F->d_r, F->d_uoff, F->d_rows, F->d_foff, F->d_front, F->d_active,
               F->nn, y, w};
  for (int d = D; d >= 0; --d) {
    if (F->level[d].empty()) continue;
    sa.nodes = F->d_level_nodes + F->level_at[d];
    FP_LAUNCH(h, k_solve_forward, (int)F->level[d].size(), NT, 0, sa);
  }
  for (int d = 0; d <= D; ++d) {
    if (F->level[d].empty()) continue;
    sa.nodes = F->d_level_nodes + F->level_at[d];
    FP_LAUNCH(h, k_solve_backward, (int)F->level[d].size(), NT, 0, sa);
  }
  FP_LAUNCH(h, k_scatter_perm, G, 256, 0, y, h->perm, n, d_x);
  FP_CHECK_LAUNCH(h, "solve");
  dev_free(h, y);
  dev_free(h, w);
  return FP_OK;
}

fp_status run_factor_export(fp_handle* h, int64_t* d_colptr, int32_t* d_rows, double* d_vals, int64_t cap,
                            int64_t* h_nnz) {
  NumericFactor* F = h->numeric;
  const int32_t n = h->n;
  std::vector<int64_t> cp((size_t)n + 1, 0);
  for (int64_t t = 0; t < F->nn; ++t) {
    const int32_t m = F->size[t];
    for (int32_t c = 0; c < m; ++c) cp[(size_t)F->begin[t] + c + 1] = (int64_t)(m - c) + F->r[t];
  }
  for (int32_t j = 0; j < n; ++j) cp[j + 1] += cp[j];
  if (h_nnz) *h_nnz = cp[n];
  if (!d_colptr && !d_rows && !d_vals) return FP_OK;
  if (!d_colptr || !d_rows || !d_vals) return fail(h, FP_ERR_INVALID_ARG, "factor export: NULL buffer");
  if (cap < cp[n]) return fail(h, FP_ERR_INVALID_ARG, "factor export: buffer too small");
  cudaError_t e = cudaMemcpyAsync(d_colptr, cp.data(), sizeof(int64_t) * cp.size(), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);      // cp is a host temporary
  if (e != cudaSuccess) return check_cuda(h, e, "factor export");
  SolveArgs sa{nullptr, h->node_begin, h->node_size, F->d_r, F->d_uoff, F->d_rows, F->d_foff, F->d_front, F->d_active,
               F->nn, nullptr, nullptr};
  for (int d = 0; d <= h->D; ++d) {
    if (F->level[d].empty()) continue;
    sa.nodes = F->d_level_nodes + F->level_at[d];
    FP_LAUNCH(h, k_front_export, (int)F->level[d].size(), NT, 0, sa, d_colptr, d_rows, d_vals);
  }
  FP_CHECK_LAUNCH(h, "factor export");
  return FP_OK;
}

void numeric_stats(const fp_handle* h, int64_t* front_doubles, int64_t* flops, int64_t* nnz) {
  const NumericFactor* F = h->numeric;
  if (front_doubles) *front_doubles = F ? F->front_doubles : 0;
  if (flops) *flops = F ? F->dense_flops : 0;
  if (nnz) *nnz = F ? F->nnz_front : 0;
}

}  // namespace fp
