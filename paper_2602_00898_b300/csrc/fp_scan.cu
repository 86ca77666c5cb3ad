// Device-wide exclusive scan and fills: three launches (tile sums, scan of the
// tile sums by one CTA, tile-local scan plus offset; 1024 items per tile), or
// one CTA for arrays of up to 16k items.
#include "fp_internal.cuh"

namespace fp {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int32_t warp_incl_scan(int32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive scan of one value per thread across the CTA; returns the CTA total
// through *total. blockDim.x must be a multiple of 32 and <= 1024.
__device__ __forceinline__ int32_t block_excl_scan(int32_t x, int32_t* total) {
  __shared__ int32_t warp_sums[32];
  __shared__ int32_t block_total;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int32_t inc = warp_incl_scan(x);
  if (lane == 31) warp_sums[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int32_t s = lane < nw ? warp_sums[lane] : 0;
    int32_t si = warp_incl_scan(s);
    if (lane < nw) warp_sums[lane] = si - s;
    if (lane == nw - 1) block_total = si;
  }
  __syncthreads();
  int32_t r = inc - x + warp_sums[wid];
  *total = block_total;
  __syncthreads();
  return r;
}

__global__ void k_tile_sums(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ sums) {
  FP_PDL_WAIT();
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  int32_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i)
    if (base + i < n) s += in[base + i];
  int32_t tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One CTA scans the tile sums in place (exclusive), chunk by chunk with a carry.
__global__ void k_scan_sums(int32_t* sums, int64_t nt, int32_t* total_out) {
  FP_PDL_WAIT();
  int32_t carry = 0;
  for (int64_t base = 0; base < nt; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int32_t x = i < nt ? sums[i] : 0;
    int32_t tot;
    int32_t ex = block_excl_scan(x, &tot);
    if (i < nt) sums[i] = ex + carry;
    carry += tot;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_tile_scan(const int32_t* __restrict__ in, int64_t n, const int32_t* __restrict__ sums,
                            int32_t* __restrict__ out) {
  FP_PDL_WAIT();
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  int32_t v[SCAN_ITEMS];
  int32_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    v[i] = base + i < n ? in[base + i] : 0;
    s += v[i];
  }
  int32_t tot;
  int32_t ex = block_excl_scan(s, &tot) + sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    if (base + i < n) out[base + i] = ex;
    ex += v[i];
  }
}

// Whole scan in one CTA for short arrays (node and patch counts): chunks of
// 1024 x 4 items with a carry, out[n] = total.
__global__ void __launch_bounds__(1024) k_scan_small(const int32_t* __restrict__ in, int64_t n,
                                                     int32_t* __restrict__ out) {
  FP_PDL_WAIT();
  int32_t carry = 0;
  for (int64_t c = 0; c < n; c += 1024 * SCAN_ITEMS) {
    const int64_t base = c + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
      v[i] = base + i < n ? in[base + i] : 0;
      s += v[i];
    }
    int32_t tot;
    int32_t ex = block_excl_scan(s, &tot) + carry;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
      if (base + i < n) out[base + i] = ex;
      ex += v[i];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) out[n] = carry;
}

// Two short scans in one launch (block 0: a -> oa, block 1: b -> ob), then b
// is zeroed (so that it can serve as the scatter cursors).
__global__ void __launch_bounds__(1024) k_scan_pair_small(const int32_t* __restrict__ a, int32_t* __restrict__ oa,
                                                          int32_t* b, int32_t* __restrict__ ob, int64_t n) {
  FP_PDL_WAIT();
  const int32_t* in = blockIdx.x == 0 ? a : b;
  int32_t* out = blockIdx.x == 0 ? oa : ob;
  int32_t carry = 0;
  for (int64_t c = 0; c < n; c += 1024 * SCAN_ITEMS) {
    const int64_t base = c + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
      v[i] = base + i < n ? in[base + i] : 0;
      s += v[i];
    }
    int32_t tot;
    int32_t ex = block_excl_scan(s, &tot) + carry;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
      if (base + i < n) out[base + i] = ex;
      ex += v[i];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) out[n] = carry;
  if (blockIdx.x == 1) {
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) b[i] = 0;
  }
}

__global__ void k_fill(int32_t* p, int32_t v, int64_t n) {
  FP_PDL_WAIT();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void k_iota(int32_t* p, int64_t n) {
  FP_PDL_WAIT();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (int32_t)i;
}

}  // namespace

int64_t scan_tmp_ints(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

void scan_exclusive(fp_handle* h, const int32_t* in, int32_t* out, int64_t n, int32_t* tmp) {
  int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nt == 0) {
    FP_LAUNCH(h, k_fill, 1, 32, 0, out, 0, 1);
    return;
  }
  if (n <= 4 * 1024 * SCAN_ITEMS) {
    // short arrays: one launch instead of three
    FP_LAUNCH(h, k_scan_small, 1, 1024, 0, in, n, out);
    return;
  }
  FP_LAUNCH(h, k_tile_sums, (unsigned)nt, SCAN_THREADS, 0, in, n, tmp);
  FP_LAUNCH(h, k_scan_sums, 1, 1024, 0, tmp, nt, out + n);
  FP_LAUNCH(h, k_tile_scan, (unsigned)nt, SCAN_THREADS, 0, in, n, tmp, out);
}

void scan_exclusive_pair_zero(fp_handle* h, const int32_t* a, int32_t* oa, int32_t* b, int32_t* ob, int64_t n,
                              int32_t* tmp) {
  if (n > 0 && n <= 4 * 1024 * SCAN_ITEMS) {
    FP_LAUNCH(h, k_scan_pair_small, 2, 1024, 0, a, oa, b, ob, n);
    return;
  }
  scan_exclusive(h, a, oa, n, tmp);
  scan_exclusive(h, b, ob, n, tmp);
  fill_i32(h, b, 0, n);
}

void fill_i32(fp_handle* h, int32_t* p, int32_t v, int64_t n) {
  if (n <= 0) return;
  FP_LAUNCH(h, k_fill, grid_for(n, 256, 16), 256, 0, p, v, n);
}

void iota_i32(fp_handle* h, int32_t* p, int64_t n) {
  if (n <= 0) return;
  FP_LAUNCH(h, k_iota, grid_for(n, 256, 16), 256, 0, p, n);
}

}  // namespace fp
