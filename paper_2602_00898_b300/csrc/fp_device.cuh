// Device building blocks shared by the kernels: warp/CTA reductions and scans,
// in-place bitonic sorts, 64-bit packing helpers.
#pragma once

#include <climits>

#include "fp_internal.cuh"

namespace fp {

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <class T>
__device__ __forceinline__ T warp_min(T x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    T y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y < x ? y : x;
  }
  return x;
}

template <class T>
__device__ __forceinline__ T warp_max(T x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    T y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y > x ? y : x;
  }
  return x;
}

template <class T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ int32_t warp_incl_scan_i32(int32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// CTA-wide reductions. `red` is a shared scratch of >= 33 elements. All threads
// of the CTA must call; the result is returned to every thread.
template <class T>
__device__ __forceinline__ T block_min(T x, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  x = warp_min(x);
  __syncthreads();
  if (lane == 0) red[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T y = lane < nw ? red[lane] : red[0];
    y = warp_min(y);
    if (lane == 0) red[32] = y;
  }
  __syncthreads();
  return red[32];
}

template <class T>
__device__ __forceinline__ T block_max(T x, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  x = warp_max(x);
  __syncthreads();
  if (lane == 0) red[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T y = lane < nw ? red[lane] : red[0];
    y = warp_max(y);
    if (lane == 0) red[32] = y;
  }
  __syncthreads();
  return red[32];
}

template <class T>
__device__ __forceinline__ T block_sum(T x, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  x = warp_sum(x);
  __syncthreads();
  if (lane == 0) red[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T y = lane < nw ? red[lane] : (T)0;
    y = warp_sum(y);
    if (lane == 0) red[32] = y;
  }
  __syncthreads();
  return red[32];
}

// CTA-wide exclusive scan of one int per thread; *total gets the sum.
// `red` is a shared scratch of >= 34 ints. blockDim.x a multiple of 32.
__device__ __forceinline__ int32_t block_excl_scan_i32(int32_t x, int32_t* total, int32_t* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int32_t inc = warp_incl_scan_i32(x);
  __syncthreads();
  if (lane == 31) red[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int32_t s = lane < nw ? red[lane] : 0;
    int32_t si = warp_incl_scan_i32(s);
    if (lane < nw) red[lane] = si - s;
    if (lane == nw - 1) red[33] = si;
  }
  __syncthreads();
  int32_t r = inc - x + red[wid];
  *total = red[33];
  __syncthreads();
  return r;
}

// Ascending bitonic sort of buf[0..N) (N a power of two) by the calling warp
// (kBlock = false) or CTA (kBlock = true). buf may be shared or global memory;
// the caller must make prior writes to buf visible (sync) before the call.
template <bool kBlock, class T>
__device__ __forceinline__ void bitonic_sort(T* buf, int N, int tid, int nthr) {
  for (int k = 2; k <= N; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < N; i += nthr) {
        int ixj = i ^ j;
        if (ixj > i) {
          T a = buf[i], c = buf[ixj];
          bool up = (i & k) == 0;
          if ((a > c) == up) { buf[i] = c; buf[ixj] = a; }
        }
      }
      if (kBlock) __syncthreads(); else __syncwarp();
    }
}

// Bitonic sort (Batcher, AFIPS 1968) of N keys (a power of two) held in one
// thread's registers, ascending: every index is a compile-time constant, so
// the array stays in registers.
template <int N, class T>
__device__ __forceinline__ void thread_sort_regs(T (&x)[N]) {
#pragma unroll
  for (int k = 2; k <= N; k <<= 1)
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const T a = x[i], c = x[l];
          const bool sw = up ? (c < a) : (a < c);
          x[i] = sw ? c : a;
          x[l] = sw ? a : c;
        }
      }
}

// Calls fn(u, aux[u]) for every neighbour u of v in CSR order. The gathers
// col -> aux are dependent, so B neighbours are loaded per round: two round
// trips per B neighbours instead of two per neighbour.
template <int B, class Fn>
__device__ __forceinline__ void for_row_gather(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                               int32_t v, const int32_t* __restrict__ aux, Fn fn) {
  const int32_t e1 = rowptr[v + 1];
  for (int32_t e0 = rowptr[v]; e0 < e1; e0 += B) {
    int32_t u[B], x[B];
#pragma unroll
    for (int k = 0; k < B; ++k) u[k] = e0 + k < e1 ? col[e0 + k] : -1;
#pragma unroll
    for (int k = 0; k < B; ++k) x[k] = u[k] >= 0 ? aux[u[k]] : 0;
#pragma unroll
    for (int k = 0; k < B; ++k)
      if (u[k] >= 0) fn(u[k], x[k]);
  }
}

__device__ __forceinline__ int pow2_at_least(int x, int lo) {
  int p = lo;
  while (p < x) p <<= 1;
  return p;
}

// Tie-break hash of a vertex for separator refinement: the high 32 bits of
// SplitMix64 at state v.
__device__ __forceinline__ uint32_t tie_hash(int32_t v) {
  return (uint32_t)(splitmix64_state((uint64_t)(uint32_t)v) >> 32);
}

// A union vertex's number inside its own mesh (fused batch), or v itself.
__device__ __forceinline__ int32_t seg_local(const SegView& s, int32_t v) {
  return s.vmesh ? v - s.voff[s.vmesh[v]] : v;
}

}  // namespace fp
