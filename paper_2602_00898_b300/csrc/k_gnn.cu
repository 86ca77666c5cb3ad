// a10 learned elimination priorities (the paper orders each patch by
// minimum degree and is silent on learned orderings; the readings used here):
//
//  * leaves of the nested-dissection tree (nodes with vertices and no
//    non-empty descendant, at most 512 vertices) get a second candidate
//    order: exact minimum degree whose ties go to the smaller (key, id), key =
//    2^23 - S, S the score of a two-layer message-passing network;
//  * the candidate is kept iff its exact fill (the sum of the leaf columns'
//    counts) is smaller than plain minimum degree's; a leaf's column counts
//    depend on its own order only, so nnz(L) never exceeds the plain method's.
//
// Network (width 32): h' = ReLU(Ws h + Wn mean_{u in N_leaf(v)} h_u + b), two
// layers, head S = w.h + c, on a fixed-point grid that BF16 represents
// exactly: feature/activation codes q in [0, 255] (value q/64), weight codes
// |q| <= 255 (value q/128), biases and scores in units of 1/8192. Every dot
// product is an exact integer below 2^23, so the FP32 accumulation of the
// tensor cores is exact and the ordering decisions are reproducible bit for
// bit. The two dense layers run on the 5th-generation tensor cores: each CTA
// (one leaf) stages a 128-row tile of [h | mean h] as BF16 in shared memory
// (canonical K-major layout, no swizzle), one thread issues tcgen05.mma
// (M=128, N=32, K=16 per instruction) into a 32-column TMEM accumulator, and
// the four warps read their 32 rows back with tcgen05.ld for the integer
// epilogue (bias, ReLU, round-to-nearest-even re-quantisation).
#include <cuda_bf16.h>

#include <algorithm>

#include "fp_device.cuh"

namespace fp {

constexpr int32_t KEY_BIAS = 1 << 23;

namespace {

constexpr int SC_THREADS = 128;
constexpr uint32_t INF_DEPTH = 0xffffu;

__device__ __forceinline__ int32_t rne_div(int32_t a, int32_t b) {   // a >= 0, b > 0
  int32_t q = a / b;
  const int32_t r = a - q * b;
  if (2 * r > b || (2 * r == b && (q & 1))) ++q;
  return q;
}

// ---- tcgen05 / mbarrier helpers (inline PTX) ----------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (r, k) of a BF16 operand with K columns in the
// canonical K-major layout without swizzle: 8x8 core matrices of 128
// contiguous bytes (8 rows of 16 B); core matrices adjacent in K are 128 B
// apart (leading byte offset), 8-row groups are K/8 * 128 B apart (stride
// byte offset).
__device__ __forceinline__ uint32_t kmajor_off(int r, int k, int K) {
  return (uint32_t)(((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading / stride byte
// offsets (>> 4), descriptor version 1 (bits 46-47), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3fffu);
  d |= (uint64_t)((lbo >> 4) & 0x3fffu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3fffu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 = 1, bits 10-12 = 1), both K-major, N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
constexpr uint32_t IDESC_BF16_M128_N32 = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_alloc32(uint32_t* slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(slot)));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tc_dealloc32(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(taddr));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t taddr, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Bounded wait for the phase with the given parity: at most `polls`
// non-blocking tests of the barrier (so that a limit counts exactly); false
// if it ran out.
constexpr int64_t SPIN_DEFAULT = (int64_t)1 << 24;
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, int64_t polls) {
  const uint32_t a = smem_u32(mbar);
  for (int64_t it = 0; it < polls; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// 32 FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void put_bf16(unsigned char* base, uint32_t off, int32_t code) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn((float)code);
}

struct ScoreArgs {
  const int32_t* rowptr;
  const int32_t* col;
  const int32_t* perm;
  const int32_t* iperm;
  const int32_t* node_begin;
  const int32_t* node_size;
  const int32_t* leaves;
  int32_t nleaves;
  const int32_t* q;        // P_COUNT codes
  int32_t cap;
  uint32_t* key;           // [n] per vertex, out
  int32_t* score;          // [n] per position, out (may be NULL)
  uint8_t* xout;           // [n][8] feature codes per position, out (may be NULL)
  int32_t* status;
  int64_t max_spin;        // polls of the tensor-core completion wait
  SegView sv;              // fused batch: the cap of the leaf's own mesh
};

// shared layout of the scoring kernel (bytes)
constexpr int SC_A = 0;                       // A tile: 128 x 64 BF16
constexpr int SC_B1 = SC_A + 128 * 64 * 2;    // W1: 32 x 16 BF16
constexpr int SC_B2 = SC_B1 + 32 * 16 * 2;    // W2: 32 x 64 BF16
constexpr int SC_X = SC_B2 + 32 * 64 * 2;     // feature codes 512 x 8
constexpr int SC_H = SC_X + GNN_LEAF_MAX * 8;  // layer-1 codes 512 x 32
constexpr int SC_DEPTH = SC_H + GNN_LEAF_MAX * 32;
constexpr int SC_DEG = SC_DEPTH + GNN_LEAF_MAX * 4;
constexpr int SC_AOFF = SC_DEG + GNN_LEAF_MAX * 4;   // local adjacency: row starts (uint16)
constexpr int SC_ECAP = 4096;                         //   and up to 4096 entries (uint16)
constexpr int SC_ADJ = SC_AOFF + GNN_LEAF_MAX * 2;
constexpr int SC_BYTES = SC_ADJ + SC_ECAP * 2;
constexpr int SC_GD = 16;                             // rows gathered on chip: at most 16 entries

// Visits the within-leaf neighbours (local indices) of local vertex i.
template <class Fn>
__device__ __forceinline__ void leaf_neighbours(const ScoreArgs& a, int32_t b, int32_t m, int32_t i, Fn fn) {
  const int32_t v = a.perm[b + i];
  const int32_t e1 = a.rowptr[v + 1];
  for (int32_t e = a.rowptr[v]; e < e1; ++e) {
    const int32_t p = a.iperm[a.col[e]] - b;
    if (p >= 0 && p < m) fn(p);
  }
}

__global__ void __launch_bounds__(SC_THREADS) k_gnn_score(ScoreArgs a) {
  FP_PDL_WAIT();
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t s_mbar;
  __shared__ uint32_t s_tmem;
  __shared__ int32_t s_flag, s_dmax;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int32_t t = a.leaves[blockIdx.x];
  const int32_t m = a.node_size[t], b = a.node_begin[t];
  if (m <= 0 || m > GNN_LEAF_MAX) return;      // uniform per CTA
  const int32_t cap = a.sv.vmesh ? a.sv.mcap[a.sv.vmesh[a.perm[b]]] : a.cap;

  uint8_t* X = sm + SC_X;
  uint8_t* H = sm + SC_H;
  uint32_t* depth = (uint32_t*)(sm + SC_DEPTH);
  int32_t* degh = (int32_t*)(sm + SC_DEG);
  uint16_t* aoff = (uint16_t*)(sm + SC_AOFF);
  uint16_t* adj = (uint16_t*)(sm + SC_ADJ);
  __shared__ int32_t s_ne, s_ovf;

  if (warp == 0) tc_alloc32(&s_tmem);
  if (tid == 0) {
    mbar_init(&s_mbar, 1);
    s_dmax = 0;
    s_ne = 0;
    s_ovf = 0;
  }
  // weights as BF16 operands: B1 = [w1s | w1n | 0] (32 x 16), B2 = [w2s | w2n] (32 x 64)
  for (int x = tid; x < 32 * 16; x += SC_THREADS) {
    const int r = x >> 4, k = x & 15;
    const int32_t c = k < 6 ? a.q[P_W1S + r * 6 + k] : (k < 12 ? a.q[P_W1N + r * 6 + k - 6] : 0);
    put_bf16(sm + SC_B1, kmajor_off(r, k, 16), c);
  }
  for (int x = tid; x < 32 * 64; x += SC_THREADS) {
    const int r = x >> 6, k = x & 63;
    const int32_t c = k < 32 ? a.q[P_W2S + r * 32 + k] : a.q[P_W2N + r * 32 + k - 32];
    put_bf16(sm + SC_B2, kmajor_off(r, k, 64), c);
  }
  __syncthreads();
  // 0. the leaf's local adjacency in shared memory, gathered once: a row's
  // entries (at most SC_GD) and their positions are loaded together, the
  // within-leaf ones appended to the list by one shared atomic. A row above
  // SC_GD entries or a list above SC_ECAP leaves every pass on the global
  // rows instead (the same neighbours; every use below is order-free).
  for (int32_t i = tid; i < m; i += SC_THREADS) {
    const int32_t v = a.perm[b + i];
    const int32_t e0 = a.rowptr[v], dg = a.rowptr[v + 1] - e0;
    depth[i] = (uint32_t)dg;                       // the degree, until step 1
    if (dg > SC_GD) {
      s_ovf = 1;
      continue;
    }
    int32_t p[SC_GD];
#pragma unroll
    for (int k = 0; k < SC_GD; ++k) p[k] = k < dg ? a.col[e0 + k] : -1;
#pragma unroll
    for (int k = 0; k < SC_GD; ++k) p[k] = p[k] >= 0 ? a.iperm[p[k]] - b : -1;
    int32_t dh = 0;
#pragma unroll
    for (int k = 0; k < SC_GD; ++k) dh += (p[k] >= 0 && p[k] < m) ? 1 : 0;
    int32_t o = atomicAdd(&s_ne, dh);
    if (o + dh > SC_ECAP) {
      s_ovf = 1;
      continue;
    }
    aoff[i] = (uint16_t)o;
    degh[i] = dh;
#pragma unroll
    for (int k = 0; k < SC_GD; ++k)
      if (p[k] >= 0 && p[k] < m) adj[o++] = (uint16_t)p[k];
  }
  __syncthreads();
  const bool on_chip = s_ovf == 0;
  auto nbrs = [&](int32_t i, auto fn) {
    if (on_chip) {
      const int32_t o = aoff[i], d = degh[i];
      for (int32_t k = 0; k < d; ++k) fn((int32_t)adj[o + k]);
    } else {
      leaf_neighbours(a, b, m, i, fn);
    }
  };
  // 1. degrees and the boundary (depth 0)
  for (int32_t i = tid; i < m; i += SC_THREADS) {
    const int32_t dg = (int32_t)depth[i];
    int32_t dh = 0;
    if (on_chip) {
      dh = degh[i];
    } else {
      leaf_neighbours(a, b, m, i, [&](int32_t) { ++dh; });
      degh[i] = dh;
    }
    depth[i] = dh < dg ? 0u : INF_DEPTH;
    X[i * 8 + 1] = (uint8_t)min(8 * dg, 255);
    X[i * 8 + 2] = dh < dg ? 64 : 0;
  }
  __syncthreads();
  // 2. hop depth from the boundary inside the leaf (level-synchronous BFS)
  for (uint32_t d = 0;; ++d) {
    if (tid == 0) s_flag = 0;
    __syncthreads();
    for (int32_t i = tid; i < m; i += SC_THREADS) {
      if (depth[i] != d) continue;
      nbrs(i, [&](int32_t j) {
        if (depth[j] == INF_DEPTH) {
          depth[j] = d + 1;
          s_flag = 1;
        }
      });
    }
    __syncthreads();
    const int32_t more = s_flag;
    __syncthreads();
    if (!more) break;
  }
  int32_t dmx = 0;
  for (int32_t i = tid; i < m; i += SC_THREADS)
    if (depth[i] != INF_DEPTH) dmx = max(dmx, (int32_t)depth[i]);
  atomicMax(&s_dmax, dmx);
  __syncthreads();
  const int32_t dmax = s_dmax;
  // 3. feature codes
  for (int32_t i = tid; i < m; i += SC_THREADS) {
    const int32_t dp = depth[i] == INF_DEPTH ? dmax + 1 : (int32_t)depth[i];
    X[i * 8 + 0] = (uint8_t)min(8 * degh[i], 255);
    X[i * 8 + 3] = (uint8_t)min(rne_div(64 * dp, dmax + 1), 255);
    X[i * 8 + 4] = (uint8_t)min(rne_div(64 * m, cap), 255);
    X[i * 8 + 5] = 64;
    X[i * 8 + 6] = X[i * 8 + 7] = 0;
    if (a.xout)
      for (int k = 0; k < 8; ++k) a.xout[(int64_t)(b + i) * 8 + k] = X[i * 8 + k];
  }
  __syncthreads();

  const uint32_t tmem = s_tmem;
  const uint32_t a_addr = smem_u32(sm + SC_A), b1_addr = smem_u32(sm + SC_B1), b2_addr = smem_u32(sm + SC_B2);
  uint32_t phase = 0;
  bool ok = true;
  const int ntile = (m + 127) >> 7;
  for (int layer = 1; layer <= 2 && ok; ++layer) {
    const int K = layer == 1 ? 16 : 64;
    for (int tile = 0; tile < ntile && ok; ++tile) {
      // stage row r = tid of the tile: [own codes | neighbour mean codes]
      const int32_t i = tile * 128 + tid;
      if (layer == 1) {
        int32_t sum[6] = {0, 0, 0, 0, 0, 0};
        if (i < m) nbrs(i, [&](int32_t j) {
#pragma unroll
          for (int k = 0; k < 6; ++k) sum[k] += X[j * 8 + k];
        });
        const int32_t dh = i < m ? degh[i] : 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          int32_t c = 0;
          if (i < m) {
            if (k < 6) c = X[i * 8 + k];
            else if (k < 12) c = dh > 0 ? rne_div(sum[k - 6], dh) : 0;
          }
          put_bf16(sm + SC_A, kmajor_off(tid, k, 16), c);
        }
      } else {
        int32_t sum[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) sum[k] = 0;
        if (i < m) nbrs(i, [&](int32_t j) {
          const uint32_t* hj = (const uint32_t*)(H + j * 32);
#pragma unroll
          for (int w = 0; w < 8; ++w) {
            const uint32_t x = hj[w];
            sum[4 * w + 0] += x & 0xff;
            sum[4 * w + 1] += (x >> 8) & 0xff;
            sum[4 * w + 2] += (x >> 16) & 0xff;
            sum[4 * w + 3] += x >> 24;
          }
        });
        const int32_t dh = i < m ? degh[i] : 0;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          put_bf16(sm + SC_A, kmajor_off(tid, k, 64), i < m ? (int32_t)H[i * 32 + k] : 0);
          put_bf16(sm + SC_A, kmajor_off(tid, 32 + k, 64), (i < m && dh > 0) ? rne_div(sum[k], dh) : 0);
        }
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t bb = layer == 1 ? b1_addr : b2_addr;
        for (int kk = 0; kk < K / 16; ++kk)
          tc_mma(tmem, smem_desc(a_addr + kk * 256, 128, (K >> 3) * 128), smem_desc(bb + kk * 256, 128, (K >> 3) * 128),
                 IDESC_BF16_M128_N32, kk > 0);
        tc_commit(&s_mbar);
      }
      ok = __syncthreads_and(mbar_wait(&s_mbar, phase, a.max_spin)) != 0;
      if (!ok) {
        // the MMA did not complete within the caller's bound: wait for it
        // once more (2^24 polls at most) so that nothing is in flight when
        // the tensor memory is freed, flag the failure, and leave with the
        // accumulator unread
        if (tid == 0) {
          mbar_wait(&s_mbar, phase, SPIN_DEFAULT);
          atomicOr(a.status, ST_TIMEOUT);
        }
        break;
      }
      phase ^= 1u;
      tc_fence_after();
      float acc[32];
      tc_ld32(tmem + ((uint32_t)(warp * 32) << 16), acc);
      if (i < m) {
        if (layer == 1) {
          uint32_t packed[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int32_t z = (int32_t)acc[j] + a.q[P_B1 + j];
            const int32_t hq = min(rne_div(max(z, 0), 128), 255);
            packed[j >> 2] |= (uint32_t)hq << (8 * (j & 3));
          }
          uint32_t* hi = (uint32_t*)(H + i * 32);
          // rows of this tile are not read before the layer ends: the means of
          // layer 2 read H only in the next layer
#pragma unroll
          for (int w = 0; w < 8; ++w) hi[w] = packed[w];
        } else {
          int32_t s = a.q[P_C];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int32_t z = (int32_t)acc[j] + a.q[P_B2 + j];
            const int32_t hq = min(rne_div(max(z, 0), 128), 255);
            s += a.q[P_W3 + j] * hq;
          }
          const int32_t v = a.perm[b + i];
          a.key[v] = (uint32_t)(KEY_BIAS - s);
          if (a.score) a.score[b + i] = s;
        }
      }
      tc_fence_before();
      __syncthreads();
    }
  }
  __syncthreads();
  if (warp == 0) tc_dealloc32(tmem);
}

// Keeps the learned order of a leaf iff its fill is smaller. stats[4 m + 0..3]
// of the leaf's mesh m (0 for one mesh): learned orders kept, summed plain
// fills, summed chosen fills, leaves.
__global__ void k_choose(const int32_t* __restrict__ leaves, int32_t nl, const int32_t* __restrict__ node_begin,
                         const int32_t* __restrict__ node_size, const int64_t* __restrict__ fill_p,
                         const int64_t* __restrict__ fill_l, const int32_t* __restrict__ perm_l,
                         int32_t* __restrict__ perm, unsigned long long* __restrict__ stats, SegView sv) {
  FP_PDL_WAIT();
  const int32_t t = leaves[blockIdx.x];
  const bool keep = fill_l[t] < fill_p[t];
  const int32_t b = node_begin[t], m = node_size[t];
  if (keep)
    for (int32_t i = threadIdx.x; i < m; i += blockDim.x) perm[b + i] = perm_l[b + i];
  if (threadIdx.x == 0) {
    unsigned long long* st = stats + (sv.vmesh ? 4 * (int64_t)sv.vmesh[perm_l[b]] : 0);
    atomicAdd(&st[0], keep ? 1ull : 0ull);
    atomicAdd(&st[1], (unsigned long long)fill_p[t]);
    atomicAdd(&st[2], (unsigned long long)(keep ? fill_l[t] : fill_p[t]));
    atomicAdd(&st[3], 1ull);
  }
}

// A provisional permutation while the separators are still being ordered on
// the auxiliary streams: every vertex takes a place inside its node's range
// (its index in the node's vertex list) ...
__global__ void k_prov_perm(const int32_t* __restrict__ nvlist, const int32_t* __restrict__ nvstart,
                            const int32_t* __restrict__ node_of, const int32_t* __restrict__ node_begin, int32_t n,
                            int32_t* __restrict__ perm_p) {
  FP_PDL_WAIT();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int32_t v = nvlist[i], t = node_of[v];
    perm_p[node_begin[t] + (i - nvstart[t])] = v;
  }
}

// ... and the listed leaves their final order (one CTA a leaf).
__global__ void k_leaf_orders(const int32_t* __restrict__ leaves, const int32_t* __restrict__ node_begin,
                              const int32_t* __restrict__ node_size, const int32_t* __restrict__ perm,
                              int32_t* __restrict__ perm_p) {
  FP_PDL_WAIT();
  const int32_t t = leaves[blockIdx.x], b = node_begin[t], m = node_size[t];
  for (int32_t i = threadIdx.x; i < m; i += blockDim.x) perm_p[b + i] = perm[b + i];
}

__global__ void k_scatter_inverse(const int32_t* __restrict__ perm, int32_t n, int32_t* __restrict__ iperm) {
  FP_PDL_WAIT();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) iperm[perm[i]] = i;
}

}  // namespace

// Leaves of the tree (nodes with vertices and no non-empty descendant) with
// at most 512 vertices, from the node sizes; returns the list on the device.
fp_status leaf_list(fp_handle* h, std::vector<int32_t>& hl, int32_t** d_list, int32_t* mmax, std::vector<int32_t>* lsz) {
  const int64_t nn = h->nnodes;
  std::vector<int32_t> sz(nn);
  cudaError_t e = cudaMemcpyAsync(sz.data(), h->node_size, sizeof(int32_t) * nn, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "node sizes");
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "node sizes");
  std::vector<int64_t> sub(sz.begin(), sz.end());
  for (int64_t t = nn - 1; t >= 0; --t)
    for (int64_t c = 2 * t + 1; c <= 2 * t + 2; ++c)
      if (c < nn) sub[t] += sub[c];
  hl.clear();
  *mmax = 0;
  for (int64_t t = 0; t < nn; ++t)
    if (sz[t] > 0 && sub[t] == sz[t] && sz[t] <= GNN_LEAF_MAX) {
      hl.push_back((int32_t)t);
      *mmax = std::max(*mmax, sz[t]);
    }
  // largest first: the per-leaf kernels that draw leaves from a queue balance better
  std::stable_sort(hl.begin(), hl.end(), [&](int32_t x, int32_t y) { return sz[x] > sz[y]; });
  if (lsz) {
    lsz->resize(hl.size());
    for (size_t i = 0; i < hl.size(); ++i) (*lsz)[i] = sz[hl[i]];
  }
  *d_list = (int32_t*)dev_alloc(h, sizeof(int32_t) * (hl.size() + 1));
  if (!*d_list) return fail(h, FP_ERR_OUT_OF_MEMORY, "leaf list");
  if (!hl.empty()) {
    e = cudaMemcpyAsync(*d_list, hl.data(), sizeof(int32_t) * hl.size(), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return check_cuda(h, e, "leaf list");
  }
  return FP_OK;
}

fp_status launch_gnn_score(fp_handle* h, const int32_t* d_leaves, int32_t nl, const int32_t* d_q, uint32_t* d_key,
                           int32_t* d_score, uint8_t* d_x, const int32_t* perm, const int32_t* iperm) {
  if (nl == 0) return FP_OK;
  ScoreArgs sa{h->rowptr, h->col, perm ? perm : h->perm, iperm ? iperm : h->iperm, h->node_begin, h->node_size,
               d_leaves, nl, d_q,
               h->opt.patch_cap, d_key, d_score, d_x, h->d_status,
               h->opt.max_spin > 0 ? h->opt.max_spin : SPIN_DEFAULT, h->seg ? h->seg->v : SegView{}};
  allow_max_dynamic_smem(k_gnn_score);
  FP_LAUNCH(h, k_gnn_score, nl, SC_THREADS, (size_t)SC_BYTES, sa);
  FP_CHECK_LAUNCH(h, "network scores");
  return FP_OK;
}

fp_status run_learned(fp_handle* h) {
  // the separator orderings left running by run_local_order are joined on
  // every way out
  struct JoinGuard {
    fp_handle* h;
    ~JoinGuard() { if (h->join_pending) finish_orderings(h); }
  } jg{h};
  const int32_t n = h->n;
  h->learned_leaves = h->learned_kept = 0;
  h->fill_plain = h->fill_chosen = 0;
  if (!h->qnet || n == 0) return finish_orderings(h);
  ProfScope ps(FP_PROF_LEARNED, h->stream);
  std::vector<int32_t> hl, lsz;
  int32_t* dl = nullptr;
  int32_t mmax = 0;
  FP_TRY(leaf_list(h, hl, &dl, &mmax, &lsz));
  const int32_t nl = (int32_t)hl.size();
  const int64_t nn = h->nnodes;
  uint32_t* key = (uint32_t*)dev_alloc(h, sizeof(uint32_t) * n);
  int32_t* vlist = (int32_t*)dev_alloc(h, sizeof(int32_t) * n);
  int32_t* loc = (int32_t*)dev_alloc(h, sizeof(int32_t) * n);
  int32_t* perm_l = (int32_t*)dev_alloc(h, sizeof(int32_t) * n);
  int32_t* iperm_l = (int32_t*)dev_alloc(h, sizeof(int32_t) * n);
  int64_t* fills = (int64_t*)dev_alloc(h, sizeof(int64_t) * 2 * nn);
  const int32_t nst = h->seg ? 4 * h->seg->M : 4;
  unsigned long long* stats = (unsigned long long*)dev_alloc(h, sizeof(unsigned long long) * nst);
  if (!key || !vlist || !loc || !perm_l || !iperm_l || !fills || !stats)
    return fail(h, FP_ERR_OUT_OF_MEMORY, "learned ordering workspace");
  cudaMemsetAsync(key, 0, sizeof(uint32_t) * n, h->stream);
  cudaMemsetAsync(fills, 0, sizeof(int64_t) * 2 * nn, h->stream);
  cudaMemsetAsync(stats, 0, sizeof(unsigned long long) * nst, h->stream);
  const int G = (int)std::min<int64_t>((n + 255) / 256, NUM_SMS_B300 * 8);
  // positions this pass reads: the final ones once the orderings are joined;
  // while the separators are still being ordered, a provisional permutation
  // with the leaves' final orders. A leaf's scores and column counts depend
  // on its own order and on which node each other vertex lies in, not on
  // the order inside those nodes.
  const int32_t* pm = h->perm;
  const int32_t* ipm = h->iperm;
  int32_t *perm_p = nullptr, *iperm_p = nullptr;
  if (h->join_pending) {
    perm_p = (int32_t*)dev_alloc(h, sizeof(int32_t) * n);
    iperm_p = (int32_t*)dev_alloc(h, sizeof(int32_t) * n);
    if (!perm_p || !iperm_p) return fail(h, FP_ERR_OUT_OF_MEMORY, "provisional permutation");
    FP_LAUNCH(h, k_prov_perm, G, 256, 0, h->pend_nvlist, h->pend_nvstart, h->node_of, h->node_begin, n, perm_p);
    if (nl > 0) FP_LAUNCH(h, k_leaf_orders, nl, 128, 0, dl, h->node_begin, h->node_size, h->perm, perm_p);
    FP_LAUNCH(h, k_scatter_inverse, G, 256, 0, perm_p, n, iperm_p);
    pm = perm_p;
    ipm = iperm_p;
  }
  FP_TRY(launch_gnn_score(h, dl, nl, h->qnet, key, h->scores, nullptr, pm, ipm));
  cudaMemcpyAsync(vlist, pm, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(perm_l, pm, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, h->stream);
  FP_TRY(run_leaf_md_keyed(h, dl, nl, mmax, vlist, loc, key, perm_l, &lsz));
  FP_LAUNCH(h, k_scatter_inverse, G, 256, 0, perm_l, n, iperm_l);
  FP_TRY(run_leaf_fill(h, pm, ipm, dl, nl, fills));
  FP_TRY(run_leaf_fill(h, perm_l, iperm_l, dl, nl, fills + nn));
  if (nl > 0)
    FP_LAUNCH(h, k_choose, nl, 128, 0, dl, nl, h->node_begin, h->node_size, fills, fills + nn, perm_l, h->perm, stats,
              h->seg ? h->seg->v : SegView{});
  ps.end();
  FP_TRY(finish_orderings(h));
  FP_LAUNCH(h, k_scatter_inverse, G, 256, 0, h->perm, n, h->iperm);
  FP_CHECK_LAUNCH(h, "learned choice");
  std::vector<unsigned long long> hs(nst);
  cudaError_t e = cudaMemcpyAsync(hs.data(), stats, sizeof(unsigned long long) * nst, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "learned stats");
  int32_t st = 0;
  FP_TRY(sync_status(h, &st));
  if (st & ST_TIMEOUT) return fail(h, FP_ERR_TIMEOUT, "tensor-core wait ran out");
  if (h->seg) h->seg->h_learned = hs;
  unsigned long long tot[3] = {0, 0, 0};
  for (int32_t i = 0; i < nst; i += 4)
    for (int c = 0; c < 3; ++c) tot[c] += hs[i + c];
  h->learned_leaves = nl;
  h->learned_kept = (int32_t)tot[0];
  h->fill_plain = (int64_t)tot[1];
  h->fill_chosen = (int64_t)tot[2];
  for (void* p : {(void*)dl, (void*)key, (void*)vlist, (void*)loc, (void*)perm_l, (void*)iperm_l, (void*)fills,
                  (void*)stats, (void*)perm_p, (void*)iperm_p})
    if (p) dev_free(h, p);
  return FP_OK;
}

}  // namespace fp
