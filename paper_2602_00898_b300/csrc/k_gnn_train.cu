// a10 training: samples (features, within-leaf graph, best-order targets) and
// the float network's gradient step.
//
// Sample of a plain ordering: per leaf, plain minimum degree and n_seeds
// minimum-degree orders whose ties go to seeded keys (the high 32 bits of
// SplitMix64 at state r*gamma + v) compete on exact fill (the sum of the leaf
// columns' counts); the winner (ties to the lower r) gives every leaf vertex
// the target (m-1-rank)/(m-1).
//
// Gradient step: the network without the fixed-point grid (activations
// clamped to [0, 255/64], the range of the codes), loss = mean squared error
// over the leaf positions, exact backward pass, then params -= lr * grad.
// Positions are split into fixed chunks of GT_CHUNK; each CTA stages its
// chunk's activations in shared memory and writes one partial gradient per
// parameter; a second kernel sums the partials in chunk order. The reduction
// order is fixed, so the step is deterministic.
#include "fp_device.cuh"

namespace fp {
namespace {

constexpr int GT_CHUNK = 64;
constexpr int GT_THREADS = 256;
constexpr float HF_MAX = 255.0f / 64.0f;

struct TrainBufs {
  float *m0, *z1, *h1, *m1, *z2, *h2, *dz2, *g, *dz1, *ds, *lossp, *partial;
  int32_t* count;
};

int64_t nchunks(int32_t n) { return ((int64_t)n + GT_CHUNK - 1) / GT_CHUNK; }

TrainBufs carve(void* work, int32_t n) {
  TrainBufs b;
  float* f = (float*)work;
  const int64_t N = n;
  b.m0 = f; f += N * 8;
  b.z1 = f; f += N * 32;
  b.h1 = f; f += N * 32;
  b.m1 = f; f += N * 32;
  b.z2 = f; f += N * 32;
  b.h2 = f; f += N * 32;
  b.dz2 = f; f += N * 32;
  b.g = f; f += N * 32;
  b.dz1 = f; f += N * 32;
  b.ds = f; f += N;
  b.lossp = f; f += nchunks(n);
  b.partial = f; f += nchunks(n) * P_COUNT;
  b.count = (int32_t*)f;
  return b;
}

__device__ __forceinline__ float xval(const uint8_t* x, int64_t p, int k) { return (float)x[p * 8 + k] * (1.0f / 64.0f); }

// layer 1 forward, one position per thread
__global__ void k_train_fwd1(const float* __restrict__ P, const uint8_t* __restrict__ x,
                             const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const uint8_t* __restrict__ mask, int32_t n, TrainBufs b) {
  FP_PDL_WAIT();
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    if (mask[p]) atomicAdd(b.count, 1);
    float m0[6] = {0, 0, 0, 0, 0, 0};
    const int32_t r0 = rp[p], r1 = rp[p + 1];
    for (int32_t e = r0; e < r1; ++e)
      for (int k = 0; k < 6; ++k) m0[k] += xval(x, col[e], k);
    if (r1 > r0)
      for (int k = 0; k < 6; ++k) m0[k] /= (float)(r1 - r0);
    for (int k = 0; k < 6; ++k) b.m0[(int64_t)p * 8 + k] = m0[k];
    for (int j = 0; j < 32; ++j) {
      float z = P[P_B1 + j];
      for (int k = 0; k < 6; ++k) z += P[P_W1S + j * 6 + k] * xval(x, p, k) + P[P_W1N + j * 6 + k] * m0[k];
      b.z1[(int64_t)p * 32 + j] = z;
      b.h1[(int64_t)p * 32 + j] = fminf(fmaxf(z, 0.0f), HF_MAX);
    }
  }
}

// layer 2 forward, head, loss residual and the layer-2 backward rows
__global__ void k_train_fwd2(const float* __restrict__ P, const int32_t* __restrict__ rp,
                             const int32_t* __restrict__ col, const uint8_t* __restrict__ mask,
                             const float* __restrict__ target, int32_t n, TrainBufs b) {
  FP_PDL_WAIT();
  const float N = fmaxf((float)*b.count, 1.0f);
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    float m1[32];
    for (int k = 0; k < 32; ++k) m1[k] = 0.0f;
    const int32_t r0 = rp[p], r1 = rp[p + 1];
    for (int32_t e = r0; e < r1; ++e)
      for (int k = 0; k < 32; ++k) m1[k] += b.h1[(int64_t)col[e] * 32 + k];
    if (r1 > r0)
      for (int k = 0; k < 32; ++k) m1[k] /= (float)(r1 - r0);
    float s = P[P_C];
    float h2[32], z2[32];
    for (int j = 0; j < 32; ++j) {
      float z = P[P_B2 + j];
      for (int k = 0; k < 32; ++k) z += P[P_W2S + j * 32 + k] * b.h1[(int64_t)p * 32 + k] + P[P_W2N + j * 32 + k] * m1[k];
      z2[j] = z;
      h2[j] = fminf(fmaxf(z, 0.0f), HF_MAX);
      s += P[P_W3 + j] * h2[j];
    }
    const float r = mask[p] ? s - target[p] : 0.0f;
    const float ds = 2.0f * r / N;
    b.ds[p] = ds;
    for (int k = 0; k < 32; ++k) {
      b.m1[(int64_t)p * 32 + k] = m1[k];
      b.z2[(int64_t)p * 32 + k] = z2[k];
      b.h2[(int64_t)p * 32 + k] = h2[k];
    }
    float dz2[32];
    for (int j = 0; j < 32; ++j) {
      dz2[j] = (z2[j] > 0.0f && z2[j] < HF_MAX) ? ds * P[P_W3 + j] : 0.0f;
      b.dz2[(int64_t)p * 32 + j] = dz2[j];
    }
    // message gradient sent back to the neighbours: Wn^T dz2 / deg
    const float inv = r1 > r0 ? 1.0f / (float)(r1 - r0) : 0.0f;
    for (int k = 0; k < 32; ++k) {
      float gk = 0.0f;
      for (int j = 0; j < 32; ++j) gk += P[P_W2N + j * 32 + k] * dz2[j];
      b.g[(int64_t)p * 32 + k] = r1 > r0 ? gk * inv : 0.0f;
    }
  }
}

// layer 1 backward rows
__global__ void k_train_bwd1(const float* __restrict__ P, const int32_t* __restrict__ rp,
                             const int32_t* __restrict__ col, int32_t n, TrainBufs b) {
  FP_PDL_WAIT();
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    float dh[32];
    for (int k = 0; k < 32; ++k) {
      float v = 0.0f;
      for (int j = 0; j < 32; ++j) v += P[P_W2S + j * 32 + k] * b.dz2[(int64_t)p * 32 + j];
      dh[k] = v;
    }
    for (int32_t e = rp[p]; e < rp[p + 1]; ++e)
      for (int k = 0; k < 32; ++k) dh[k] += b.g[(int64_t)col[e] * 32 + k];
    for (int k = 0; k < 32; ++k) {
      const float z = b.z1[(int64_t)p * 32 + k];
      b.dz1[(int64_t)p * 32 + k] = (z > 0.0f && z < HF_MAX) ? dh[k] : 0.0f;
    }
  }
}

// per-chunk partial gradients (one CTA per chunk, activations in shared memory)
__global__ void __launch_bounds__(GT_THREADS) k_train_partial(const uint8_t* __restrict__ x,
                                                              const uint8_t* __restrict__ mask,
                                                              const float* __restrict__ target,
                                                              const float* __restrict__ P, int32_t n, TrainBufs b) {
  FP_PDL_WAIT();
  __shared__ float sx[GT_CHUNK][6], sm0[GT_CHUNK][6], sh1[GT_CHUNK][32], sm1[GT_CHUNK][32], sh2[GT_CHUNK][32],
      sdz2[GT_CHUNK][32], sdz1[GT_CHUNK][32], sds[GT_CHUNK];
  const int64_t c = blockIdx.x;
  const int32_t p0 = (int32_t)(c * GT_CHUNK);
  const int cnt = min(GT_CHUNK, n - p0);
  for (int i = threadIdx.x; i < GT_CHUNK * 32; i += GT_THREADS) {
    const int r = i >> 5, k = i & 31;
    const bool in = r < cnt;
    const int64_t p = (int64_t)p0 + r;
    sh1[r][k] = in ? b.h1[p * 32 + k] : 0.0f;
    sm1[r][k] = in ? b.m1[p * 32 + k] : 0.0f;
    sh2[r][k] = in ? b.h2[p * 32 + k] : 0.0f;
    sdz2[r][k] = in ? b.dz2[p * 32 + k] : 0.0f;
    sdz1[r][k] = in ? b.dz1[p * 32 + k] : 0.0f;
    if (k < 6) {
      sx[r][k] = in ? xval(x, p, k) : 0.0f;
      sm0[r][k] = in ? b.m0[p * 8 + k] : 0.0f;
    }
    if (k == 0) sds[r] = in ? b.ds[p] : 0.0f;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < P_COUNT; j += GT_THREADS) {
    float acc = 0.0f;
    if (j < P_W1N) {
      const int a = (j - P_W1S) / 6, k = (j - P_W1S) % 6;
      for (int r = 0; r < GT_CHUNK; ++r) acc += sdz1[r][a] * sx[r][k];
    } else if (j < P_B1) {
      const int a = (j - P_W1N) / 6, k = (j - P_W1N) % 6;
      for (int r = 0; r < GT_CHUNK; ++r) acc += sdz1[r][a] * sm0[r][k];
    } else if (j < P_W2S) {
      const int a = j - P_B1;
      for (int r = 0; r < GT_CHUNK; ++r) acc += sdz1[r][a];
    } else if (j < P_W2N) {
      const int a = (j - P_W2S) / 32, k = (j - P_W2S) % 32;
      for (int r = 0; r < GT_CHUNK; ++r) acc += sdz2[r][a] * sh1[r][k];
    } else if (j < P_B2) {
      const int a = (j - P_W2N) / 32, k = (j - P_W2N) % 32;
      for (int r = 0; r < GT_CHUNK; ++r) acc += sdz2[r][a] * sm1[r][k];
    } else if (j < P_W3) {
      const int a = j - P_B2;
      for (int r = 0; r < GT_CHUNK; ++r) acc += sdz2[r][a];
    } else if (j < P_C) {
      const int a = j - P_W3;
      for (int r = 0; r < GT_CHUNK; ++r) acc += sds[r] * sh2[r][a];
    } else {
      for (int r = 0; r < GT_CHUNK; ++r) acc += sds[r];
    }
    b.partial[c * P_COUNT + j] = acc;
  }
  if (threadIdx.x == 0) {
    // loss partial: sum of squared residuals of the chunk, in position order
    const float N = fmaxf((float)*b.count, 1.0f);
    float l = 0.0f;
    for (int r = 0; r < cnt; ++r) {
      const float res = sds[r] * N * 0.5f;
      l += res * res;
    }
    b.lossp[c] = l;
  }
}

// sum of the partials in chunk order, the loss, and the update
__global__ void k_train_reduce(float* __restrict__ P, float* __restrict__ grad, float lr, int64_t nch,
                               float* __restrict__ loss, TrainBufs b) {
  FP_PDL_WAIT();
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P_COUNT; j += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int64_t c = 0; c < nch; ++c) s += b.partial[c * P_COUNT + j];
    grad[j] = s;
    P[j] -= lr * s;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
    float l = 0.0f;
    for (int64_t c = 0; c < nch; ++c) l += b.lossp[c];
    *loss = l / fmaxf((float)*b.count, 1.0f);
  }
}

__global__ void k_quantise(const float* __restrict__ P, int32_t* __restrict__ Q) {
  FP_PDL_WAIT();
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P_COUNT; j += gridDim.x * blockDim.x) {
    const bool bias = (j >= P_B1 && j < P_W2S) || (j >= P_B2 && j < P_W3) || j == P_C;
    const float scale = bias ? 8192.0f : 128.0f;
    const float lim = bias ? 1048576.0f : 255.0f;
    Q[j] = (int32_t)fminf(fmaxf(rintf(P[j] * scale), -lim), lim);
  }
}

// ---- samples -------------------------------------------------------------------

__global__ void k_scatter_positions(const int32_t* __restrict__ perm, int32_t n, int32_t* __restrict__ iperm) {
  FP_PDL_WAIT();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) iperm[perm[i]] = i;
}

__global__ void k_seed_keys(int32_t n, uint64_t r, uint32_t* __restrict__ key) {
  FP_PDL_WAIT();
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    key[v] = r == 0 ? 0u : (uint32_t)(splitmix64_state(r * 0x9E3779B97F4A7C15ull + (uint64_t)(uint32_t)v) >> 32);
}

// keeps candidate r of a leaf if its fill is lower than the best so far
__global__ void k_keep_best(const int32_t* __restrict__ leaves, const int32_t* __restrict__ node_begin,
                            const int32_t* __restrict__ node_size, const int64_t* __restrict__ fill, int32_t r,
                            int64_t* __restrict__ best_fill, const int32_t* __restrict__ perm_r,
                            int32_t* __restrict__ best_perm) {
  FP_PDL_WAIT();
  const int32_t t = leaves[blockIdx.x];
  const bool take = r == 0 || fill[t] < best_fill[t];
  if (take) {
    const int32_t b = node_begin[t], m = node_size[t];
    for (int32_t i = threadIdx.x; i < m; i += blockDim.x) best_perm[b + i] = perm_r[b + i];
  }
  __syncthreads();
  if (threadIdx.x == 0 && take) best_fill[t] = fill[t];
}

__global__ void k_targets(const int32_t* __restrict__ leaves, const int32_t* __restrict__ node_begin,
                          const int32_t* __restrict__ node_size, const int32_t* __restrict__ best_perm,
                          const int32_t* __restrict__ iperm, float* __restrict__ target, int32_t* __restrict__ rank,
                          uint8_t* __restrict__ mask) {
  FP_PDL_WAIT();
  const int32_t t = leaves[blockIdx.x];
  const int32_t b = node_begin[t], m = node_size[t];
  for (int32_t k = threadIdx.x; k < m; k += blockDim.x) {
    const int32_t p = iperm[best_perm[b + k]];
    target[p] = m == 1 ? 1.0f : (float)(m - 1 - k) / (float)(m - 1);
    if (rank) rank[p] = k;
    mask[p] = 1;
  }
}

// within-leaf neighbour counts per position, then the neighbour positions
__global__ void k_leaf_degree(const int32_t* __restrict__ leaves, const int32_t* __restrict__ node_begin,
                              const int32_t* __restrict__ node_size, const int32_t* __restrict__ perm,
                              const int32_t* __restrict__ iperm, const int32_t* __restrict__ rowptr,
                              const int32_t* __restrict__ col, int32_t* __restrict__ deg, int32_t* __restrict__ lcol,
                              const int32_t* __restrict__ lrowptr) {
  FP_PDL_WAIT();
  const int32_t t = leaves[blockIdx.x];
  const int32_t b = node_begin[t], m = node_size[t];
  for (int32_t i = threadIdx.x; i < m; i += blockDim.x) {
    const int32_t v = perm[b + i];
    int32_t c = 0;
    for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
      const int32_t q = iperm[col[e]];
      if (q >= b && q < b + m) {
        if (lcol) lcol[lrowptr[b + i] + c] = q;
        ++c;
      }
    }
    if (deg) deg[b + i] = c;
  }
}

}  // namespace

int64_t train_work_bytes(int32_t n) {
  const int64_t N = n > 0 ? n : 1;
  return sizeof(float) * (N * 8 + N * 32 * 8 + N + nchunks((int32_t)N) + nchunks((int32_t)N) * P_COUNT) + 64;
}

fp_status train_step(float* P, float* grad, const uint8_t* x, const uint8_t* mask, const float* target,
                     const int32_t* lrp, const int32_t* lcol, int32_t n, float lr, float* loss, void* work,
                     int64_t work_bytes, cudaStream_t s) {
  if (!P || !grad || !x || !mask || !target || !lrp || n < 1 || !work || work_bytes < train_work_bytes(n))
    return fail(nullptr, FP_ERR_INVALID_ARG, "bad training arguments");
  TrainBufs b = carve(work, n);
  const int G = (int)std::min<int64_t>(((int64_t)n + 127) / 128, NUM_SMS_B300 * 8);
  ProfScope ps(FP_PROF_TRAIN, s);
  cudaMemsetAsync(b.count, 0, sizeof(int32_t), s);
  k_train_fwd1<<<G, 128, 0, s>>>(P, x, lrp, lcol, mask, n, b);
  k_train_fwd2<<<G, 128, 0, s>>>(P, lrp, lcol, mask, target, n, b);
  k_train_bwd1<<<G, 128, 0, s>>>(P, lrp, lcol, n, b);
  const int64_t nch = nchunks(n);
  k_train_partial<<<(unsigned)nch, GT_THREADS, 0, s>>>(x, mask, target, P, n, b);
  k_train_reduce<<<(P_COUNT + 255) / 256, 256, 0, s>>>(P, grad, lr, nch, loss, b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(nullptr, FP_ERR_CUDA, cudaGetErrorString(e));
  return FP_OK;
}

fp_status quantise_params(const float* P, int32_t* Q, cudaStream_t s) {
  if (!P || !Q) return fail(nullptr, FP_ERR_INVALID_ARG, "NULL parameters");
  k_quantise<<<(P_COUNT + 255) / 256, 256, 0, s>>>(P, Q);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FP_OK : fail(nullptr, FP_ERR_CUDA, cudaGetErrorString(e));
}

fp_status gnn_sample(fp_handle* h, int32_t n_seeds, uint8_t* d_x, uint8_t* d_mask, float* d_target, int32_t* d_rank,
                     int32_t* d_lrowptr, int32_t* d_lcol, int64_t lcol_cap, int64_t* h_lnnz) {
  const int32_t n = h->n;
  if (n_seeds < 0 || n_seeds > 64 || !d_x || !d_mask || !d_target || !d_lrowptr || !h_lnnz)
    return fail(h, FP_ERR_INVALID_ARG, "bad sample arguments");
  ProfScope ps(FP_PROF_TRAIN, h->stream);
  std::vector<int32_t> hl, lsz;
  int32_t* dl = nullptr;
  int32_t mmax = 0;
  FP_TRY(leaf_list(h, hl, &dl, &mmax, &lsz));
  const int32_t nl = (int32_t)hl.size();
  const int64_t nn = h->nnodes;
  // within-leaf graph: counts -> scan -> neighbour positions
  int32_t* deg = (int32_t*)dev_alloc(h, sizeof(int32_t) * (n + 1));
  int32_t* tmp = (int32_t*)dev_alloc(h, sizeof(int32_t) * (scan_tmp_ints(n) + 8));
  if (!deg || !tmp) return fail(h, FP_ERR_OUT_OF_MEMORY, "sample workspace");
  fill_i32(h, deg, 0, n);
  if (nl) FP_LAUNCH(h, k_leaf_degree, nl, 128, 0, dl, h->node_begin, h->node_size, h->perm, h->iperm, h->rowptr,
                    h->col, deg, (int32_t*)nullptr, (const int32_t*)nullptr);
  scan_exclusive(h, deg, d_lrowptr, n, tmp);
  int32_t tot = 0;
  cudaError_t e = cudaMemcpyAsync(&tot, d_lrowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "sample sizes");
  *h_lnnz = tot;
  if (tot > lcol_cap || (tot > 0 && !d_lcol)) return fail(h, FP_ERR_INVALID_ARG, "lcol_cap too small");
  if (nl && tot) FP_LAUNCH(h, k_leaf_degree, nl, 128, 0, dl, h->node_begin, h->node_size, h->perm, h->iperm,
                           h->rowptr, h->col, (int32_t*)nullptr, d_lcol, (const int32_t*)d_lrowptr);
  // features (the scoring kernel with a zero network writes the codes)
  int32_t* q = (int32_t*)dev_alloc(h, sizeof(int32_t) * P_COUNT);
  uint32_t* key = (uint32_t*)dev_alloc(h, sizeof(uint32_t) * n);
  int32_t* vlist = (int32_t*)dev_alloc(h, sizeof(int32_t) * n);
  int32_t* loc = (int32_t*)dev_alloc(h, sizeof(int32_t) * n);
  int32_t* perm_r = (int32_t*)dev_alloc(h, sizeof(int32_t) * n);
  int32_t* iperm_r = (int32_t*)dev_alloc(h, sizeof(int32_t) * n);
  int32_t* best = (int32_t*)dev_alloc(h, sizeof(int32_t) * n);
  int64_t* fill = (int64_t*)dev_alloc(h, sizeof(int64_t) * 2 * nn);
  if (!q || !key || !vlist || !loc || !perm_r || !iperm_r || !best || !fill)
    return fail(h, FP_ERR_OUT_OF_MEMORY, "sample workspace");
  cudaMemsetAsync(q, 0, sizeof(int32_t) * P_COUNT, h->stream);
  cudaMemsetAsync(d_x, 0, (size_t)8 * n, h->stream);
  cudaMemsetAsync(d_mask, 0, (size_t)n, h->stream);
  cudaMemsetAsync(d_target, 0, sizeof(float) * n, h->stream);
  if (d_rank) fill_i32(h, d_rank, -1, n);
  FP_TRY(launch_gnn_score(h, dl, nl, q, key, nullptr, d_x));
  // candidates r = 0 (plain) .. n_seeds
  const int G = (int)std::min<int64_t>(((int64_t)n + 255) / 256, NUM_SMS_B300 * 8);
  for (int32_t r = 0; r <= n_seeds; ++r) {
    FP_LAUNCH(h, k_seed_keys, G, 256, 0, n, (uint64_t)r, key);
    cudaMemcpyAsync(vlist, h->perm, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync(perm_r, h->perm, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, h->stream);
    FP_TRY(run_leaf_md_keyed(h, dl, nl, mmax, vlist, loc, r == 0 ? nullptr : key, perm_r, &lsz));
    FP_LAUNCH(h, k_scatter_positions, G, 256, 0, perm_r, n, iperm_r);
    FP_TRY(run_leaf_fill(h, perm_r, iperm_r, dl, nl, fill));
    if (nl) FP_LAUNCH(h, k_keep_best, nl, 128, 0, dl, h->node_begin, h->node_size, fill, r, fill + nn, perm_r, best);
  }
  if (nl) FP_LAUNCH(h, k_targets, nl, 128, 0, dl, h->node_begin, h->node_size, best, h->iperm, d_target, d_rank, d_mask);
  FP_CHECK_LAUNCH(h, "training sample");
  int32_t st = 0;
  FP_TRY(sync_status(h, &st));
  for (void* p : {(void*)dl, (void*)deg, (void*)tmp, (void*)q, (void*)key, (void*)vlist, (void*)loc, (void*)perm_r,
                  (void*)iperm_r, (void*)best, (void*)fill})
    dev_free(h, p);
  if (st & ST_TIMEOUT) return fail(h, FP_ERR_TIMEOUT, "tensor-core wait ran out");
  return FP_OK;
}

}  // namespace fp

using namespace fp;

extern "C" {

int64_t fp_gnn_train_work_bytes(int32_t n) { return train_work_bytes(n); }

fp_status fp_gnn_train_step(float* d_params, float* d_grad, const uint8_t* d_x, const uint8_t* d_mask,
                            const float* d_target, const int32_t* d_lrowptr, const int32_t* d_lcol, int32_t n,
                            float lr, float* d_loss, void* d_work, int64_t work_bytes, void* stream) {
  return train_step(d_params, d_grad, d_x, d_mask, d_target, d_lrowptr, d_lcol, n, lr, d_loss, d_work, work_bytes,
                    (cudaStream_t)stream);
}

fp_status fp_gnn_quantise(const float* d_params, int32_t* d_codes, void* stream) {
  return quantise_params(d_params, d_codes, (cudaStream_t)stream);
}

fp_status fp_gnn_sample(fp_handle* h, int32_t n_seeds, uint8_t* d_x, uint8_t* d_mask, float* d_target,
                        int32_t* d_rank, int32_t* d_lrowptr, int32_t* d_lcol, int64_t lcol_cap, int64_t* h_lnnz) {
  if (!h) return fail(nullptr, FP_ERR_INVALID_ARG, "NULL handle");
  if (h->poisoned) return fail(h, FP_ERR_STATE, "handle poisoned by an earlier failure");
  if (!h->permuted || h->qnet) return fail(h, FP_ERR_STATE, "fp_gnn_sample needs a plain fp_permute first");
  return gnn_sample(h, n_seeds, d_x, d_mask, d_target, d_rank, d_lrowptr, d_lcol, lcol_cap, h_lnnz);
}

}  // extern "C"
