// Allocation-free variant of the CSR assembly (fp_graph_from_faces_static).
//
// Some callers cannot allocate device memory when they need the graph: a
// process whose device memory is entirely reserved by another framework's
// caching allocator (a cudaMalloc would fail or fragment it), or a latency-
// critical loop that must not enter the CUDA allocator at all. For them
// this entry point builds the same CSR as fp_create_from_faces + fp_get_graph
// into caller-provided buffers, with all intermediate data in one fixed-size
// scratch array that lives in the library image itself (a file-scope
// __device__ array): every GPU that loads the library holds it, about 4.5 MB
// (SCRATCH_INTS int32), until the process exits. Nothing here calls cudaMalloc, cudaFree or any routine
// that allocates.
//
// Host code cannot use the array's name as a device address (it denotes a
// host-side shadow), so the device address is looked up once per device with
// cudaGetSymbolAddress and cached.
#include <climits>
#include <mutex>

#include "fp_device.cuh"

namespace fp {
namespace {

constexpr int32_t STATIC_MAX_VERTICES = 65536;
constexpr int64_t STATIC_MAX_FACES = 131072;
constexpr int STATIC_ROW_CAP = 256;          // raw entries of one row sorted on chip

// scratch layout, in ints
constexpr int64_t SV = STATIC_MAX_VERTICES + 1;
constexpr int64_t OFF_CNT = 0;                               // per-vertex raw counts
constexpr int64_t OFF_RAWOFF = OFF_CNT + SV;                 // raw row offsets (scan of counts)
constexpr int64_t OFF_FILL = OFF_RAWOFF + SV;                // fill cursors
constexpr int64_t OFF_UCNT = OFF_FILL + SV;                  // unique counts per row
constexpr int64_t OFF_STATUS = OFF_UCNT + SV;                // error flags
constexpr int64_t OFF_RAW = OFF_STATUS + 64;                 // raw rows: 6 entries per face
constexpr int64_t SCRATCH_INTS = OFF_RAW + 6 * STATIC_MAX_FACES;

enum : int32_t { SS_BAD_INDEX = 1, SS_ROW_TOO_LONG = 2, SS_COL_CAP = 4 };

static __device__ __align__(256) int32_t g_static_scratch[SCRATCH_INTS];

__global__ void ks_zero(int32_t* s, int32_t n) {
  FP_PDL_WAIT();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
    s[OFF_CNT + i] = 0;
    s[OFF_FILL + i] = 0;
    s[OFF_UCNT + i] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) s[OFF_STATUS] = 0;
}

__global__ void ks_count(const int32_t* __restrict__ faces, int64_t nf, int32_t n, int32_t* s) {
  FP_PDL_WAIT();
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c[3] = {faces[3 * f], faces[3 * f + 1], faces[3 * f + 2]};
    if (c[0] < 0 || c[0] >= n || c[1] < 0 || c[1] >= n || c[2] < 0 || c[2] >= n) {
      atomicOr(&s[OFF_STATUS], SS_BAD_INDEX);
      continue;
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int32_t a = c[e], b = c[(e + 1) % 3];
      if (a == b) continue;
      atomicAdd(&s[OFF_CNT + a], 1);
      atomicAdd(&s[OFF_CNT + b], 1);
    }
  }
}

// Exclusive scan of in[0..n) into out[0..n] by one CTA (n <= 65537).
__global__ void ks_scan(const int32_t* in, int32_t* out, int32_t n) {
  FP_PDL_WAIT();
  __shared__ int32_t red[40];
  int32_t carry = 0;
  for (int32_t base = 0; base < n; base += blockDim.x) {
    const int32_t i = base + threadIdx.x;
    const int32_t x = i < n ? in[i] : 0;
    int32_t tot;
    const int32_t ex = block_excl_scan_i32(x, &tot, red);
    if (i < n) out[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) out[n] = carry;
}

__global__ void ks_fill(const int32_t* __restrict__ faces, int64_t nf, int32_t n, int32_t* s) {
  FP_PDL_WAIT();
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c[3] = {faces[3 * f], faces[3 * f + 1], faces[3 * f + 2]};
    if (c[0] < 0 || c[0] >= n || c[1] < 0 || c[1] >= n || c[2] < 0 || c[2] >= n) continue;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int32_t a = c[e], b = c[(e + 1) % 3];
      if (a == b) continue;
      s[OFF_RAW + s[OFF_RAWOFF + a] + atomicAdd(&s[OFF_FILL + a], 1)] = b;
      s[OFF_RAW + s[OFF_RAWOFF + b] + atomicAdd(&s[OFF_FILL + b], 1)] = a;
    }
  }
}

// One warp per row: sort the raw row in shared memory, keep the unique prefix.
__global__ void __launch_bounds__(256) ks_dedupe(int32_t n, int32_t* s) {
  FP_PDL_WAIT();
  __shared__ int32_t sbuf[8][STATIC_ROW_CAP];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* buf = sbuf[wid];
  for (int32_t v = blockIdx.x * 8 + wid; v < n; v += gridDim.x * 8) {
    const int32_t b = s[OFF_RAWOFF + v], L = s[OFF_RAWOFF + v + 1] - b;
    if (L > STATIC_ROW_CAP) {
      if (lane == 0) atomicOr(&s[OFF_STATUS], SS_ROW_TOO_LONG);
      continue;
    }
    const int N = pow2_at_least(L, 32);
    for (int i = lane; i < N; i += 32) buf[i] = i < L ? s[OFF_RAW + b + i] : INT_MAX;
    __syncwarp();
    bitonic_sort<false>(buf, N, lane, 32);
    int32_t cnt = 0;
    for (int i0 = 0; i0 < L; i0 += 32) {
      const int i = i0 + lane;
      const bool keep = i < L && (i == 0 || buf[i] != buf[i - 1]);
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) s[OFF_RAW + b + cnt + __popc(m & lanemask_lt())] = buf[i];
      cnt += __popc(m);
    }
    if (lane == 0) s[OFF_UCNT + v] = cnt;
    __syncwarp();
  }
}

__global__ void ks_compact(int32_t n, const int32_t* s, const int32_t* __restrict__ rowptr, int32_t* __restrict__ col,
                           int64_t col_cap, int32_t* status) {
  FP_PDL_WAIT();
  const int lane = threadIdx.x & 31;
  for (int32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += (gridDim.x * blockDim.x) >> 5) {
    const int32_t src = s[OFF_RAWOFF + v], dst = rowptr[v], L = rowptr[v + 1] - dst;
    if ((int64_t)dst + L > col_cap) {
      if (lane == 0) atomicOr(status, SS_COL_CAP);
      continue;
    }
    for (int i = lane; i < L; i += 32) col[dst + i] = s[OFF_RAW + src + i];
  }
}

std::mutex g_static_mu;
int32_t* g_static_addr[128];

// Device address of the scratch array on `device` (current), looked up once.
fp_status static_scratch(int device, int32_t** out) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (device < 0 || device >= 128) return fail(nullptr, FP_ERR_CUDA, "device index out of range");
  if (!g_static_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(nullptr, FP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    g_static_addr[device] = (int32_t*)p;
  }
  *out = g_static_addr[device];
  return FP_OK;
}

}  // namespace
}  // namespace fp

using namespace fp;

extern "C" fp_status fp_graph_from_faces_static(const int32_t* d_faces, int64_t n_faces, int32_t n_vertices,
                                                int32_t* d_rowptr, int32_t* d_col, int64_t col_cap,
                                                int64_t* h_nnz, void* stream) {
  if (n_vertices < 0 || n_faces < 0 || (n_faces > 0 && !d_faces) || !d_rowptr || col_cap < 0 ||
      (col_cap > 0 && !d_col))
    return fail(nullptr, FP_ERR_INVALID_ARG, "bad sizes or NULL pointers");
  if (n_vertices > STATIC_MAX_VERTICES || n_faces > STATIC_MAX_FACES)
    return fail(nullptr, FP_ERR_UNSUPPORTED,
                "fp_graph_from_faces_static: at most 65536 vertices and 131072 faces (fixed scratch)");
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return fail(nullptr, FP_ERR_CUDA, cudaGetErrorString(e));
  int32_t* s = nullptr;
  FP_TRY(static_scratch(device, &s));
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = n_vertices;
  const int gz = (n + 256) / 256;
  ks_zero<<<gz < 296 ? gz : 296, 256, 0, st>>>(s, n);
  const int gf = (int)((n_faces + 255) / 256);
  if (n_faces > 0) ks_count<<<gf < 592 ? gf : 592, 256, 0, st>>>(d_faces, n_faces, n, s);
  ks_scan<<<1, 1024, 0, st>>>(s + OFF_CNT, s + OFF_RAWOFF, n);
  if (n_faces > 0) ks_fill<<<gf < 592 ? gf : 592, 256, 0, st>>>(d_faces, n_faces, n, s);
  const int gr = (n + 7) / 8;
  if (n > 0) ks_dedupe<<<gr < 1184 ? gr : 1184, 256, 0, st>>>(n, s);
  ks_scan<<<1, 1024, 0, st>>>(s + OFF_UCNT, d_rowptr, n);
  const int gc = (int)(((int64_t)n * 32 + 255) / 256);
  if (n > 0) ks_compact<<<gc < 1184 ? gc : 1184, 256, 0, st>>>(n, s, d_rowptr, d_col, col_cap, s + OFF_STATUS);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(nullptr, FP_ERR_CUDA, cudaGetErrorString(e));
  int32_t status = 0, nnz = 0;
  e = cudaMemcpyAsync(&status, s + OFF_STATUS, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nnz, d_rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(nullptr, FP_ERR_CUDA, cudaGetErrorString(e));
  if (status & SS_BAD_INDEX) return fail(nullptr, FP_ERR_INVALID_ARG, "face corner out of range");
  if (status & SS_ROW_TOO_LONG) return fail(nullptr, FP_ERR_UNSUPPORTED, "a vertex has more than 256 raw face-edges");
  if (status & SS_COL_CAP) return fail(nullptr, FP_ERR_INVALID_ARG, "col_cap smaller than the number of entries");
  if (h_nnz) *h_nnz = nnz;
  return FP_OK;
}
