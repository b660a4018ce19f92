// Modularity of a membership without any allocation by the library.
//
// Some callers cannot let a library allocate device memory: applications
// that hand the whole device to their own pool allocator (a serving process
// with a fixed memory budget), or code that must not call cudaMalloc while
// it runs.  louvain_modularity_of allocates its scratch (one int64 community
// weight per vertex and a few counters) on every call; this variant keeps
// the scratch in a fixed array that lives in the library's device image
// instead, so a call allocates nothing.  The caller passes the graph and the
// membership in device memory and receives the scalars on the host.
//
// The array, kNoAllocMaxVertices community weights plus five counters
// (8 MiB + 40 bytes), is part of the library: every GPU that loads it holds
// the array until the process exits.  All calls share it, so calls that
// overlap on the GPU (other threads, other streams) race and give wrong
// results; serialise them.  Each call clears the part it uses first.  The
// first call on a device is its set-up: it loads the library's device code
// there, which reserves the array; make it before the caller's own pool
// claims the device's memory.  Every call looks the array's device address
// up again (cudaGetSymbolAddress, which allocates nothing once the code is
// loaded), so no address outlives a reset of the device.
//
// The CSR is the caller's and is read without a prior validation pass, so
// the kernel checks every row before it reads the row's entries:
// 0 <= offsets[i] <= offsets[i+1] <= nnz, and offsets[0] = 0, offsets[n] =
// nnz are read back first (two 8-byte copies into a host array).
#include <cstdio>

#include "../../include/louvain.h"
#include "internal.h"

namespace lv {
namespace {

constexpr int64_t kNoAllocMaxVertices = 1 << 20;
constexpr int kNoAllocCounters = 4;  // internal weight, 2m, sum Sigma^2 low / high halves, error
constexpr int64_t kNoAllocWords = kNoAllocCounters + 1 + kNoAllocMaxVertices;

// Layout: [0] internal weight S_in, [1] total weight 2m, [2] low halves of
// Sigma_c^2, [3] high halves, [4] error flag, [5 ...] Sigma_c per community.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocWords];

__global__ void k_na_clear(unsigned long long *scr, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n + kNoAllocCounters + 1;
       i += (int64_t)gridDim.x * blockDim.x)
    scr[i] = 0;
}

// Warp per vertex: S_in (entries inside the vertex's community, self-loops
// once), 2m, and K_i added into Sigma of its community.  A row outside
// [0, nnz) or with decreasing offsets, an id out of range or a non-positive
// weight sets the error flag, and nothing of that row or entry is read
// further or counted.
__global__ void k_na_rows(int64_t n, int64_t nnz, const int64_t *off, const int32_t *col, const int32_t *w,
                          const int32_t *memb, unsigned long long *scr) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  unsigned long long sin = 0, tot = 0, bad = 0;
  for (int64_t i = warp; i < n; i += nw) {
    const int32_t ci = memb[i];
    const int64_t rb = off[i], re = off[i + 1];
    if (ci < 0 || ci >= n || rb < 0 || rb > re || re > nnz) {
      bad = 1;
      continue;
    }
    unsigned long long in = 0, k = 0;
    for (int64_t e = rb + lane; e < re; e += 32) {
      const int32_t j = col[e];
      const int32_t wi = w ? w[e] : 1;
      if (wi <= 0 || j < 0 || j >= n) {
        bad = 1;
        continue;
      }
      const unsigned long long we = (unsigned long long)wi;
      k += we;
      if (memb[j] == ci) in += we;
    }
    in = warp_sum_u(in);
    k = warp_sum_u(k);
    if (lane == 0 && k) atomicAdd(scr + kNoAllocCounters + 1 + ci, k);
    sin += in;
    tot += k;
  }
  if (lane == 0) {
    if (sin) atomicAdd(scr + 0, sin);
    if (tot) atomicAdd(scr + 1, tot);
  }
  if (bad) scr[4] = 1;
}

__global__ void k_na_sigma_sq(int64_t n, unsigned long long *scr) {
  unsigned long long lo = 0, hi = 0;
  const unsigned long long *sig = scr + kNoAllocCounters + 1;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long sq = sig[c] * sig[c];  // valid while 2m < 2^32 (checked by the host)
    lo += sq & 0xFFFFFFFFull;
    hi += sq >> 32;
  }
  lo = warp_sum_u(lo);
  hi = warp_sum_u(hi);
  if ((threadIdx.x & 31) == 0) {
    if (lo) atomicAdd(scr + 2, lo);
    if (hi) atomicAdd(scr + 3, hi);
  }
}

// Device address of the scratch array on the current device, looked up on
// every call.
cudaError_t scratch_for_current_device(unsigned long long **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = (unsigned long long *)p;
  return cudaSuccess;
}

}  // namespace
}  // namespace lv

using namespace lv;

extern "C" louvain_status louvain_modularity_noalloc(const louvain_graph *graph, const int32_t *membership,
                                                     void *stream, double *q, int64_t *num_hi_lo,
                                                     int64_t *den_hi_lo) {
  if (!graph || !membership || !graph->on_device || graph->n < 0 || (graph->n > 0 && !graph->offsets) ||
      (graph->nnz > 0 && !graph->cols))
    return LOUVAIN_E_INVAL;
  if (graph->n > kNoAllocMaxVertices) return LOUVAIN_E_INVAL;  // beyond the fixed scratch array
  if (graph->nnz < 0 || (graph->n == 0 && graph->nnz != 0)) return LOUVAIN_E_INVAL;
  const int64_t n = graph->n;
  cudaStream_t s = (cudaStream_t)stream;
  typedef __int128 i128;
  i128 num = 0, den = 0;
  if (n > 0) {
    unsigned long long *scr = nullptr;
    if (scratch_for_current_device(&scr) != cudaSuccess) return LOUVAIN_E_CUDA;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      return LOUVAIN_E_CUDA;
    // offsets[0] = 0 and offsets[n] = nnz (the kernel checks every row
    // against [0, nnz) before it reads the row's entries)
    int64_t ends[2] = {-1, -1};
    if (cudaMemcpyAsync(&ends[0], graph->offsets, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&ends[1], graph->offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return LOUVAIN_E_CUDA;
    if (ends[0] != 0 || ends[1] != graph->nnz) return LOUVAIN_E_INVAL;
    k_na_clear<<<grid_for(n + kNoAllocCounters + 1, 256, sms, 8), 256, 0, s>>>(scr, n);
    k_na_rows<<<grid_for(n * 32, 256, sms, 16), 256, 0, s>>>(n, graph->nnz, graph->offsets, graph->cols,
                                                             graph->weights, membership, scr);
    k_na_sigma_sq<<<grid_for(n, 256, sms, 8), 256, 0, s>>>(n, scr);
    unsigned long long h[kNoAllocCounters + 1];
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h, scr, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return LOUVAIN_E_CUDA;
    if (h[4]) return LOUVAIN_E_INVAL;                   // a bad row, id or weight
    if (h[1] >= (1ull << 32)) return LOUVAIN_E_OVERFLOW;  // 2m too large for the squares
    const i128 two_m = (i128)h[1];
    num = two_m * (i128)h[0] - (((i128)h[3] << 32) + (i128)h[2]);
    den = two_m * two_m;
  }
  if (q) *q = den ? (double)num / (double)den : 0.0;
  if (num_hi_lo) {
    num_hi_lo[0] = (int64_t)(num >> 64);
    num_hi_lo[1] = (int64_t)(uint64_t)num;
  }
  if (den_hi_lo) {
    den_hi_lo[0] = (int64_t)(den >> 64);
    den_hi_lo[1] = (int64_t)(uint64_t)den;
  }
  return LOUVAIN_OK;
}
