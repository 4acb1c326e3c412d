// Allocation-free Euclidean norm of a device vector: rsc_norm2_noalloc.
//
// Same two-pass reduction as rsc_norm2 (block partial sums of squares, then
// one block that adds them up), but the partial sums live in a file-scope
// device array instead of a library-allocated buffer, and no context is
// needed.  The call allocates nothing: no cudaMalloc, cudaFree or allocating
// library routine.  Every GPU that loads this library holds the array
// (kMaxBlocks doubles = 16 KiB) until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "rsc.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr long kChunk = (long)kThreads * kPerThread;  // elements per block
constexpr int kMaxBlocks = RSC_NORM2_NOALLOC_MAX_N / (kThreads * kPerThread);
constexpr int kMaxDevices = 64;
static_assert((long)kMaxBlocks * kChunk == RSC_NORM2_NOALLOC_MAX_N, "size bound");

// Scratch shared by every call on a device: one partial sum per block.  Each
// call overwrites the first ceil(n / kChunk) entries before it reads them.
static __device__ __align__(256) double g_partials[kMaxBlocks];

__global__ void k_sumsq_partials(const double* __restrict__ v, long n,
                                 double* __restrict__ partials) {
  __shared__ double red[kThreads / 32];
  const long base = (long)blockIdx.x * kChunk;
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kPerThread; ++q) {
    const long i = base + (long)q * kThreads + threadIdx.x;
    if (i < n) s = fma(v[i], v[i], s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < kThreads / 32) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
  }
}

__global__ void k_sumsq_finish(const double* __restrict__ partials, int nblk,
                               double* __restrict__ out) {
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += kThreads) s += partials[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < kThreads / 32) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[0] = sqrt(s);
  }
}

// Device address of g_partials, looked up once per device (with that device
// current) on the first call made on it.  In host code the symbol itself is
// only a host-side stand-in and must never be passed to a kernel.
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

}  // namespace

extern "C" rsc_status rsc_norm2_noalloc(const double* v, size_t n, double* out, void* stream) {
  if (!v || !out) return RSC_EINVAL;
  if (n > (size_t)RSC_NORM2_NOALLOC_MAX_N) return RSC_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RSC_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return RSC_EINVAL;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess) return RSC_ECUDA;
      g_addr[dev] = static_cast<double*>(p);
    }
    scratch = g_addr[dev];
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int nblk = (int)((n + kChunk - 1) / kChunk);
  // Each launch is checked through its own return code: cudaGetLastError would also
  // return (and clear) an error that unrelated code left pending on this thread.
  long nl = (long)n;
  if (nblk > 0) {
    void* args1[] = {(void*)&v, (void*)&nl, (void*)&scratch};
    if (cudaLaunchKernel((const void*)k_sumsq_partials, dim3(nblk), dim3(kThreads), args1, 0, s) !=
        cudaSuccess)
      return RSC_ECUDA;
  }
  int nb = nblk;
  void* args2[] = {(void*)&scratch, (void*)&nb, (void*)&out};
  if (cudaLaunchKernel((const void*)k_sumsq_finish, dim3(1), dim3(kThreads), args2, 0, s) !=
      cudaSuccess)
    return RSC_ECUDA;
  return RSC_OK;
}
