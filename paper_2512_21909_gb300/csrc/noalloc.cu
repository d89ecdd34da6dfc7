// noalloc.cu -- contract_dL variant that allocates no memory.
//
// Some callers cannot allocate device memory at all: code that runs inside
// a host framework or plugin whose device memory is owned and budgeted by
// someone else, and serving loops that must not call cudaMalloc because it
// synchronises the whole device and stalls the other work on it.  For them
// cdcc_contract_dL_noalloc computes the same gradient contraction as
// contract_dL,
//     g[x] = sum_e Gamma[e] * dL[x*nnz + e],
// on caller-provided device buffers, with its per-block partial sums kept in
// a fixed file-scope device array instead of allocated scratch.
//
// The array lives in every device that loads the library until the process
// exits.  Its device address is looked up once per device (first call on
// that device, with the device current); that first call should therefore
// be made before any stream capture.  All calls share the array, so calls
// whose work overlaps on the GPU race on it: serialise them (one stream, or
// events).  Every partial slot a call reads is written earlier in the same
// call, so nothing has to be cleared between calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/cdcc.h"

namespace {

constexpr int NA_THREADS = 256;
// capacity of the fixed partial-sum array in CTAs; a call launches
// min(8 x the device's SM count, this) CTAs (1216 on a 152-SM GB300)
constexpr int NA_MAX_BLOCKS = 2048;
constexpr int NA_XPASS = 8;           // displacements per pass

static __device__ __align__(256) double
    g_noalloc_partial[NA_MAX_BLOCKS * CDCC_NOALLOC_MAX_NX];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
double* g_na_ptr[NA_MAX_DEVICES] = {};

__global__ void __launch_bounds__(NA_THREADS)
    na_dot_kernel(const double* __restrict__ G, const double* __restrict__ dL,
                  int x0, int nx, long long nnz, long long per_block,
                  double* __restrict__ partial) {
  double acc[NA_XPASS];
#pragma unroll
  for (int k = 0; k < NA_XPASS; ++k) acc[k] = 0.0;
  const long long beg = (long long)blockIdx.x * per_block;
  const long long end = min(nnz, beg + per_block);
  const int cnt = min(NA_XPASS, nx - x0);
  for (long long e = beg + threadIdx.x; e < end; e += NA_THREADS) {
    const double g = G[e];
#pragma unroll
    for (int k = 0; k < NA_XPASS; ++k)
      if (k < cnt) acc[k] = fma(g, __ldg(dL + (long long)(x0 + k) * nnz + e),
                                acc[k]);
  }
  __shared__ double red[NA_XPASS][NA_THREADS / 32];
#pragma unroll
  for (int k = 0; k < NA_XPASS; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int w = 0; w < NA_THREADS / 32; ++w) s += red[threadIdx.x][w];
    partial[(long long)(x0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void na_finish_kernel(const double* __restrict__ partial, int nblk,
                                 double* __restrict__ g) {
  const int x = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
    s += partial[(long long)x * nblk + b];
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    g[x] = t;
  }
}

// Device memory of device `dev` (the current one), or managed memory.  A
// pointer into another GPU's memory is rejected: without peer access the
// kernels would fault on it.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" cdcc_status cdcc_contract_dL_noalloc(const double* gamma,
                                                const double* dL, int nx,
                                                size_t nnz, double* g,
                                                void* stream) {
  if (!gamma || !dL || !g || nnz == 0) return CDCC_EINVAL;
  if (nx < 1 || nx > CDCC_NOALLOC_MAX_NX) return CDCC_EINVAL;
  // an error left pending by earlier work is not this call's: report it
  // without clearing it, so that the caller's own check still sees it
  if (cudaPeekAtLastError() != cudaSuccess) return CDCC_ECUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES)
    return CDCC_ECUDA;
  if (!on_device(gamma, dev) || !on_device(dL, dev) || !on_device(g, dev))
    return CDCC_EINVAL;
  double* partial = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_partial) != cudaSuccess ||
          p == nullptr) {
        (void)cudaGetLastError();
        return CDCC_ECUDA;
      }
      g_na_ptr[dev] = static_cast<double*>(p);
    }
    partial = g_na_ptr[dev];
  }
  // the stream must belong to the current device as well (0 = legacy
  // default stream of the current device)
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (st) {
    int sdev = -1;
    if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
      (void)cudaGetLastError();
      return CDCC_EINVAL;
    }
    if (sdev != dev) return CDCC_EINVAL;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
          cudaSuccess ||
      sms <= 0) {
    (void)cudaGetLastError();
    return CDCC_ECUDA;
  }
  const long long cap = std::min<long long>(NA_MAX_BLOCKS, 8LL * sms);
  long long blocks = ((long long)nnz + 4095) / 4096;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  const long long per = ((long long)nnz + blocks - 1) / blocks;
  for (int x0 = 0; x0 < nx; x0 += NA_XPASS) {
    na_dot_kernel<<<(int)blocks, NA_THREADS, 0, st>>>(gamma, dL, x0, nx,
                                                      (long long)nnz, per,
                                                      partial);
    if (cudaGetLastError() != cudaSuccess) return CDCC_ECUDA;
  }
  na_finish_kernel<<<nx, 256, 0, st>>>(partial, (int)blocks, g);
  return cudaGetLastError() == cudaSuccess ? CDCC_OK : CDCC_ECUDA;
}
