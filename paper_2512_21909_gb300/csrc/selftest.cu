// selftest.cu -- exercise the bounded-wait error path without faulting.
//
// Every mbarrier wait in the tensor-core kernels spins a bounded number of
// times and then records an error code that the host turns into
// CDCC_ETIMEOUT.  This self-test runs one CTA whose thread 0 waits on a
// barrier phase that nothing ever completes (the barrier is initialised
// with one expected arrival that is never made), with the same bounded-spin
// loop; the wait therefore runs out, the kernel records the code and exits
// normally, and the context stays usable.
#include <cuda_runtime.h>

#include "../../include/cdcc.h"

namespace {

__global__ void bounded_wait_kernel(unsigned int* err, long long limit) {
  __shared__ uint64_t bar;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool done = false;
    for (long long i = 0; i < limit && !done; ++i) {
      uint32_t ok;
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ok)
          : "r"(a)
          : "memory");
      done = ok != 0;
    }
    if (!done) atomicExch(err, 99u);
  }
}

}  // namespace

extern "C" cdcc_status cdcc_selftest_bounded_wait(void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned int* d = nullptr;
  if (cudaMallocAsync((void**)&d, sizeof(unsigned int), st) != cudaSuccess)
    return CDCC_ENOMEM;
  unsigned int h = 0;
  cdcc_status s = CDCC_OK;
  if (cudaMemsetAsync(d, 0, sizeof(unsigned int), st) != cudaSuccess)
    s = CDCC_ECUDA;
  if (s == CDCC_OK) {
    bounded_wait_kernel<<<1, 32, 0, st>>>(d, 1LL << 16);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      s = CDCC_ECUDA;
  }
  cudaFreeAsync(d, st);
  cudaStreamSynchronize(st);
  if (s != CDCC_OK) return s;
  return h == 99u ? CDCC_ETIMEOUT : CDCC_OK;
}
