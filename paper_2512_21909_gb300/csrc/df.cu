// df.cu -- metric factorisation for the density-fitting / Cholesky
// three-term gradient (Sec. 2.1 Eqs. dfcd and cv_2ndstep, Sec. 2.6 Eq.
// 2el_grad_cont).
//
// The metric M_PQ = (P|Q) is block diagonal by the irrep of the Cholesky
// vectors (Sec. 3.1); its blocks are small (a few hundred rows), so each is
// factorised by one CTA in FP64: first M = K K^T (Cholesky, in place), then
// the transposed inverse K^{-T}, which turns the Cholesky-basis density and
// vectors into the transformed quantities of Eq. eri_cddf_der through one
// grouped contraction each.
#include <cuda_runtime.h>

#include "kernels.h"

namespace cdcc {

namespace {

constexpr int DF_THREADS = 256;

// Left-looking Cholesky of block b in place (lower factor; the upper
// triangle is zeroed).  A pivot <= 0 (not positive definite) sets *err.
__global__ void __launch_bounds__(DF_THREADS)
    chol_blocks_kernel(double* __restrict__ A, const __grid_constant__ MetricBlocks B,
                       unsigned int* err) {
  const int b = blockIdx.x;
  const int n = B.n[b];
  double* M = A + B.off[b];
  __shared__ double red[DF_THREADS / 32];
  __shared__ double diag;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int k = t; k < j; k += DF_THREADS) {
      const double v = M[(int64_t)j * n + k];
      s = fma(v, v, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (t == 0) {
      double tot = 0.0;
      for (int w = 0; w < DF_THREADS / 32; ++w) tot += red[w];
      const double dd = M[(int64_t)j * n + j] - tot;
      double d = 1.0;
      if (dd > 0.0)
        d = sqrt(dd);
      else
        atomicExch(err, 1u);
      M[(int64_t)j * n + j] = d;
      diag = d;
    }
    __syncthreads();
    const double dj = diag;
    for (int i = j + 1 + t; i < n; i += DF_THREADS) {
      double v = M[(int64_t)i * n + j];
      for (int k = 0; k < j; ++k)
        v = fma(-M[(int64_t)i * n + k], M[(int64_t)j * n + k], v);
      M[(int64_t)i * n + j] = v / dj;
    }
    __syncthreads();
  }
  for (int64_t e = t; e < (int64_t)n * n; e += DF_THREADS) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (j > i) M[e] = 0.0;
  }
}

// KinvT = (K^{-1})^T for lower-triangular K, block by block: thread c
// solves K x = e_c by forward substitution and stores x as row c.
__global__ void __launch_bounds__(DF_THREADS)
    trinv_t_kernel(const double* __restrict__ K, double* __restrict__ Kt,
                   const __grid_constant__ MetricBlocks B) {
  const int b = blockIdx.x;
  const int n = B.n[b];
  const double* L = K + B.off[b];
  double* X = Kt + B.off[b];
  for (int c = threadIdx.x; c < n; c += DF_THREADS) {
    double* x = X + (int64_t)c * n;
    for (int i = 0; i < c; ++i) x[i] = 0.0;
    x[c] = 1.0 / L[(int64_t)c * n + c];
    for (int i = c + 1; i < n; ++i) {
      double s = 0.0;
      for (int k = c; k < i; ++k) s = fma(L[(int64_t)i * n + k], x[k], s);
      x[i] = -s / L[(int64_t)i * n + i];
    }
  }
}

}  // namespace

int metric_factor(double* M, double* KinvT, const MetricBlocks& B,
                  unsigned int* d_err, cudaStream_t st) {
  if (B.nblk <= 0) return 0;
  chol_blocks_kernel<<<B.nblk, DF_THREADS, 0, st>>>(M, B, d_err);
  trinv_t_kernel<<<B.nblk, DF_THREADS, 0, st>>>(M, KinvT, B);
  return 2;
}

}  // namespace cdcc
