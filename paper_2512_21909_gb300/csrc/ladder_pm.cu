// ladder_pm.cu -- symmetric/antisymmetric (+/-) packing of the on-the-fly
// particle-particle ladder (Sec. 2.3).
//
// For amplitudes symmetric under the pair swap, X_{ij,cd} = X_{ji,dc}, the
// ladder Y_{ij,ab} = sum_cd X_{ij,cd} (ac|bd) only needs canonical pairs
// (p,q) of each index pair: irrep(p) > irrep(q), or the same irrep and
// p >= q.  With
//   A+-_{ij,cd} = (X_{ij,cd} + X_{ji,dc} +- (X_{ij,dc} + X_{ji,cd})) / 4
//   W+-_{ab,cd} = (ac|bd) +- (ad|bc)          (c != d)
//   W+_{ab,cc}  = (ac|bc),  W-_{ab,cc} = 0
//   S+-        = A+- W+-^T   (canonical ij rows, ab rows, cd columns)
// every ordered element follows from its canonical representative:
//   Y_{ij,ab} += S+ + s S-,  s = -1 when exactly one of (ij), (ab) is
// swapped against its representative.  Each product runs over half the
// pairs of all three index pairs: a quarter of the flops of the plain map,
// in two GEMMs.  A+- uses both (ij) and (ji), so for any X the result is the
// ladder of the pair-symmetrised amplitudes, which is the ladder of X
// itself when X is pair-symmetric (the amplitudes and the adjoints of the
// symmetrised residual are).
//
// Index tables (built once per layout on the host; offsets inside the DPD
// block of pair irrep G, rows (i,j) and columns (c,d) as the layout stores
// them):
//   orow[2][uo]: row offsets of (i,j) and (j,i) per canonical (ij)
//   vcol[2][uv]: column offsets of (c,d) and (d,c) per canonical (cd)
//   vrow[3][nv]: per canonical (ab) of a row batch: its row in the batch's
//                (ab|cd) rows, the columns of (a,b) and (b,a) in Y
//                (-1 for a == b in the same irrep)
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.h"

namespace cdcc {

namespace {

constexpr int PM_THREADS = 256;

__global__ void __launch_bounds__(PM_THREADS)
    pm_pack_x_kernel(const double* __restrict__ X, int64_t ncol,
                     const int* __restrict__ orow, int uo,
                     const int* __restrict__ vcol, int uv,
                     double* __restrict__ Ap, double* __restrict__ Am) {
  for (int r = blockIdx.y; r < uo; r += gridDim.y) {
    const double* x1 = X + (int64_t)orow[r] * ncol;
    const double* x2 = X + (int64_t)orow[uo + r] * ncol;
    for (int u = blockIdx.x * PM_THREADS + threadIdx.x; u < uv;
         u += gridDim.x * PM_THREADS) {
      const int c1 = vcol[u], c2 = vcol[uv + u];
      const double s = x1[c1] + x2[c2];
      const double t = x1[c2] + x2[c1];
      Ap[(int64_t)r * uv + u] = 0.25 * (s + t);
      Am[(int64_t)r * uv + u] = 0.25 * (s - t);
    }
  }
}

__global__ void __launch_bounds__(PM_THREADS)
    pm_pack_w_kernel(const double* __restrict__ W, int64_t ncol,
                     const int* __restrict__ vrow, int nv,
                     const int* __restrict__ vcol, int uv,
                     double* __restrict__ Wp, double* __restrict__ Wm) {
  for (int v = blockIdx.y; v < nv; v += gridDim.y) {
    const double* w = W + (int64_t)vrow[v] * ncol;
    for (int u = blockIdx.x * PM_THREADS + threadIdx.x; u < uv;
         u += gridDim.x * PM_THREADS) {
      const int c1 = vcol[u], c2 = vcol[uv + u];
      const double w1 = w[c1], w2 = w[c2];
      const bool diag = c1 == c2;
      Wp[(int64_t)v * uv + u] = diag ? w1 : w1 + w2;
      Wm[(int64_t)v * uv + u] = diag ? 0.0 : w1 - w2;
    }
  }
}

__global__ void __launch_bounds__(PM_THREADS)
    pm_unpack_kernel(const double* __restrict__ Sp,
                     const double* __restrict__ Sm, int uo, int nv,
                     const int* __restrict__ orow,
                     const int* __restrict__ vrow, double alpha,
                     double* __restrict__ Y, int64_t ncol) {
  for (int r = blockIdx.y; r < uo; r += gridDim.y) {
    const int r1 = orow[r], r2 = orow[uo + r];
    double* y1 = Y + (int64_t)r1 * ncol;
    double* y2 = Y + (int64_t)r2 * ncol;
    for (int v = blockIdx.x * PM_THREADS + threadIdx.x; v < nv;
         v += gridDim.x * PM_THREADS) {
      const double p = Sp[(int64_t)r * nv + v];
      const double m = Sm[(int64_t)r * nv + v];
      const int k1 = vrow[nv + v], k2 = vrow[2 * nv + v];
      y1[k1] += alpha * (p + m);
      if (k2 >= 0) y1[k2] += alpha * (p - m);
      if (r2 != r1) {
        y2[k1] += alpha * (p - m);
        if (k2 >= 0) y2[k2] += alpha * (p + m);
      }
    }
  }
}

dim3 pm_grid(int64_t inner, int64_t outer) {
  const int gx = (int)std::max<int64_t>(
      1, std::min<int64_t>((inner + PM_THREADS - 1) / PM_THREADS, 64));
  const int gy = (int)std::max<int64_t>(1, std::min<int64_t>(outer, 65535));
  return dim3(gx, gy);
}

}  // namespace

int pm_pack_x(const double* X, int64_t ncol, const int* orow, int uo,
              const int* vcol, int uv, double* Ap, double* Am,
              cudaStream_t st) {
  if (uo <= 0 || uv <= 0) return 0;
  pm_pack_x_kernel<<<pm_grid(uv, uo), PM_THREADS, 0, st>>>(
      X, ncol, orow, uo, vcol, uv, Ap, Am);
  return 1;
}

int pm_pack_w(const double* W, int64_t ncol, const int* vrow, int nv,
              const int* vcol, int uv, double* Wp, double* Wm,
              cudaStream_t st) {
  if (nv <= 0 || uv <= 0) return 0;
  pm_pack_w_kernel<<<pm_grid(uv, nv), PM_THREADS, 0, st>>>(
      W, ncol, vrow, nv, vcol, uv, Wp, Wm);
  return 1;
}

int pm_unpack(const double* Sp, const double* Sm, int uo, int nv,
              const int* orow, const int* vrow, double alpha, double* Y,
              int64_t ncol, cudaStream_t st) {
  if (uo <= 0 || nv <= 0) return 0;
  pm_unpack_kernel<<<pm_grid(nv, uo), PM_THREADS, 0, st>>>(
      Sp, Sm, uo, nv, orow, vrow, alpha, Y, ncol);
  return 1;
}

}  // namespace cdcc
