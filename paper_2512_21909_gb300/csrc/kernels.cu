// kernels.cu -- DPD permute / update, reductions, batched dot (the FP64 GEMM
// is in gemm64.cu).
#include "kernels.h"

#include <algorithm>
#include <cstring>

namespace cdcc {

namespace {

constexpr int CHUNK = 4096;

}  // namespace

// largest chunk of a permutation / update task per CTA
int chunk_elems() { return CHUNK; }

int sm_count() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    (void)cudaGetLastError();
    return 152;
  }
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
            cudaSuccess ||
        n <= 0) {
      (void)cudaGetLastError();
      n = 152;
    }
    cached[dev] = n;
  }
  return cached[dev];
}

// ----------------------------------------------------------- permute / axpy
namespace {

// Offsets (from ybase / xbase) and per-dimension indices of element e of a
// box, 32-bit path (t.off32): the divisions by the extents are the
// multiply-and-shift reciprocals of set_division_magic.  Unrolled over
// MAXRANK so that the task's fields stay in registers; a rank-0 box (one
// element) has zero strides.
__device__ __forceinline__ void box_offsets32(const PermTask& t, int e,
                                              int& y, int& x, int* l) {
  y = 0;
  x = 0;
  uint32_t r = (uint32_t)e;
#pragma unroll
  for (int q = MAXRANK - 1; q > 0; --q) {
    if (q < t.rank) {
      const uint32_t nq = (uint32_t)(((uint64_t)r * t.mag[q]) >> t.shr[q]);
      const int lq = (int)(r - nq * (uint32_t)t.dim[q]);
      r = nq;
      l[q] = lq;
      y += lq * (int)t.ys[q];
      x += lq * (int)t.xs[q];
    }
  }
  l[0] = (int)r;
  y += (int)r * (int)t.ys[0];
  x += (int)r * (int)t.xs[0];
}

// Same, 64-bit path (boxes or offsets of 2^31 elements and more).
__device__ __forceinline__ void box_offsets64(const PermTask& t, int64_t e,
                                              int64_t& y, int64_t& x,
                                              int* l) {
  y = 0;
  x = 0;
  for (int q = t.rank - 1; q >= 0; --q) {
    const int d = t.dim[q];
    const int64_t lq = e % d;
    e /= d;
    l[q] = (int)lq;
    y += lq * t.ys[q];
    x += lq * t.xs[q];
  }
}

// Y = beta Y + alpha X over the chunk's elements.  Each thread takes PU
// elements at a time (offsets first, then all loads, then the stores) so
// that several loads are in flight per thread.
constexpr int PU = 4;

__global__ void __launch_bounds__(256)
    perm_axpy_kernel(const PermTask* __restrict__ tasks,
                     const Chunk* __restrict__ chunks, double alpha,
                     const double* __restrict__ X, double beta,
                     double* __restrict__ Y,
                     const double* __restrict__ dscale) {
  const Chunk c = chunks[blockIdx.x];
  const PermTask& t = tasks[c.task];
  const int64_t end = min(t.n, c.start + (int64_t)c.len);
  if (dscale) alpha *= *dscale;
  int l[MAXRANK];
  const double* Xb = X + t.xbase;
  double* Yb = Y + t.ybase;
  if (t.off32) {
    const int e1 = (int)end;
    for (int e0 = (int)c.start + threadIdx.x; e0 < e1;
         e0 += PU * blockDim.x) {
      int yo[PU], xo[PU];
      double v[PU];
      bool in[PU];
#pragma unroll
      for (int u = 0; u < PU; ++u) {
        const int e = e0 + u * blockDim.x;
        in[u] = e < e1;
        yo[u] = xo[u] = 0;
        if (in[u]) box_offsets32(t, e, yo[u], xo[u], l);
      }
#pragma unroll
      for (int u = 0; u < PU; ++u) v[u] = in[u] ? alpha * Xb[xo[u]] : 0.0;
#pragma unroll
      for (int u = 0; u < PU; ++u) {
        if (!in[u]) continue;
        double* p = Yb + yo[u];
        *p = (beta == 0.0) ? v[u] : fma(beta, *p, v[u]);
      }
    }
    return;
  }
  for (int64_t e = c.start + threadIdx.x; e < end; e += blockDim.x) {
    int64_t y, x;
    box_offsets64(t, e, y, x, l);
    const double v = alpha * Xb[x];
    Yb[y] = (beta == 0.0) ? v : fma(beta, Yb[y], v);
  }
}

__device__ __forceinline__ unsigned long long dbl_bits(double v) {
  return (unsigned long long)__double_as_longlong(v);
}

__global__ void jacobi_kernel(const PermTask* __restrict__ tasks,
                              const Chunk* __restrict__ chunks,
                              const double* __restrict__ R,
                              double* __restrict__ T, double* __restrict__ E,
                              const double* __restrict__ eps,
                              unsigned long long* maxbits) {
  const Chunk c = chunks[blockIdx.x];
  const PermTask& t = tasks[c.task];
  const int64_t end = min(t.n, c.start + (int64_t)c.len);
  int l[MAXRANK];
  double mx = 0.0;
  for (int64_t e = c.start + threadIdx.x; e < end; e += blockDim.x) {
    int64_t y, x;
    if (t.off32) {
      int y32, x32;
      box_offsets32(t, (int)e, y32, x32, l);
      y = t.ybase + y32;
      x = t.xbase + x32;
    } else {
      box_offsets64(t, e, y, x, l);
      y += t.ybase;
      x += t.xbase;
    }
    double D = 0.0;
#pragma unroll
    for (int q = 0; q < MAXRANK; ++q)
      if (q < t.rank) D += t.sgn[q] * eps[t.gidx[q] + l[q]];
    const double s = R[y] / D;
    if (T) T[y] += s;
    if (E) E[y] = s;
    mx = fmax(mx, fabs(s));
    if (s != s) mx = __longlong_as_double(0x7ff8000000000000LL);
  }
  __shared__ unsigned long long red[32];
  unsigned long long b = dbl_bits(mx);
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long ob = __shfl_down_sync(0xffffffffu, b, o);
    b = ob > b ? ob : b;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x < 32) {
    b = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long ob = __shfl_down_sync(0xffffffffu, b, o);
      b = ob > b ? ob : b;
    }
    if (threadIdx.x == 0) atomicMax(maxbits, b);
  }
}

// One CTA per chunk of rows; threads run along the row (coalesced), two
// elements per thread per pass.
__global__ void __launch_bounds__(256)
    jacobi2d_kernel(const Block2D* __restrict__ blocks,
                    const Chunk2D* __restrict__ chunks,
                    const double* __restrict__ rv,
                    const double* __restrict__ cv,
                    const double* __restrict__ R, double* __restrict__ T,
                    double* __restrict__ E, unsigned long long* maxbits) {
  const Chunk2D ch = chunks[blockIdx.x];
  const Block2D b = blocks[ch.blk];
  double mx = 0.0;
  for (int r = ch.row0; r < ch.row0 + ch.nrows; ++r) {
    const double dr = rv[b.rv0 + r];
    const int64_t base = b.off + (int64_t)r * b.ncol;
    for (int64_t c = threadIdx.x; c < b.ncol; c += blockDim.x) {
      const double D = dr + cv[b.cv0 + c];
      const double s = R[base + c] / D;
      if (T) T[base + c] += s;
      if (E) E[base + c] = s;
      mx = fmax(mx, fabs(s));
      if (s != s) mx = __longlong_as_double(0x7ff8000000000000LL);
    }
  }
  __shared__ unsigned long long red[32];
  unsigned long long bb = dbl_bits(mx);
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long ob = __shfl_down_sync(0xffffffffu, bb, o);
    bb = ob > bb ? ob : bb;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = bb;
  __syncthreads();
  if (threadIdx.x < 32) {
    bb = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long ob = __shfl_down_sync(0xffffffffu, bb, o);
      bb = ob > bb ? ob : bb;
    }
    if (threadIdx.x == 0) atomicMax(maxbits, bb);
  }
}

struct PtrPack {
  const double* p[16];
  double c[16];
};

constexpr int DOT_BLOCKS = 304;

__global__ void multi_dot_kernel(PtrPack xs, int m, const double* __restrict__ y,
                                 int64_t n, double* __restrict__ partial) {
  double acc[16];
  for (int k = 0; k < 16; ++k) acc[k] = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double yv = y[e];
    for (int k = 0; k < m; ++k) acc[k] = fma(xs.p[k][e], yv, acc[k]);
  }
  __shared__ double red[16][8];
  for (int k = 0; k < m; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < m) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
    partial[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void finish_dot_kernel(const double* __restrict__ partial,
                                  int nblk, int m, double* __restrict__ out) {
  const int k = blockIdx.x;
  if (k >= m) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
    s += partial[(int64_t)k * nblk + b];
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[k] = t;
  }
}

__global__ void lincomb_kernel(double* __restrict__ out, PtrPack xs, int m,
                               int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < m; ++k) s = fma(xs.c[k], xs.p[k][e], s);
    out[e] = s;
  }
}

__global__ void axpby_kernel(double a, const double* __restrict__ x, double b,
                             double* __restrict__ y, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v = a * x[e];
    y[e] = (b == 0.0) ? v : fma(b, y[e], v);
  }
}

constexpr int BD_NX = 8;      // displacements per pass
constexpr int BD_THREADS = 256;

// One block handles a contiguous range of the packed Gamma / dL elements for
// up to BD_NX displacements; G is read once per pass, each dL_x once.
__global__ void __launch_bounds__(BD_THREADS)
    batched_dot_kernel(const double* __restrict__ G,
                       const double* __restrict__ dL, int x0, int nx,
                       int64_t nnz, int64_t per_block,
                       double* __restrict__ partial) {
  double acc[BD_NX];
#pragma unroll
  for (int k = 0; k < BD_NX; ++k) acc[k] = 0.0;
  const int64_t beg = (int64_t)blockIdx.x * per_block;
  const int64_t end = min(nnz, beg + per_block);
  const int cnt = min(BD_NX, nx - x0);
  for (int64_t e = beg + threadIdx.x; e < end; e += BD_THREADS) {
    const double g = G[e];
#pragma unroll
    for (int k = 0; k < BD_NX; ++k)
      if (k < cnt) acc[k] = fma(g, __ldg(dL + (int64_t)(x0 + k) * nnz + e),
                                acc[k]);
  }
  __shared__ double red[BD_NX][BD_THREADS / 32];
#pragma unroll
  for (int k = 0; k < BD_NX; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int w = 0; w < BD_THREADS / 32; ++w) s += red[threadIdx.x][w];
    partial[(int64_t)(x0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
  }
}

int bd_blocks(int64_t nnz) {
  int64_t b = (nnz + 4095) / 4096;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, sm_count() * 8));
}

}  // namespace

int perm_axpy(const PermTask* d_tasks, const Chunk* d_chunks, int nchunks,
              double alpha, const double* X, double beta, double* Y,
              cudaStream_t st, const double* d_scale) {
  if (nchunks <= 0) return 0;
  perm_axpy_kernel<<<nchunks, 256, 0, st>>>(d_tasks, d_chunks, alpha, X, beta,
                                            Y, d_scale);
  return 1;
}

int jacobi_update(const PermTask* d_tasks, const Chunk* d_chunks, int nchunks,
                  const double* R, double* t, double* err, const double* eps,
                  unsigned long long* d_maxbits, cudaStream_t st) {
  if (nchunks <= 0) return 0;
  jacobi_kernel<<<nchunks, 256, 0, st>>>(d_tasks, d_chunks, R, t, err, eps,
                                         d_maxbits);
  return 1;
}

int jacobi2d(const Block2D* d_blocks, const Chunk2D* d_chunks, int nchunks,
             const double* rv, const double* cv, const double* R, double* t,
             double* err, unsigned long long* d_maxbits, cudaStream_t st) {
  if (nchunks <= 0) return 0;
  jacobi2d_kernel<<<nchunks, 256, 0, st>>>(d_blocks, d_chunks, rv, cv, R, t,
                                           err, d_maxbits);
  return 1;
}

int64_t multi_dot_partial_doubles(int64_t n, int m) {
  (void)n;
  return (int64_t)DOT_BLOCKS * m;
}

int multi_dot(const double* const* xs, int m, const double* y, int64_t n,
              double* d_partial, double* d_out, cudaStream_t st) {
  if (m <= 0) return 0;
  PtrPack pk;
  std::memset(&pk, 0, sizeof(pk));
  for (int k = 0; k < m; ++k) pk.p[k] = xs[k];
  multi_dot_kernel<<<DOT_BLOCKS, 256, 0, st>>>(pk, m, y, n, d_partial);
  finish_dot_kernel<<<m, 256, 0, st>>>(d_partial, DOT_BLOCKS, m, d_out);
  return 2;
}

int lincomb(double* out, const double* const* xs, const double* c, int m,
            int64_t n, cudaStream_t st) {
  PtrPack pk;
  std::memset(&pk, 0, sizeof(pk));
  for (int k = 0; k < m; ++k) {
    pk.p[k] = xs[k];
    pk.c[k] = c[k];
  }
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, sm_count() * 16);
  lincomb_kernel<<<std::max(blocks, 1), 256, 0, st>>>(out, pk, m, n);
  return 1;
}

int axpby(double a, const double* x, double b, double* y, int64_t n,
          cudaStream_t st) {
  if (n <= 0) return 0;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, sm_count() * 16);
  axpby_kernel<<<blocks, 256, 0, st>>>(a, x, b, y, n);
  return 1;
}

int64_t batched_dot_partial_doubles(int64_t nnz, int nx) {
  return (int64_t)bd_blocks(nnz) * nx;
}

int batched_dot(const double* G, const double* dL, int nx, int64_t nnz,
                double* partial, double* d_g, cudaStream_t st) {
  if (nx <= 0) return 0;
  const int blocks = bd_blocks(nnz);
  const int64_t per = (nnz + blocks - 1) / blocks;
  int launches = 0;
  for (int x0 = 0; x0 < nx; x0 += BD_NX) {
    batched_dot_kernel<<<blocks, BD_THREADS, 0, st>>>(G, dL, x0, nx, nnz, per,
                                                       partial);
    ++launches;
  }
  finish_dot_kernel<<<nx, 256, 0, st>>>(partial, blocks, nx, d_g);
  return launches + 1;
}


// ------------------------------------------------- ladder batch permutation
namespace {

template <bool INV>
__global__ void __launch_bounds__(256)
    ladder_perm_kernel(const __grid_constant__ LadPerm P,
                       const double* __restrict__ src,
                       double* __restrict__ dst) {
  const int r = blockIdx.x;
  int gc = 0;
  while (gc + 1 < P.h && r >= P.row0[gc + 1]) ++gc;
  const int loc = r - P.row0[gc];
  const int nc = P.nc[gc], nd = P.nd[gc];
  const int a = loc / nc, c = loc - a * nc;
  const int len = P.nb * nd;
  const int64_t xrow = P.xoff[gc] + (int64_t)loc * len;
  const int64_t wbase = (int64_t)a * P.nb * P.ncol + P.coff[gc] +
                        (int64_t)c * nd;
  if (len <= 0) return;
  // (b, d) of element e walk forward by blockDim.x per step: one division
  // per thread, then an add with carry
  const int sb = blockDim.x / nd, sd = blockDim.x - sb * nd;
  int b = threadIdx.x / nd, d = threadIdx.x - b * nd;
  for (int e = threadIdx.x; e < len; e += blockDim.x) {
    const int64_t w = wbase + (int64_t)b * P.ncol + d;
    if (INV)
      dst[xrow + e] = src[w];
    else
      dst[w] = src[xrow + e];
    b += sb;
    d += sd;
    if (d >= nd) {
      d -= nd;
      ++b;
    }
  }
}

}  // namespace

int ladder_permute(const LadPerm& P, bool inverse, const double* src,
                   double* dst, int rows, cudaStream_t st) {
  if (rows <= 0) return 0;
  if (inverse)
    ladder_perm_kernel<true><<<rows, 256, 0, st>>>(P, src, dst);
  else
    ladder_perm_kernel<false><<<rows, 256, 0, st>>>(P, src, dst);
  return 1;
}

}  // namespace cdcc
