// kernels.cu -- FP64 grouped GEMM, DPD permute / update, reductions.
//
// The FP64 GEMM is a plain DFMA SIMT kernel (64x64x16 tiles, 256 threads,
// 4x4 outputs per thread, shared-memory staging, register double buffering).
// All irrep blocks of one contraction go through one grouped launch; thin
// products (few output tiles, long K) are split along K with a deterministic
// second-pass reduction.
#include "kernels.h"

#include <algorithm>
#include <cstring>

namespace cdcc {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
constexpr int CHUNK = 4096;

struct GemmLaunch {
  GemmProb p[GEMM_MAXPROB];
  int tile0[GEMM_MAXPROB + 1];
  int tm[GEMM_MAXPROB], tn[GEMM_MAXPROB], ks[GEMM_MAXPROB];
  int64_t poff[GEMM_MAXPROB];
  int np;
  double alpha, beta;
  double* scratch;
};

__device__ __forceinline__ void load_tile_a(const GemmProb& P, int m0, int k0,
                                            int kend, double (&ra)[4]) {
  const int t = threadIdx.x;
  if (!P.ta) {
    const int c = t & 15;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = (t >> 4) + 16 * i;
      const int m = m0 + r, k = k0 + c;
      ra[i] = (m < P.M && k < kend) ? P.A[(int64_t)m * P.lda + k] : 0.0;
    }
  } else {
    const int c = t & 63;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = (t >> 6) + 4 * i;
      const int m = m0 + c, k = k0 + r;
      ra[i] = (m < P.M && k < kend) ? P.A[(int64_t)k * P.lda + m] : 0.0;
    }
  }
}

__device__ __forceinline__ void store_tile_a(const GemmProb& P,
                                             double (*As)[BM + 1],
                                             const double (&ra)[4]) {
  const int t = threadIdx.x;
  if (!P.ta) {
    const int c = t & 15;
#pragma unroll
    for (int i = 0; i < 4; ++i) As[c][(t >> 4) + 16 * i] = ra[i];
  } else {
    const int c = t & 63;
#pragma unroll
    for (int i = 0; i < 4; ++i) As[(t >> 6) + 4 * i][c] = ra[i];
  }
}

__device__ __forceinline__ void load_tile_b(const GemmProb& P, int n0, int k0,
                                            int kend, double (&rb)[4]) {
  const int t = threadIdx.x;
  if (!P.tb) {
    const int c = t & 63;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = (t >> 6) + 4 * i;
      const int n = n0 + c, k = k0 + r;
      rb[i] = (n < P.N && k < kend) ? P.B[(int64_t)k * P.ldb + n] : 0.0;
    }
  } else {
    const int c = t & 15;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = (t >> 4) + 16 * i;
      const int n = n0 + r, k = k0 + c;
      rb[i] = (n < P.N && k < kend) ? P.B[(int64_t)n * P.ldb + k] : 0.0;
    }
  }
}

__device__ __forceinline__ void store_tile_b(const GemmProb& P,
                                             double (*Bs)[BN + 1],
                                             const double (&rb)[4]) {
  const int t = threadIdx.x;
  if (!P.tb) {
    const int c = t & 63;
#pragma unroll
    for (int i = 0; i < 4; ++i) Bs[(t >> 6) + 4 * i][c] = rb[i];
  } else {
    const int c = t & 15;
#pragma unroll
    for (int i = 0; i < 4; ++i) Bs[c][(t >> 4) + 16 * i] = rb[i];
  }
}

__global__ void __launch_bounds__(NT)
    gemm64_kernel(const __grid_constant__ GemmLaunch L) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int bid = blockIdx.x;
  int pi = 0;
  while (pi + 1 < L.np && bid >= L.tile0[pi + 1]) ++pi;
  const GemmProb& P = L.p[pi];
  int local = bid - L.tile0[pi];
  const int ksn = L.ks[pi];
  const int ks = local % ksn;
  local /= ksn;
  const int tn = local % L.tn[pi];
  const int tm = local / L.tn[pi];
  const int m0 = tm * BM, n0 = tn * BN;
  int kper = (P.K + ksn - 1) / ksn;
  kper = (kper + BK - 1) / BK * BK;
  const int kbeg = ks * kper;
  const int kend = min(P.K, kbeg + kper);

  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  double ra[4], rb[4];
  if (kbeg < kend) {
    load_tile_a(P, m0, kbeg, kend, ra);
    load_tile_b(P, n0, kbeg, kend, rb);
  }
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    __syncthreads();
    store_tile_a(P, As, ra);
    store_tile_b(P, Bs, rb);
    __syncthreads();
    if (k0 + BK < kend) {
      load_tile_a(P, m0, k0 + BK, kend, ra);
      load_tile_b(P, n0, k0 + BK, kend, rb);
    }
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
  if (ksn == 1) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + ty + 16 * i;
      if (m >= P.M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = n0 + tx + 16 * j;
        if (n >= P.N) continue;
        double* c = P.C + (int64_t)m * P.ldc + n;
        const double v = L.alpha * acc[i][j];
        *c = (L.beta == 0.0) ? v : fma(L.beta, *c, v);
      }
    }
  } else {
    double* part = L.scratch + L.poff[pi] + (int64_t)ks * P.M * P.N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + ty + 16 * i;
      if (m >= P.M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = n0 + tx + 16 * j;
        if (n >= P.N) continue;
        part[(int64_t)m * P.N + n] = acc[i][j];
      }
    }
  }
}

struct ReduceLaunch {
  double* C[GEMM_MAXPROB];
  int M[GEMM_MAXPROB], N[GEMM_MAXPROB], ldc[GEMM_MAXPROB], ks[GEMM_MAXPROB];
  int64_t poff[GEMM_MAXPROB];
  int64_t elem0[GEMM_MAXPROB + 1];
  int np;
  double alpha, beta;
  const double* scratch;
};

__global__ void splitk_reduce_kernel(const __grid_constant__ ReduceLaunch R) {
  const int64_t total = R.elem0[R.np];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int pi = 0;
    while (pi + 1 < R.np && e >= R.elem0[pi + 1]) ++pi;
    const int64_t loc = e - R.elem0[pi];
    const int m = (int)(loc / R.N[pi]), n = (int)(loc % R.N[pi]);
    const int64_t MN = (int64_t)R.M[pi] * R.N[pi];
    const double* part = R.scratch + R.poff[pi] + loc;
    double s = 0.0;
    for (int k = 0; k < R.ks[pi]; ++k) s += part[k * MN];
    double* c = R.C[pi] + (int64_t)m * R.ldc[pi] + n;
    const double v = R.alpha * s;
    *c = (R.beta == 0.0) ? v : fma(R.beta, *c, v);
  }
}

void plan_splitk(const GemmProb& p, int& tm, int& tn, int& ks) {
  tm = (p.M + BM - 1) / BM;
  tn = (p.N + BN - 1) / BN;
  ks = 1;
  const int tiles = tm * tn;
  if (tiles < 64 && p.K >= 2048) {
    ks = std::min((int)((p.K + 1023) / 1024), std::max(1, 256 / tiles));
    ks = std::max(1, std::min(ks, 512));
  }
}

}  // namespace

int chunk_elems() { return CHUNK; }

int64_t gemm_scratch_doubles(const GemmProb* p, int np) {
  int64_t s = 0;
  for (int i = 0; i < np; ++i) {
    if (p[i].M <= 0 || p[i].N <= 0) continue;
    int tm, tn, ks;
    plan_splitk(p[i], tm, tn, ks);
    if (ks > 1) s += (int64_t)ks * p[i].M * p[i].N;
  }
  return s;
}

int gemm64_grouped(const GemmProb* p, int np, double alpha, double beta,
                   double* scratch, cudaStream_t st) {
  GemmLaunch L;
  std::memset(&L, 0, sizeof(L));
  ReduceLaunch R;
  std::memset(&R, 0, sizeof(R));
  L.alpha = alpha;
  L.beta = beta;
  L.scratch = scratch;
  R.alpha = alpha;
  R.beta = beta;
  R.scratch = scratch;
  int n = 0, nr = 0, tiles = 0;
  int64_t poff = 0, relem = 0;
  for (int i = 0; i < np; ++i) {
    if (p[i].M <= 0 || p[i].N <= 0) continue;
    int tm, tn, ks;
    plan_splitk(p[i], tm, tn, ks);
    L.p[n] = p[i];
    L.tm[n] = tm;
    L.tn[n] = tn;
    L.ks[n] = ks;
    L.tile0[n] = tiles;
    L.poff[n] = ks > 1 ? poff : 0;
    tiles += tm * tn * ks;
    if (ks > 1) {
      R.C[nr] = p[i].C;
      R.M[nr] = p[i].M;
      R.N[nr] = p[i].N;
      R.ldc[nr] = p[i].ldc;
      R.ks[nr] = ks;
      R.poff[nr] = poff;
      R.elem0[nr] = relem;
      relem += (int64_t)p[i].M * p[i].N;
      poff += (int64_t)ks * p[i].M * p[i].N;
      ++nr;
    }
    ++n;
  }
  if (n == 0) return 0;
  L.np = n;
  L.tile0[n] = tiles;
  gemm64_kernel<<<tiles, NT, 0, st>>>(L);
  int launches = 1;
  if (nr > 0) {
    R.np = nr;
    R.elem0[nr] = relem;
    const int blocks = (int)std::min<int64_t>((relem + 255) / 256, 4096);
    splitk_reduce_kernel<<<blocks, 256, 0, st>>>(R);
    ++launches;
  }
  return launches;
}

// ----------------------------------------------------------- permute / axpy
namespace {

__device__ __forceinline__ void box_offsets(const PermTask& t, int64_t e,
                                            int64_t& y, int64_t& x,
                                            int* l) {
  y = t.ybase;
  x = t.xbase;
  for (int q = t.rank - 1; q >= 0; --q) {
    const int d = t.dim[q];
    const int64_t lq = e % d;
    e /= d;
    l[q] = (int)lq;
    y += lq * t.ys[q];
    x += lq * t.xs[q];
  }
}

__global__ void perm_axpy_kernel(const PermTask* __restrict__ tasks,
                                 const Chunk* __restrict__ chunks,
                                 double alpha, const double* __restrict__ X,
                                 double beta, double* __restrict__ Y) {
  const Chunk c = chunks[blockIdx.x];
  const PermTask t = tasks[c.task];
  const int64_t end = min(t.n, c.start + (int64_t)CHUNK);
  int l[MAXRANK];
  for (int64_t e = c.start + threadIdx.x; e < end; e += blockDim.x) {
    int64_t y, x;
    box_offsets(t, e, y, x, l);
    const double v = alpha * X[x];
    Y[y] = (beta == 0.0) ? v : fma(beta, Y[y], v);
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
  const PermTask t = tasks[c.task];
  const int64_t end = min(t.n, c.start + (int64_t)CHUNK);
  int l[MAXRANK];
  double mx = 0.0;
  for (int64_t e = c.start + threadIdx.x; e < end; e += blockDim.x) {
    int64_t y, x;
    box_offsets(t, e, y, x, l);
    double D = 0.0;
    for (int q = 0; q < t.rank; ++q) D += t.sgn[q] * eps[t.gidx[q] + l[q]];
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
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 8));
}

}  // namespace

int perm_axpy(const PermTask* d_tasks, const Chunk* d_chunks, int nchunks,
              double alpha, const double* X, double beta, double* Y,
              cudaStream_t st) {
  if (nchunks <= 0) return 0;
  perm_axpy_kernel<<<nchunks, 256, 0, st>>>(d_tasks, d_chunks, alpha, X, beta,
                                            Y);
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
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  lincomb_kernel<<<std::max(blocks, 1), 256, 0, st>>>(out, pk, m, n);
  return 1;
}

int axpby(double a, const double* x, double b, double* y, int64_t n,
          cudaStream_t st) {
  if (n <= 0) return 0;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
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

}  // namespace cdcc
