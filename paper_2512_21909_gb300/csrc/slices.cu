// slices.cu -- FP64 operands -> K-major BF16 slices for the tensor-core GEMMs.
//
// Output layout: dst[slice][row][Kp] (Kp = K rounded up to 8, zero padded),
// row = output row of the GEMM side (op(A) rows, or op(B)^T rows).
// Source element (row, k) = trans ? src[k*ld + row] : src[row*ld + k].
//   float slices : x = x0 + x1 + ..., x_i = bf16(residual)      (tc_gemm.cu)
//   exact slices : x = 2^e * sum_i X_i 2^(-8-7i), X_0 in [-256,256],
//                  X_i in [-64,63] integers, e from the row maximum
//                  (tc_ozaki.cu)
// Non-transposed sources: one CTA covers 2048 k of one row, 8 per thread,
// one 16-byte store per slice.  Transposed sources: 64 (k) x 32 (rows)
// tiles through shared memory so that reads and writes are both coalesced.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.h"

namespace cdcc {

namespace {

constexpr int SK_PER_THREAD = 8;
constexpr int SK_THREADS = 256;
constexpr int SK_SPAN = SK_PER_THREAD * SK_THREADS;   // 2048 k per CTA

struct Pack8 {
  __nv_bfloat16 v[8];
};

// Slices of 8 consecutive k of one row, written as one 16-byte store per
// slice.  The arithmetic stays off the FP64 pipe (at most one conversion per
// element):
//   float: x -> FP32 (24 bits, all that three BF16 slices can hold), then
//          x_i = bf16(r), r -= x_i in FP32 (exact)
//   exact: q = round(x * 2^(8 - e + 7(s-1))) as a 64-bit integer, taken
//          from the bit pattern of x with integer operations, then balanced base-128
//          digits X_{s-1}..X_1 in [-64, 63] and the leading X_0 = the rest,
//          |X_0| <= 256; sum_i X_i 2^(-7i) = q 2^(-7(s-1)), i.e. x rounded
//          to 8 + 7(s-1) bits below the row maximum
// round(x * 2^sh) to the nearest integer, ties to even (the rounding of
// __double2ll_rn), from the bit pattern with integer operations only.
// Valid while |x * 2^sh| < 2^62; zero and subnormal x give 0.
__device__ __forceinline__ long long round_scaled(double x, int sh) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  if (E == 0) return 0;
  const long long mant = (b & 0xfffffffffffffLL) | (1LL << 52);
  const int shift = E - 1075 + sh;          // |x| 2^sh = mant 2^shift
  long long q;
  if (shift >= 0) {
    q = mant << min(shift, 9);
  } else if (shift < -63) {
    q = 0;
  } else {
    const int r = -shift;
    q = mant >> r;
    const unsigned long long rem =
        (unsigned long long)mant & ((1ULL << r) - 1ULL);
    const unsigned long long half = 1ULL << (r - 1);
    if (rem > half || (rem == half && (q & 1))) ++q;
  }
  return b < 0 ? -q : q;
}

template <bool EXACT>
__device__ __forceinline__ void slice8(const double (&x)[8], int e, int s,
                                       __nv_bfloat16* dst, int64_t stride) {
  if (EXACT) {
    const int sh = 8 - e + 7 * (s - 1);
    int dig[4][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      long long v = round_scaled(x[q], sh);
#pragma unroll
      for (int i = 3; i >= 1; --i) {
        if (i < s) {
          const int d = (int)((v + 64) & 127) - 64;
          dig[i][q] = d;
          v = (v - d) >> 7;
        }
      }
      dig[0][q] = (int)v;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i < s) {
        Pack8 p;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          p.v[q] = __float2bfloat16_rn((float)dig[i][q]);
        *reinterpret_cast<uint4*>(dst + (int64_t)i * stride) =
            *reinterpret_cast<const uint4*>(&p);
      }
    }
  } else {
    float r[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) r[q] = __double2float_rn(x[q]);
    for (int i = 0; i < s; ++i) {
      Pack8 p;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const __nv_bfloat16 b = __float2bfloat16_rn(r[q]);
        p.v[q] = b;
        r[q] -= __bfloat162float(b);
      }
      *reinterpret_cast<uint4*>(dst + (int64_t)i * stride) =
          *reinterpret_cast<const uint4*>(&p);
    }
  }
}

template <bool EXACT>
__global__ void __launch_bounds__(SK_THREADS)
    split_rows_kernel(const double* __restrict__ src, int rows, int K,
                      int64_t ld, const int* __restrict__ exps,
                      __nv_bfloat16* __restrict__ dst, int Kp, int s,
                      int kblocks) {
  const int row = blockIdx.x / kblocks;
  const int kb = blockIdx.x % kblocks;
  const int k0 = kb * SK_SPAN + threadIdx.x * SK_PER_THREAD;
  if (row >= rows || k0 >= Kp) return;
  double x[8];
  const double* s0 = src + (int64_t)row * ld;
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = (k0 + q < K) ? s0[k0 + q] : 0.0;
  const int e = EXACT ? exps[row] : 0;
  slice8<EXACT>(x, e, s, dst + (int64_t)row * Kp + k0, (int64_t)rows * Kp);
}

constexpr int TT_K = 64, TT_R = 32;

template <bool EXACT>
__global__ void __launch_bounds__(256)
    split_trans_kernel(const double* __restrict__ src, int rows, int K,
                       int64_t ld, const int* __restrict__ exps,
                       __nv_bfloat16* __restrict__ dst, int Kp, int s,
                       int rblocks) {
  __shared__ double tile[TT_K][TT_R + 1];
  const int rb = blockIdx.x % rblocks, kb = blockIdx.x / rblocks;
  const int r0 = rb * TT_R, k0 = kb * TT_K;
  const int t = threadIdx.x;
  // load: 64 k-lines of 32 consecutive rows
  for (int i = t; i < TT_K * TT_R; i += 256) {
    const int kk = i / TT_R, rr = i % TT_R;
    const int k = k0 + kk, r = r0 + rr;
    tile[kk][rr] = (k < K && r < rows) ? src[(int64_t)k * ld + r] : 0.0;
  }
  __syncthreads();
  // each thread: one row, 8 consecutive k
  const int rr = t % TT_R, kq = (t / TT_R) * 8;   // 8 groups of 8 k
  const int r = r0 + rr, k = k0 + kq;
  if (r >= rows || k >= Kp) return;
  double x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = tile[kq + q][rr];
  const int e = EXACT ? exps[r] : 0;
  slice8<EXACT>(x, e, s, dst + (int64_t)r * Kp + k, (int64_t)rows * Kp);
}

// exponent e of each row (max |x| < 2^e); non-transposed: a warp per row
__global__ void rowexp_rows_kernel(const double* __restrict__ src, int rows,
                                   int K, int64_t ld, int* __restrict__ e) {
  const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;
  // |x| compared as bit patterns (monotone for non-negative doubles)
  long long mb = 0;
  const double* s0 = src + (int64_t)w * ld;
  for (int k = lane; k < K; k += 32)
    mb = max(mb, __double_as_longlong(s0[k]) & 0x7fffffffffffffffLL);
  for (int o = 16; o > 0; o >>= 1)
    mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  const double m = __longlong_as_double(mb);
  if (lane == 0) e[w] = (m > 0.0) ? ilogb(m) + 1 : -100000;
}

// transposed: a thread per row over a chunk of k, combined with atomicMax
__global__ void rowexp_trans_kernel(const double* __restrict__ src, int rows,
                                    int K, int64_t ld, int kchunk,
                                    int* __restrict__ e) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int k0 = blockIdx.y * kchunk, k1 = min(K, k0 + kchunk);
  if (r >= rows) return;
  long long mb = 0;
  for (int k = k0; k < k1; ++k)
    mb = max(mb, __double_as_longlong(src[(int64_t)k * ld + r]) &
                     0x7fffffffffffffffLL);
  const double m = __longlong_as_double(mb);
  if (m > 0.0) atomicMax(e + r, ilogb(m) + 1);
}

__global__ void fix_exps_kernel(int* e, int rows) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < rows && e[r] < -99999) e[r] = 0;
}

__global__ void fill_int_kernel(int* e, int rows, int v) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < rows) e[r] = v;
}

template <bool EXACT>
int launch_split(const double* src, int rows, int K, int64_t ld, int trans,
                 const int* exps, __nv_bfloat16* dst, int Kp, int s,
                 cudaStream_t st) {
  if (rows <= 0 || Kp <= 0) return 0;
  if (!trans) {
    const int kblocks = (Kp + SK_SPAN - 1) / SK_SPAN;
    split_rows_kernel<EXACT><<<rows * kblocks, SK_THREADS, 0, st>>>(
        src, rows, K, ld, exps, dst, Kp, s, kblocks);
  } else {
    const int rblocks = (rows + TT_R - 1) / TT_R;
    const int kblocks = (Kp + TT_K - 1) / TT_K;
    split_trans_kernel<EXACT><<<rblocks * kblocks, 256, 0, st>>>(
        src, rows, K, ld, exps, dst, Kp, s, rblocks);
  }
  return 1;
}

}  // namespace

int slice_kp(int K) { return (K + 7) / 8 * 8; }

int split_float(const double* src, int rows, int K, int64_t ld, int trans,
                int nslice, void* dst, cudaStream_t st) {
  return launch_split<false>(src, rows, K, ld, trans, nullptr,
                             (__nv_bfloat16*)dst, slice_kp(K), nslice, st);
}

int split_exact(const double* src, int rows, int K, int64_t ld, int trans,
                int nslice, void* dst, int* exps, cudaStream_t st) {
  if (rows <= 0) return 0;
  int n = 0;
  if (!trans) {
    const int64_t thr = (int64_t)rows * 32;
    rowexp_rows_kernel<<<(int)((thr + 255) / 256), 256, 0, st>>>(src, rows, K,
                                                                 ld, exps);
    ++n;
  } else {
    fill_int_kernel<<<(rows + 255) / 256, 256, 0, st>>>(exps, rows, -100000);
    const int kchunk = 512;
    dim3 grid((rows + 255) / 256, std::max(1, (K + kchunk - 1) / kchunk));
    rowexp_trans_kernel<<<grid, 256, 0, st>>>(src, rows, K, ld, kchunk, exps);
    n += 2;
  }
  fix_exps_kernel<<<(rows + 255) / 256, 256, 0, st>>>(exps, rows);
  ++n;
  n += launch_split<true>(src, rows, K, ld, trans, exps, (__nv_bfloat16*)dst,
                          slice_kp(K), nslice, st);
  return n;
}

}  // namespace cdcc
