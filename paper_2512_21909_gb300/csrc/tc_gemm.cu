// tc_gemm.cu -- split-precision tensor-core GEMM for sm_103a (tcgen05 + TMA).
//
// C (FP64) = beta*C + alpha * op(A) op(B) with FP64 operands, computed on
// the 5th-generation tensor cores:
//   * each FP64 operand element is split into s BF16 slices
//       x = x0 + x1 (+ x2),  x0 = bf16(x), x1 = bf16(x - x0), ...
//     (residuals formed exactly in FP64), stored K-major;
//   * the products x_i * y_j with i + j < s (1, 3 or 6 of them) are summed
//     by tcgen05.mma.kind::f16 into ONE FP32 accumulator in tensor memory;
//     s = 2 keeps ~16 significant bits per operand ("BF16x3"), s = 3 keeps
//     ~24 bits (FP32-class products);
//   * operand tiles are staged by TMA (128B swizzle, OOB rows/cols read as
//     zero) through a multi-stage mbarrier pipeline; one thread issues the
//     MMAs, tcgen05.commit frees smem stages; 4 warps drain the accumulator
//     with tcgen05.ld and write FP64 (split-K partials go to scratch and are
//     summed in a fixed order).
// Tile: 128 rows (MMA M = 128) x BN in {32, 64, 128, 256} columns (MMA N =
// BN); the larger output dimension is mapped to the 128-row side (C is then
// written transposed).  The kernel is persistent (one CTA per SM walks its
// tiles) with two TMEM accumulators, so one tile's epilogue overlaps the
// next tile's loads and MMAs.  Every mbarrier wait is bounded; on a timeout
// the kernel sets an error flag, stops issuing work, waits (bounded) for its
// own copies in flight and still releases its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <stdexcept>
#include <string>

#include <cmath>

#include "fp64_bits.cuh"
#include "kernels.h"

namespace cdcc {

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;          // K per stage: one 128-byte swizzle row
// TMA warp, MMA warp, and 8 epilogue warps: two per TMEM sub-partition,
// each draining half of a tile's columns (a single warp per scheduler left
// the epilogue latency bound)
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;
constexpr int TC_STG_BYTES = 2432;   // staging per epilogue warp
constexpr int TC_MAXPROB = 8;
constexpr int TC_SMEM_BUDGET = 200 * 1024;
constexpr long long TC_SPIN_LIMIT = 1LL << 22;

struct TcLaunch {
  CUtensorMap ta[TC_MAXPROB];  // A slices: dims {Kp, rows, s}, box {64,128,1}
  CUtensorMap tb[TC_MAXPROB];  // B slices: dims {Kp, cols, s}, box {64,BN,1}
  double* C[TC_MAXPROB];
  int64_t poff[TC_MAXPROB];
  int M[TC_MAXPROB], N[TC_MAXPROB], ldc[TC_MAXPROB], nkb[TC_MAXPROB];
  int tm[TC_MAXPROB], tn[TC_MAXPROB], ks[TC_MAXPROB];
  int tile0[TC_MAXPROB + 1];
  int np, nslice, bn, stages, trans_out;
  double alpha, beta;
  Pow2 ap2;                    // alpha as +-2^k (folded into the exponent)
  double* scratch;
  unsigned int* err;
  // fused ladder epilogue: outputs go to BF16 slices of (ab|cd) rows
  TcLadEpi lad[TC_MAXPROB];
  int lad_on;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)),
               "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
          smem_u32(b)),
      "r"(bytes)
      : "memory");
}

// Bounded wait on an mbarrier phase; false (and *err = code) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity,
                                          unsigned int* err,
                                          unsigned int code) {
  const uint32_t a = smem_u32(b);
  for (long long i = 0; i < TC_SPIN_LIMIT; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  atomicExch(err, code);
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map,
                                            int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::"
      "complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128B swizzle, 8-row groups
// 1024 bytes apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused, swizzled)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad,
                                         uint64_t bd, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
          tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
      "[%0];" ::"r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, "
      "[%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]),
        "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]),
        "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b))
               : "memory");
}

// Tile t of the launch -> problem, 128-row tile, column tile, K split.
struct TcTile {
  int pi, m0, n0, ksi, kb0, kb1;
};

__device__ __forceinline__ TcTile tc_tile(const TcLaunch& L, int t) {
  TcTile r;
  int pi = 0;
  while (pi + 1 < L.np && t >= L.tile0[pi + 1]) ++pi;
  int local = t - L.tile0[pi];
  const int ksn = L.ks[pi];
  r.pi = pi;
  r.ksi = local % ksn;
  local /= ksn;
  r.n0 = (local % L.tn[pi]) * L.bn;
  r.m0 = (local / L.tn[pi]) * TC_BM;
  const int nkb = L.nkb[pi];
  const int per = (nkb + ksn - 1) / ksn;
  r.kb0 = r.ksi * per;
  r.kb1 = min(nkb, r.kb0 + per);
  if (r.kb1 < r.kb0) r.kb1 = r.kb0;
  return r;
}

// Persistent and warp-specialised: CTA b takes tiles b, b + gridDim.x, ...
// warp 0 issues the TMA loads of the K blocks into a ring of shared-memory
// stages, warp 1 issues the MMAs of a tile into one of two TMEM accumulators
// (alternating per tile), warps 2..5 drain the other accumulator (the
// previous tile) and write its outputs, so the epilogue of one tile overlaps
// the loads and MMAs of the next.  The three roles walk the same tile
// sequence with running counters.
// LAD: the fused ladder epilogue (outputs to BF16 slices of (ab|cd) rows);
// a separate instance so that each epilogue is compiled without the other
template <bool LAD>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ TcLaunch L) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = L.stages, s = L.nslice, BN = L.bn;
  const uint32_t a_bytes = TC_BM * 128, b_bytes = (uint32_t)BN * 128;
  const uint32_t stage_bytes = (uint32_t)s * (a_bytes + b_bytes);
  uint64_t* full = (uint64_t*)(smem + (size_t)S * stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;   // [2] accumulator ready
  uint64_t* acce = accf + 2;    // [2] accumulator drained
  uint64_t* fin = acce + 2;     // every MMA of this CTA complete
  uint32_t* tmem_slot = (uint32_t*)(fin + 1);
  int* consumed = (int*)(tmem_slot + 1);
  // per epilogue warp TC_STG_BYTES of staging (a 32 x 17 float sub-tile,
  // or for the fused ladder a 32 x 18 float sub-tile and 32 row offsets)
  uint8_t* stage_out = smem + (size_t)S * stage_bytes + 256;

  const int ntile = L.tile0[L.np];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ncols = 2u * (uint32_t)BN;   // two accumulators

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], TC_EPI_WARPS);   // one arrive per epilogue warp
    }
    mbar_init(fin, 1);
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], "
        "%1;" ::"r"(smem_u32(tmem_slot)),
        "r"(ncols)
        : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                         ((uint32_t)(BN >> 3) << 17) |
                         ((uint32_t)(TC_BM >> 4) << 24);
  int issued = 0;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      int g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
        const TcTile T = tc_tile(L, t);
        for (int kb = T.kb0; kb < T.kb1; ++kb, ++g) {
          const int st = g % S, round = g / S;
          if (round > 0 && !mbar_wait(&empty[st], (round - 1) & 1, L.err, 1)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[st], stage_bytes);
          uint8_t* sa = smem + (size_t)st * stage_bytes;
          uint8_t* sb = sa + (size_t)s * a_bytes;
          const int kc = kb * TC_BK;
          for (int i = 0; i < s; ++i) {
            tma_load_3d(sa + (size_t)i * a_bytes, &L.ta[T.pi], kc, T.m0, i,
                        &full[st]);
            tma_load_3d(sb + (size_t)i * b_bytes, &L.tb[T.pi], kc, T.n0, i,
                        &full[st]);
          }
          issued = g + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer: tile c (with K blocks) -> accumulator c & 1
      bool ok = true;
      int g = 0, c = 0;
      for (int t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
        const TcTile T = tc_tile(L, t);
        if (T.kb1 <= T.kb0) continue;   // empty K split: no accumulator
        const int set = c & 1;
        if (c >= 2 && !mbar_wait(&acce[set], ((c >> 1) - 1) & 1, L.err, 4)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(set * BN);
        int first = 1;
        for (int kb = T.kb0; kb < T.kb1; ++kb, ++g) {
          const int st = g % S, round = g / S;
          if (!mbar_wait(&full[st], round & 1, L.err, 2)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(smem + (size_t)st * stage_bytes);
          const uint32_t sb = sa + (uint32_t)s * a_bytes;
          for (int d = 0; d < s; ++d)        // slice products i + j = d
            for (int i = 0; i <= d; ++i) {
              const int j = d - i;
#pragma unroll
              for (int kk = 0; kk < TC_BK / 16; ++kk) {
                const uint64_t ad = smem_desc(sa + i * a_bytes + kk * 32);
                const uint64_t bd = smem_desc(sb + j * b_bytes + kk * 32);
                mma_bf16(acc, ad, bd, idesc, first ? 0u : 1u);
                first = 0;
              }
            }
          mma_commit(&empty[st]);
          *(volatile int*)consumed = g + 1;
        }
        if (!ok) break;
        mma_commit(&accf[set]);
        ++c;
      }
      mma_commit(fin);   // arrives once every MMA issued above completed
    }
  } else {
    // ---- epilogue warps 2..9: TMEM sub-partition warp % 4 (32 rows each),
    // half (warp - 2) / 4 of the tile's columns.  With the logical rows on
    // the 128-row side (trans_out = 0) a lane holds one row of C; the warp
    // passes 32 x 16 sub-tiles through shared memory so that consecutive
    // lanes write consecutive columns.
    const int sub = warp & 3;
    const int half = (warp - 2) >> 2;
    float* stg = reinterpret_cast<float*>(stage_out +
                                          (size_t)(warp - 2) * TC_STG_BYTES);
    bool ok = true;
    int c = 0;
    for (int t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
      const TcTile T = tc_tile(L, t);
      const int pi = T.pi;
      const bool have = T.kb1 > T.kb0;
      const int set = c & 1;
      if (have) {
        if (!mbar_wait(&accf[set], (c >> 1) & 1, L.err, 3)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
      const int Mr = L.trans_out ? L.N[pi] : L.M[pi];
      const int Nc = L.trans_out ? L.M[pi] : L.N[pi];
      double* C = L.C[pi];
      const int ldc = L.ldc[pi];
      const int ksn = L.ks[pi];
      // logical C element (m, n) from the FP32 accumulator value v; FP64
      // values are built with integer operations (fp64_bits.cuh)
      auto put = [&](int m, int n, float v) {
        if (LAD) {
          // X_gc[(a,c),(b,d)] -> row (a,b), column coff + c*nd + d of the
          // batch's (ab|cd) rows, cut into BF16 slices hi + lo (+ ...)
          const TcLadEpi& E = L.lad[pi];
          const int a = m / E.nc, c = m - a * E.nc;
          const int b = n / E.nd, d = n - b * E.nd;
          const int64_t off = (int64_t)(a * E.nb + b) * E.Kp + E.coff +
                              (int64_t)c * E.nd + d;
          float w = v;
#pragma unroll 1
          for (int q = 0; q < E.ns; ++q) {
            const __nv_bfloat16 hq = __float2bfloat16_rn(w);
            ((__nv_bfloat16*)E.W)[(int64_t)q * E.rows * E.Kp + off] = hq;
            w -= __bfloat162float(hq);
          }
          return;
        }
        if (ksn == 1) {
          double* p = C + (int64_t)m * ldc + n;
          double val;
          if (L.ap2.ok) {
            val = f32_to_f64_scaled(v, L.ap2.sh);
            if (L.ap2.neg) val = -val;
          } else {
            val = L.alpha * f32_to_f64_scaled(v, 0);
          }
          if (L.beta == 0.0)
            *p = val;
          else if (L.beta == 1.0)
            *p += val;
          else
            *p = fma(L.beta, *p, val);
        } else {
          L.scratch[L.poff[pi] + (int64_t)T.ksi * L.M[pi] * L.N[pi] +
                    (int64_t)m * L.N[pi] + n] = f32_to_f64_scaled(v, 0);
        }
      };
      float v[32];
      float* stf = stg;
      const int cbeg = half * (BN / 2), cend = BN < 64 ? (half ? 0 : BN)
                                                       : cbeg + BN / 2;
      for (int c0 = BN < 64 ? 0 : cbeg; c0 < cend; c0 += 32) {
        __syncwarp();   // tcgen05.ld is warp-aligned
        if (have) {
          tmem_ld32(tmem + ((uint32_t)(sub * 32) << 16) +
                        (uint32_t)(set * BN + c0),
                    v);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = 0.f;
        }
        if (L.trans_out) {
          // lanes run along n already
          const int r = T.m0 + sub * 32 + lane;
          if (r < Mr) {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const int cc = T.n0 + c0 + i;
              if (cc >= Nc) break;
              put(cc, r, v[i]);
            }
          }
        } else if (LAD) {
          // fused ladder rows.  Each 32 x 16 half of the warp's chunk is
          // staged in shared memory; a lane then writes two adjacent columns
          // of one row per step (8 lanes cover a row's 16 columns, 4 rows
          // per step): the (a,c) part of a row's target offset is computed
          // once per row, the (b,d) part once per half.  A pair inside one
          // (b) group at an even offset is stored as one packed BF16 pair
          // per slice, otherwise as two values (with nd odd the second
          // column may start the next (b) group).
          const TcLadEpi& E = L.lad[pi];
          float* stc = stf;                                  // [32][18]
          int32_t* rbase = reinterpret_cast<int32_t*>(stf + 32 * 18);
          if (c0 == (BN < 64 ? 0 : cbeg)) {
            __syncwarp();
            const int m = T.m0 + sub * 32 + lane;
            const int a = m / E.nc, c = m - a * E.nc;
            rbase[lane] = (int32_t)((int64_t)a * E.nb * E.Kp + E.coff +
                                    (int64_t)c * E.nd);
          }
          __nv_bfloat16* W0 = (__nv_bfloat16*)E.W;
          const int32_t sstride = (int32_t)(E.rows * E.Kp);
          __nv_bfloat16* W1 = W0 + sstride;
          const int rows_ok = Mr - (T.m0 + sub * 32);
          const int p2 = (lane & 7) * 2;             // column pair
          const int rsel = lane >> 3;                // row within a step
#pragma unroll
          for (int h = 0; h < 32; h += 16) {
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 16; ++j) stc[lane * 18 + j] = v[h + j];
            __syncwarp();
            const int n = T.n0 + c0 + h + p2;
            const int nn = n < Nc ? n : Nc - 1;   // guarded below
            const int b = nn / E.nd, d = nn - b * E.nd;
            const int32_t noff = (int32_t)((int64_t)b * E.Kp + d);
            // second column of the pair: same (b) group, or the first of
            // the next one
            const bool same = d + 1 < E.nd;
            const int32_t noff1 =
                same ? noff + 1 : (int32_t)((int64_t)(b + 1) * E.Kp);
            const bool two = n + 1 < Nc;
            if (E.ns == 2) {
#pragma unroll 4
              for (int rr = 0; rr < 32; rr += 4) {
                const int row = rr + rsel;
                if (row >= rows_ok || n >= Nc) continue;
                const int32_t rb = rbase[row];
                const int32_t off = rb + noff;
                const float2 w = *reinterpret_cast<const float2*>(
                    stc + row * 18 + p2);
                const __nv_bfloat162 hi = __float22bfloat162_rn(w);
                const float2 hf = __bfloat1622float2(hi);
                const __nv_bfloat162 lo = __float22bfloat162_rn(
                    make_float2(w.x - hf.x, w.y - hf.y));
                if (two && same && !(off & 1)) {
                  *reinterpret_cast<__nv_bfloat162*>(W0 + off) = hi;
                  *reinterpret_cast<__nv_bfloat162*>(W1 + off) = lo;
                } else {
                  W0[off] = hi.x;
                  W1[off] = lo.x;
                  if (two) {
                    const int32_t off1 = rb + noff1;
                    W0[off1] = hi.y;
                    W1[off1] = lo.y;
                  }
                }
              }
            } else {
              for (int rr = 0; rr < 32; rr += 4) {
                const int row = rr + rsel;
                if (row >= rows_ok || n >= Nc) continue;
                const int32_t rb = rbase[row];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                  if (k == 1 && !two) continue;
                  const int32_t off = rb + (k == 0 ? noff : noff1);
                  float w = stc[row * 18 + p2 + k];
#pragma unroll 1
                  for (int q = 0; q < E.ns; ++q) {
                    const __nv_bfloat16 hq = __float2bfloat16_rn(w);
                    W0[q * sstride + off] = hq;
                    w -= __bfloat162float(hq);
                  }
                }
              }
            }
          }
        } else {
#pragma unroll
          for (int h = 0; h < 32; h += 16) {
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 16; ++j) stf[lane * 17 + j] = v[h + j];
            __syncwarp();
#pragma unroll 4
            for (int rr = 0; rr < 32; rr += 2) {
              const int row = rr + (lane >> 4), col = lane & 15;
              const int m = T.m0 + sub * 32 + row, n = T.n0 + c0 + h + col;
              if (m < Mr && n < Nc) put(m, n, stf[row * 17 + col]);
            }
          }
        }
      }
      if (have) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[set]);
        ++c;
      }
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0 && lane == 0) {
    // loads issued but never consumed (only after a timeout): wait for them
    // to land before the CTA leaves (bounded)
    for (int g = *(volatile int*)consumed; g < issued; ++g)
      mbar_wait(&full[g % S], (g / S) & 1, L.err, 5);
  }
  if (warp == 1) {
    if (lane == 0) mbar_wait(fin, 0, L.err, 6);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(
                     tmem),
                 "r"(ncols)
                 : "memory");
  }
}

struct ReduceL {
  double* C[TC_MAXPROB];
  int M[TC_MAXPROB], N[TC_MAXPROB], ldc[TC_MAXPROB], ks[TC_MAXPROB];
  int64_t poff[TC_MAXPROB], elem0[TC_MAXPROB + 1];
  int np;
  double alpha, beta;
  const double* scratch;
};

__global__ void tc_reduce_kernel(const __grid_constant__ ReduceL R) {
  const int64_t total = R.elem0[R.np];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int pi = 0;
    while (pi + 1 < R.np && e >= R.elem0[pi + 1]) ++pi;
    const int64_t loc = e - R.elem0[pi];
    const int m = (int)(loc / R.N[pi]), n = (int)(loc % R.N[pi]);
    const int64_t MN = (int64_t)R.M[pi] * R.N[pi];
    const double* part = R.scratch + R.poff[pi] + loc;
    double acc = 0.0;
    for (int k = 0; k < R.ks[pi]; ++k) acc += part[k * MN];
    double* c = R.C[pi] + (int64_t)m * R.ldc[pi] + n;
    const double v = R.alpha * acc;
    *c = (R.beta == 0.0) ? v : fma(R.beta, *c, v);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

void encode_init() {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                       cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    fn = nullptr;
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
}

void make_map(CUtensorMap* m, const __nv_bfloat16* base, int Kp, int rows,
              int s, int box_rows) {
  std::call_once(g_encode_once, encode_init);
  if (!g_encode) throw std::runtime_error("cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)s};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * rows};
  cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, 1};
  cuuint32_t est[3] = {1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base,
                        dims, strides, box, est, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw std::runtime_error("cuTensorMapEncodeTiled failed: " +
                             std::to_string((int)r));
}

struct TcPlan {
  bool swap;                     // 128-row side = logical N
  int bn, stages;
  int tm[TC_MAXPROB], tn[TC_MAXPROB], ks[TC_MAXPROB], nkb[TC_MAXPROB];
  int64_t scratch;               // FP64 split-K partials
};

TcPlan tc_plan(const TcProb* p, int np, int s) {
  TcPlan pl;
  std::memset(&pl, 0, sizeof(pl));
  int64_t sumM = 0, sumN = 0;
  for (int i = 0; i < np; ++i) {
    sumM += p[i].M;
    sumN += p[i].N;
  }
  pl.swap = sumN > sumM;
  int maxc = 0;
  for (int i = 0; i < np; ++i)
    maxc = std::max(maxc, pl.swap ? p[i].M : p[i].N);
  pl.bn = maxc <= 32 ? 32 : maxc <= 64 ? 64 : maxc <= 128 ? 128 : 256;
  // short K (a few K blocks per tile, as in the ladder builds with K = nL
  // of one irrep): 128-wide column tiles with three stages in flight beat
  // 256-wide ones with two (fused c3 build launch 462 -> 412 us; a 4048^3
  // product with long K is 15 % slower with them, so only for short K)
  int maxkb = 0;
  for (int i = 0; i < np; ++i)
    maxkb = std::max(maxkb, (p[i].K + TC_BK - 1) / TC_BK);
  if (pl.bn == 256 && maxkb <= 8) pl.bn = 128;
  // at least two stages in flight: narrower column tiles otherwise
  while (pl.bn > 32 && TC_SMEM_BUDGET / (s * (TC_BM * 128 + pl.bn * 128)) < 2)
    pl.bn /= 2;
  const int stage = s * (TC_BM * 128 + pl.bn * 128);
  pl.stages = std::max(1, std::min(4, TC_SMEM_BUDGET / stage));
  int64_t tiles = 0;
  for (int i = 0; i < np; ++i) {
    const int R = pl.swap ? p[i].N : p[i].M;
    const int Cc = pl.swap ? p[i].M : p[i].N;
    pl.nkb[i] = (p[i].K + TC_BK - 1) / TC_BK;
    pl.tm[i] = (R + TC_BM - 1) / TC_BM;
    pl.tn[i] = (Cc + pl.bn - 1) / pl.bn;
    tiles += (int64_t)pl.tm[i] * pl.tn[i];
  }
  for (int i = 0; i < np; ++i) {
    pl.ks[i] = 1;
    const int64_t sms2 = 2 * (int64_t)sm_count();
    if (tiles < sms2 && pl.nkb[i] >= 8) {
      int ks = (int)((sms2 + tiles - 1) / std::max<int64_t>(tiles, 1));
      ks = std::min(ks, pl.nkb[i] / 4);
      pl.ks[i] = std::max(1, std::min(ks, 32));
    }
    if (pl.ks[i] > 1)
      pl.scratch += (int64_t)pl.ks[i] * p[i].M * p[i].N;
  }
  return pl;
}

}  // namespace

namespace {
// Largest dynamic shared memory of any launch: stages within the budget,
// barriers, epilogue staging.  The attribute belongs to the kernel on the
// device, shared by every host thread and stream, so it is set once to this
// maximum: a per-launch value could be lowered by a concurrent launch of a
// smaller configuration between another thread's set and launch.
constexpr int TC_SMEM_MAX =
    TC_SMEM_BUDGET + 1024 + 256 + TC_EPI_WARPS * TC_STG_BYTES;

void tc_smem_attr(int smem) {
  if (smem > TC_SMEM_MAX)
    throw std::runtime_error("tc: shared memory plan above its maximum");
  static std::once_flag once[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  std::call_once(once[dev], [] {
    cudaFuncSetAttribute(tc_gemm_kernel<false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         TC_SMEM_MAX);
    cudaFuncSetAttribute(tc_gemm_kernel<true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         TC_SMEM_MAX);
  });
}
}  // namespace

int64_t tc_sliced_scratch_doubles(const TcProb* p, int np, int nslice) {
  return tc_plan(p, np, nslice).scratch;
}

int tc_gemm_sliced(const TcProb* p, int np, double alpha, double beta,
                   int nslice, double* scratch, unsigned int* d_err,
                   cudaStream_t st) {
  if (np <= 0) return 0;
  if (np > TC_MAXPROB) throw std::runtime_error("tc: too many blocks");
  if (nslice < 1 || nslice > 3) throw std::runtime_error("tc: nslice");
  const TcPlan pl = tc_plan(p, np, nslice);
  TcLaunch* L = new TcLaunch;
  std::memset(L, 0, sizeof(TcLaunch));
  ReduceL R;
  std::memset(&R, 0, sizeof(R));
  int64_t poff = 0, relem = 0;
  int tiles = 0, nr = 0;
  for (int i = 0; i < np; ++i) {
    const TcProb& g = p[i];
    const SlicedOp& rowop = pl.swap ? g.b : g.a;
    const SlicedOp& colop = pl.swap ? g.a : g.b;
    make_map(&L->ta[i], (const __nv_bfloat16*)rowop.data, rowop.Kp,
             rowop.rows, nslice, TC_BM);
    make_map(&L->tb[i], (const __nv_bfloat16*)colop.data, colop.Kp,
             colop.rows, nslice, pl.bn);
    L->C[i] = g.C;
    L->M[i] = g.M;
    L->N[i] = g.N;
    L->ldc[i] = g.ldc;
    L->nkb[i] = pl.nkb[i];
    L->tm[i] = pl.tm[i];
    L->tn[i] = pl.tn[i];
    L->ks[i] = pl.ks[i];
    L->tile0[i] = tiles;
    L->poff[i] = pl.ks[i] > 1 ? poff : 0;
    tiles += pl.tm[i] * pl.tn[i] * pl.ks[i];
    if (pl.ks[i] > 1) {
      R.C[nr] = g.C;
      R.M[nr] = g.M;
      R.N[nr] = g.N;
      R.ldc[nr] = g.ldc;
      R.ks[nr] = pl.ks[i];
      R.poff[nr] = poff;
      R.elem0[nr] = relem;
      relem += (int64_t)g.M * g.N;
      poff += (int64_t)pl.ks[i] * g.M * g.N;
      ++nr;
    }
  }
  L->tile0[np] = tiles;
  L->np = np;
  L->nslice = nslice;
  L->bn = pl.bn;
  L->stages = pl.stages;
  L->trans_out = pl.swap ? 1 : 0;
  L->alpha = alpha;
  L->beta = beta;
  L->ap2 = pow2_of(alpha);
  L->scratch = scratch;
  L->err = d_err;
  const int stage = nslice * (TC_BM * 128 + pl.bn * 128);
  // stages, barriers, and the epilogue warps' staging tiles
  const int smem = pl.stages * stage + 1024 + 256 + TC_EPI_WARPS * TC_STG_BYTES;
  tc_smem_attr(smem);
  // persistent: one CTA per SM (at most one fits), tiles strided over them
  const int grid = std::max(1, std::min(tiles, sm_count()));
  tc_gemm_kernel<false><<<grid, TC_THREADS, smem, st>>>(*L);
  delete L;
  int launches = 1;
  if (nr > 0) {
    R.np = nr;
    R.elem0[nr] = relem;
    R.alpha = alpha;
    R.beta = beta;
    R.scratch = scratch;
    const int blocks = (int)std::min<int64_t>((relem + 255) / 256, 4096);
    tc_reduce_kernel<<<std::max(blocks, 1), 256, 0, st>>>(R);
    ++launches;
  }
  return launches;
}

int tc_gemm_ladder(const TcProb* p, int np, int nslice, const TcLadEpi* epi,
                   unsigned int* d_err, cudaStream_t st) {
  if (np <= 0) return 0;
  if (np > TC_MAXPROB) throw std::runtime_error("tc: too many blocks");
  if (nslice < 1 || nslice > 3) throw std::runtime_error("tc: nslice");
  TcPlan pl = tc_plan(p, np, nslice);
  TcLaunch* L = new TcLaunch;
  std::memset(L, 0, sizeof(TcLaunch));
  int tiles = 0;
  for (int i = 0; i < np; ++i) {
    const TcProb& g = p[i];
    const SlicedOp& rowop = pl.swap ? g.b : g.a;
    const SlicedOp& colop = pl.swap ? g.a : g.b;
    make_map(&L->ta[i], (const __nv_bfloat16*)rowop.data, rowop.Kp,
             rowop.rows, nslice, TC_BM);
    make_map(&L->tb[i], (const __nv_bfloat16*)colop.data, colop.Kp,
             colop.rows, nslice, pl.bn);
    L->C[i] = g.C;
    L->M[i] = g.M;
    L->N[i] = g.N;
    L->ldc[i] = g.ldc;
    L->nkb[i] = pl.nkb[i];
    L->tm[i] = pl.tm[i];
    L->tn[i] = pl.tn[i];
    L->ks[i] = 1;               // whole K per tile: outputs go to slices
    L->tile0[i] = tiles;
    L->lad[i] = epi[i];
    tiles += pl.tm[i] * pl.tn[i];
  }
  L->tile0[np] = tiles;
  L->np = np;
  L->nslice = nslice;
  L->bn = pl.bn;
  L->stages = pl.stages;
  L->trans_out = pl.swap ? 1 : 0;
  L->alpha = 1.0;
  L->beta = 0.0;
  L->err = d_err;
  L->lad_on = 1;
  const int stage = nslice * (TC_BM * 128 + pl.bn * 128);
  const int smem = pl.stages * stage + 1024 + 256 + TC_EPI_WARPS * TC_STG_BYTES;
  tc_smem_attr(smem);
  const int grid = std::max(1, std::min(tiles, sm_count()));
  tc_gemm_kernel<true><<<grid, TC_THREADS, smem, st>>>(*L);
  delete L;
  return 1;
}

// ---- convenience: slice both operands of plain GemmProbs into `workspace`
namespace {
int prepare_sliced(const GemmProb* pin, int np_in, int nslice, bool exact,
                   void* workspace, TcProb* out, cudaStream_t st,
                   int* launches) {
  uint8_t* ws = (uint8_t*)workspace;
  int64_t off = 0;
  auto take = [&](int64_t bytes) {
    uint8_t* q = ws + off;
    off += (bytes + 1023) / 1024 * 1024;
    return q;
  };
  int np = 0;
  for (int i = 0; i < np_in; ++i) {
    const GemmProb& g = pin[i];
    if (g.M <= 0 || g.N <= 0) continue;
    const int Kp = slice_kp(g.K);
    TcProb t;
    std::memset(&t, 0, sizeof(t));
    t.C = g.C;
    t.M = g.M;
    t.N = g.N;
    t.K = g.K;
    t.ldc = g.ldc;
    void* da = take((int64_t)nslice * g.M * Kp * 2);
    void* db = take((int64_t)nslice * g.N * Kp * 2);
    int* ea = exact ? (int*)take((int64_t)g.M * 4) : nullptr;
    int* eb = exact ? (int*)take((int64_t)g.N * 4) : nullptr;
    // op(A)(m,k): A[m][k] (ta = 0) or A[k][m];  op(B)^T(n,k): B[n][k] (tb)
    // or B[k][n]
    if (exact) {
      *launches += split_exact(g.A, g.M, g.K, g.lda, g.ta, nslice, da, ea, st);
      *launches += split_exact(g.B, g.N, g.K, g.ldb, g.tb ? 0 : 1, nslice, db,
                               eb, st);
    } else {
      *launches += split_float(g.A, g.M, g.K, g.lda, g.ta, nslice, da, st);
      *launches += split_float(g.B, g.N, g.K, g.ldb, g.tb ? 0 : 1, nslice, db,
                               st);
    }
    t.a = {da, ea, g.M, Kp};
    t.b = {db, eb, g.N, Kp};
    out[np++] = t;
  }
  return np;
}
}  // namespace

int64_t sliced_workspace_bytes(const GemmProb* p, int np, int nslice,
                               bool exact) {
  int64_t b = 0;
  for (int i = 0; i < np; ++i) {
    if (p[i].M <= 0 || p[i].N <= 0) continue;
    const int64_t Kp = slice_kp(p[i].K);
    b += (int64_t)nslice * (p[i].M + p[i].N) * Kp * 2 + 4 * 1024;
    if (exact) b += (int64_t)(p[i].M + p[i].N) * 4;
  }
  return b + 1024;
}

int64_t tc_workspace_bytes(const GemmProb* p, int np, int nslice) {
  return sliced_workspace_bytes(p, np, nslice, false);
}

int64_t tc_scratch_doubles(const GemmProb* p, int np, int nslice) {
  TcProb t[TC_MAXPROB];
  int n = 0;
  for (int i = 0; i < np && n < TC_MAXPROB; ++i)
    if (p[i].M > 0 && p[i].N > 0) {
      std::memset(&t[n], 0, sizeof(TcProb));
      t[n].M = p[i].M;
      t[n].N = p[i].N;
      t[n].K = p[i].K;
      ++n;
    }
  return tc_plan(t, n, nslice).scratch;
}

int tc_gemm_grouped(const GemmProb* p, int np, double alpha, double beta,
                    int nslice, void* workspace, double* scratch,
                    unsigned int* d_err, cudaStream_t st) {
  TcProb t[TC_MAXPROB];
  int launches = 0;
  const int n = prepare_sliced(p, np, nslice, false, workspace, t, st,
                               &launches);
  return launches + tc_gemm_sliced(t, n, alpha, beta, nslice, scratch, d_err,
                                   st);
}

namespace {
// split-K partials of the exact-slice kernel for plain GemmProbs
int64_t oz_scratch_doubles(const GemmProb* p, int np) {
  TcProb t[TC_MAXPROB];
  int n = 0;
  for (int i = 0; i < np && n < TC_MAXPROB; ++i)
    if (p[i].M > 0 && p[i].N > 0) {
      std::memset(&t[n], 0, sizeof(TcProb));
      t[n].M = p[i].M;
      t[n].N = p[i].N;
      t[n].K = p[i].K;
      t[n].a.rows = p[i].M;
      t[n].b.rows = p[i].N;
      ++n;
    }
  return oz_sliced_scratch_doubles(t, n);
}

int64_t oz_slices_bytes(const GemmProb* p, int np, int nslice) {
  return (sliced_workspace_bytes(p, np, nslice, true) + 1023) / 1024 * 1024;
}
}  // namespace

int64_t oz_workspace_bytes(const GemmProb* p, int np, int nslice) {
  return oz_slices_bytes(p, np, nslice) + 8 * oz_scratch_doubles(p, np);
}

int oz_gemm_grouped(const GemmProb* p, int np, double alpha, double beta,
                    int nslice, void* workspace, unsigned int* d_err,
                    cudaStream_t st) {
  TcProb t[TC_MAXPROB];
  int launches = 0;
  const int n = prepare_sliced(p, np, nslice, true, workspace, t, st,
                               &launches);
  double* scratch =
      (double*)((uint8_t*)workspace + oz_slices_bytes(p, np, nslice));
  return launches +
         oz_gemm_sliced(t, n, alpha, beta, nslice, scratch, d_err, st);
}

}  // namespace cdcc
