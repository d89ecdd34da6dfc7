// tc_ozaki.cu -- FP64-accurate GEMM on the BF16 tensor cores (sm_103a).
//
// Error-free slicing (in the spirit of the Ozaki scheme):
//   * every row r of op(A) is scaled by 2^-e_r (max |A[r,:]| < 2^e_r) and
//     every column c of op(B) by 2^-f_c, then cut into integer slices
//         A[r,k] = 2^e_r * sum_i A_i[r,k] 2^(-8-7i),
//     A_0 in [-256, 256] (8 bits), A_i in [-64, 64] (7 bits) for i >= 1;
//     the integers are exact in BF16.  With s slices 8 + 7(s-1) bits of
//     every element relative to its row maximum are kept (s = 4: 29 bits).
//   * C[r,c] = 2^(e_r+f_c) sum_d 2^(-16-7d) P_d,  P_d = sum_{i+j=d} A_i B_j,
//     products with d < s.  Each P_d accumulates in its own FP32 tensor-
//     memory accumulator and stays an exact integer below 2^24 for a K chunk
//     of 192 (|terms| <= 2^16 for d = 0, <= 2^15 + 2^13 per k for d > 0).
//   * after each chunk eight drain warps (two per TMEM sub-partition, each
//     owning 32 of the 64 columns) read the s accumulators (tcgen05.ld) and
//     add 2^(-16-7d) P_d into a per-thread double-float (hi, lo) FP32 pair
//     with error-free TwoSum, so the only rounding is the final 2^-48-level
//     one.  Two accumulator sets alternate so that the drain of chunk n
//     overlaps the MMAs of chunk n+1; the second warp on each sub-partition
//     computes while the first waits for its tensor-memory loads.
// Operands are staged by TMA (128B swizzle) through a 2-stage pipeline; one
// thread issues tcgen05.mma.kind::f16, s instructions per 16 of K (A_i
// against the stacked B slices, N = (s - i) * 64) instead of one per slice
// product.  Tile: 128 rows x 64 columns (the
// larger output dimension on the 128-row side); the kernel is persistent
// (one CTA per SM walks its tiles), so one tile's drain and write overlap
// the next tile's loads and MMAs.  Every mbarrier wait is bounded and sets
// the error flag on timeout.
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

constexpr int OZ_BM = 128, OZ_BN = 64, OZ_BK = 64;
constexpr int OZ_KBLK_PER_CHUNK = 3;        // exact FP32 chunk: 192 of K
constexpr int OZ_DRAIN_WARPS = 8;
constexpr int OZ_THREADS = 64 + 32 * OZ_DRAIN_WARPS;   // 10 warps
constexpr int OZ_MAXPROB = 8;
constexpr int OZ_MAXS = 4;
constexpr int OZ_STAGES = 2;
constexpr long long OZ_SPIN_LIMIT = 1LL << 22;

struct OzLaunch {
  CUtensorMap ta[OZ_MAXPROB];   // 128-row side slices {Kp, rows, s}
  CUtensorMap tb[OZ_MAXPROB];   // 64-col side slices {Kp, cols, s}
  const int* erow[OZ_MAXPROB];  // exponents of the 128-row side
  const int* ecol[OZ_MAXPROB];  // exponents of the column side
  double* C[OZ_MAXPROB];
  int M[OZ_MAXPROB], N[OZ_MAXPROB], ldc[OZ_MAXPROB], nkb[OZ_MAXPROB];
  int tm[OZ_MAXPROB], tn[OZ_MAXPROB];
  // split K: part kp of a tile takes the K blocks of chunks
  // [kp * cps, (kp + 1) * cps) and writes its unscaled FP64 partial to
  // scratch + poff + kp * M * N (logical row-major); oz_reduce_kernel adds
  // the parts in order
  int ks[OZ_MAXPROB], cps[OZ_MAXPROB];
  int64_t poff[OZ_MAXPROB];
  int tile0[OZ_MAXPROB + 1];   // counts (tile, part) pairs
  int np, nslice, trans_out;
  double alpha, beta;
  Pow2 ap2;                     // alpha as +-2^k (folded into the exponent)
  double* scratch;
  unsigned int* err;
};

struct OzReduce {
  double* C[OZ_MAXPROB];
  int M[OZ_MAXPROB], N[OZ_MAXPROB], ldc[OZ_MAXPROB], ks[OZ_MAXPROB];
  int64_t poff[OZ_MAXPROB], elem0[OZ_MAXPROB + 1];
  int np;
  double alpha, beta;
  const double* scratch;
};

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)),
               "r"(n)
               : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b))
               : "memory");
}

__device__ __forceinline__ void bar_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   su32(b)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity,
                                         unsigned int* err,
                                         unsigned int code) {
  const uint32_t a = su32(b);
  for (long long i = 0; i < OZ_SPIN_LIMIT; ++i) {
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

__device__ __forceinline__ void tma3(void* dst, const CUtensorMap* map,
                                     int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::"
      "complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(su32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void umma(uint32_t tmem, uint64_t ad, uint64_t bd,
                                     uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
          tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void ucommit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
      "[%0];" ::"r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void tld32(uint32_t taddr, float* v) {
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

// two 32-column loads (columns a.. and b..) behind one wait
__device__ __forceinline__ void tld32x2(uint32_t ta, uint32_t tb, float* v,
                                        float* w) {
  uint32_t r[32], q[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, "
      "[%64];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
      "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, "
      "[%65];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]),
        "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]),
        "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31]), "=r"(q[0]), "=r"(q[1]), "=r"(q[2]),
        "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
        "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]),
        "=r"(q[13]), "=r"(q[14]), "=r"(q[15]), "=r"(q[16]), "=r"(q[17]),
        "=r"(q[18]), "=r"(q[19]), "=r"(q[20]), "=r"(q[21]), "=r"(q[22]),
        "=r"(q[23]), "=r"(q[24]), "=r"(q[25]), "=r"(q[26]), "=r"(q[27]),
        "=r"(q[28]), "=r"(q[29]), "=r"(q[30]), "=r"(q[31])
      : "r"(ta), "r"(tb)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    v[i] = __uint_as_float(r[i]);
    w[i] = __uint_as_float(q[i]);
  }
}

// error-free (hi, lo) += v
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (v - bp);
  hi = s;
  lo += e;
}

// Work item t of the launch -> (problem, 128-row tile, 64-column tile,
// K blocks [kb0, kb1) of its split part).
__device__ __forceinline__ void oz_tile(const OzLaunch& L, int t, int& pi,
                                        int& m0, int& n0, int& kp, int& kb0,
                                        int& kb1) {
  pi = 0;
  while (pi + 1 < L.np && t >= L.tile0[pi + 1]) ++pi;
  const int local = t - L.tile0[pi];
  const int tile = local / L.ks[pi];
  kp = local - tile * L.ks[pi];
  m0 = (tile / L.tn[pi]) * OZ_BM;
  n0 = (tile % L.tn[pi]) * OZ_BN;
  kb0 = min(L.nkb[pi], kp * L.cps[pi] * OZ_KBLK_PER_CHUNK);
  kb1 = min(L.nkb[pi], kb0 + L.cps[pi] * OZ_KBLK_PER_CHUNK);
}

__global__ void oz_reduce_kernel(const __grid_constant__ OzReduce R) {
  const int64_t total = R.elem0[R.np];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int pi = 0;
    while (pi + 1 < R.np && e >= R.elem0[pi + 1]) ++pi;
    const int64_t loc = e - R.elem0[pi];
    const int m = (int)(loc / R.N[pi]), n = (int)(loc - (int64_t)m * R.N[pi]);
    const int64_t MN = (int64_t)R.M[pi] * R.N[pi];
    const double* part = R.scratch + R.poff[pi] + loc;
    double acc = 0.0;
    for (int k = 0; k < R.ks[pi]; ++k) acc += part[k * MN];
    double* c = R.C[pi] + (int64_t)m * R.ldc[pi] + n;
    const double v = R.alpha * acc;
    *c = (R.beta == 0.0) ? v : fma(R.beta, *c, v);
  }
}

// Persistent: CTA b takes tiles b, b + gridDim.x, ...  The three roles walk
// the same tile sequence with running counters (K blocks for the smem
// stages, K chunks for the two accumulator sets), so the loads and MMAs of
// the next tile proceed while the drain warps finish and write this one.
__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_gemm_kernel(const __grid_constant__ OzLaunch L) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int s = L.nslice;
  constexpr uint32_t A_BYTES = OZ_BM * 128, B_BYTES = OZ_BN * 128;
  const uint32_t stage_bytes = (uint32_t)s * (A_BYTES + B_BYTES);
  uint64_t* full = (uint64_t*)(smem + (size_t)OZ_STAGES * stage_bytes);
  uint64_t* empty = full + OZ_STAGES;
  uint64_t* accf = empty + OZ_STAGES;   // [2] accumulator set ready
  uint64_t* acce = accf + 2;            // [2] accumulator set drained
  uint64_t* fin = acce + 2;             // all MMAs of this CTA complete
  uint32_t* tmem_slot = (uint32_t*)(fin + 1);
  int* consumed = (int*)(tmem_slot + 1);   // K blocks the MMA side used
  // per drain warp a 32 x 16 staging tile (XOR-swizzled columns) for
  // coalesced writes of C
  double* stage_out =
      (double*)(smem + (size_t)OZ_STAGES * stage_bytes + 256);

  const int ntile = L.tile0[L.np];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t NCOLS = 512;   // two sets of s (<= 4) x 64 columns

  if (threadIdx.x == 0) {
    for (int i = 0; i < OZ_STAGES; ++i) {
      bar_init(&full[i], 1);
      bar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      bar_init(&accf[i], 1);
      bar_init(&acce[i], OZ_DRAIN_WARPS);   // one arrive per drain warp
    }
    bar_init(fin, 1);
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], "
        "%1;" ::"r"(su32(tmem_slot)),
        "r"(NCOLS)
        : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  // F32 accumulate, BF16 A and B, both K-major, M = 128; N is or-ed in
  // per instruction
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                         ((uint32_t)(OZ_BM >> 4) << 24);
  int issued = 0;   // producer: K blocks whose loads were issued

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      int g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
        int pi, m0, n0, kp, kbb, kbe;
        oz_tile(L, t, pi, m0, n0, kp, kbb, kbe);
        for (int kb = kbb; kb < kbe; ++kb, ++g) {
          const int st = g % OZ_STAGES, round = g / OZ_STAGES;
          if (round > 0 && !bar_wait(&empty[st], (round - 1) & 1, L.err, 11)) {
            ok = false;
            break;
          }
          bar_expect(&full[st], stage_bytes);
          uint8_t* sa = smem + (size_t)st * stage_bytes;
          uint8_t* sb = sa + (size_t)s * A_BYTES;
          for (int i = 0; i < s; ++i) {
            tma3(sa + (size_t)i * A_BYTES, &L.ta[pi], kb * OZ_BK, m0, i,
                 &full[st]);
            tma3(sb + (size_t)i * B_BYTES, &L.tb[pi], kb * OZ_BK, n0, i,
                 &full[st]);
          }
          issued = g + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer: chunk c -> accumulator set c & 1
      bool ok = true;
      int g = 0, c = 0;
      for (int t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
        int pi, m0, n0, kp, kbb, kbe;
        oz_tile(L, t, pi, m0, n0, kp, kbb, kbe);
        const int nch =
            (kbe - kbb + OZ_KBLK_PER_CHUNK - 1) / OZ_KBLK_PER_CHUNK;
        for (int ch = 0; ch < nch && ok; ++ch, ++c) {
          const int set = c & 1;
          if (c >= 2 &&
              !bar_wait(&acce[set], ((c >> 1) - 1) & 1, L.err, 12)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int kb0 = kbb + ch * OZ_KBLK_PER_CHUNK;
          const int kb1 = min(kbe, kb0 + OZ_KBLK_PER_CHUNK);
          for (int kb = kb0; kb < kb1; ++kb, ++g) {
            const int st = g % OZ_STAGES, round = g / OZ_STAGES;
            if (!bar_wait(&full[st], round & 1, L.err, 13)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = su32(smem + (size_t)st * stage_bytes);
            const uint32_t sb = sa + (uint32_t)s * A_BYTES;
            // B_0 .. B_{s-1} lie back to back in the stage, i.e. one
            // operand of s*64 rows: A_i times its first (s-i)*64 rows,
            // written from column block i on, adds A_i B_j to block i+j = d
            // for every j at once.  The i = 0 product covers all s blocks,
            // so it alone starts a chunk's accumulation.
#pragma unroll
            for (int kk = 0; kk < OZ_BK / 16; ++kk) {
              for (int i = 0; i < s; ++i) {
                const uint32_t acc_addr =
                    tmem + (uint32_t)((set * s + i) * OZ_BN);
                const uint32_t nn = (uint32_t)((s - i) * OZ_BN);
                umma(acc_addr, sdesc(sa + i * A_BYTES + kk * 32),
                     sdesc(sb + kk * 32), idesc | ((nn >> 3) << 17),
                     (kb == kb0 && kk == 0 && i == 0) ? 0u : 1u);
              }
            }
            ucommit(&empty[st]);
            *(volatile int*)consumed = g + 1;
          }
          if (!ok) break;
          ucommit(&accf[set]);
        }
      }
      ucommit(fin);   // arrives once every MMA issued above has completed
    }
  } else {
    // ---- drain warps 2..9: TMEM sub-partition (warp % 4), 32 rows each;
    // warps 2..5 own columns 0..31 of the tile, warps 6..9 columns 32..63
    constexpr int HW = OZ_BN / 2;
    const int sub = warp & 3;
    const int half = (warp - 2) >> 2;
    bool ok = true;
    int c = 0;
    for (int t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
      int pi, m0, n0, kp, kbb, kbe;
      oz_tile(L, t, pi, m0, n0, kp, kbb, kbe);
      const int nch = (kbe - kbb + OZ_KBLK_PER_CHUNK - 1) / OZ_KBLK_PER_CHUNK;
      float hi[HW], lo[HW];
#pragma unroll
      for (int i = 0; i < HW; ++i) hi[i] = lo[i] = 0.f;
      for (int ch = 0; ch < nch; ++ch, ++c) {
        const int set = c & 1;
        if (!bar_wait(&accf[set], (c >> 1) & 1, L.err, 14)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t tbase = tmem + ((uint32_t)(sub * 32) << 16) +
                               (uint32_t)(set * s * OZ_BN + half * HW);
        // s is 2, 3 or 4: accumulators d and d + 1 behind one wait
        for (int d = 0; d < s; d += 2) {
          float v[32], w[32];
          const int d1 = d + 1 < s ? d + 1 : d;
          tld32x2(tbase + (uint32_t)(d * OZ_BN),
                  tbase + (uint32_t)(d1 * OZ_BN), v, w);
          const float sc = exp2f(-16.0f - 7.0f * d);
#pragma unroll
          for (int q = 0; q < 32; ++q) two_sum_add(hi[q], lo[q], v[q] * sc);
          if (d1 != d) {
            const float sc1 = sc * (1.0f / 128.0f);
#pragma unroll
            for (int q = 0; q < 32; ++q)
              two_sum_add(hi[q], lo[q], w[q] * sc1);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) bar_arrive(&acce[set]);
      }
      if (!ok) break;
      // ---- write: row r of the 128-row side, this warp's 32 columns.  With
      // the logical rows on that side (trans_out = 0) the warp passes 32 x 16
      // sub-tiles through shared memory so that lanes run along n.
      const int r = m0 + sub * 32 + lane;
      const int nb = n0 + half * HW;
      const int Mr = L.trans_out ? L.N[pi] : L.M[pi];
      const int Nc = L.trans_out ? L.M[pi] : L.N[pi];
      const int er = r < Mr ? L.erow[pi][r] : 0;
      // split K: the unscaled partial goes to this part's scratch slab
      // (logical M x N, row-major; put() takes logical coordinates)
      const bool part = L.ks[pi] > 1;
      double* C = part ? L.scratch + L.poff[pi] +
                             (int64_t)kp * L.M[pi] * L.N[pi]
                       : L.C[pi];
      const int ldc = part ? L.N[pi] : L.ldc[pi];
      // value 2^(sh) (hi + lo) as FP64: both halves converted with integer
      // operations (scale folded into the exponent), one FP64 addition
      const int ash = (L.ap2.ok && !part) ? L.ap2.sh : 0;
      auto value = [&](float h, float l, int sh) {
        const double v = f32_to_f64_scaled(h, sh + ash) +
                         f32_to_f64_scaled(l, sh + ash);
        if (part) return v;
        if (L.ap2.ok) return L.ap2.neg ? -v : v;
        return L.alpha * v;
      };
      auto put = [&](int m, int n, double out) {
        double* p = C + (int64_t)m * ldc + n;
        if (part || L.beta == 0.0)
          *p = out;
        else if (L.beta == 1.0)
          *p += out;
        else
          *p = fma(L.beta, *p, out);
      };
      if (L.trans_out) {
        if (r < Mr) {
#pragma unroll
          for (int q = 0; q < HW; ++q) {
            const int cc = nb + q;
            if (cc < Nc)
              put(cc, r, value(hi[q], lo[q], er + L.ecol[pi][cc]));
          }
        }
      } else {
        // element (row, col) of the 32 x 16 tile sits at
        // row * 16 + (col ^ (row & 15)): a row written by one lane and a
        // row read by 16 lanes both touch 16 distinct bank pairs
        double* stg = stage_out + (warp - 2) * (32 * 16);
#pragma unroll
        for (int h = 0; h < HW; h += 16) {
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int cc = nb + h + j;
            const int ec = cc < Nc ? L.ecol[pi][cc] : 0;
            stg[lane * 16 + (j ^ (lane & 15))] =
                value(hi[h + j], lo[h + j], er + ec);
          }
          __syncwarp();
#pragma unroll 4
          for (int rr = 0; rr < 32; rr += 2) {
            const int row = rr + (lane >> 4), col = lane & 15;
            const int m = m0 + sub * 32 + row, n = nb + h + col;
            if (m < Mr && n < Nc)
              put(m, n, stg[row * 16 + (col ^ (row & 15))]);
          }
        }
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
      bar_wait(&full[g % OZ_STAGES], (g / OZ_STAGES) & 1, L.err, 15);
  }
  if (warp == 1) {
    if (lane == 0) bar_wait(fin, 0, L.err, 16);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(
                     tmem),
                 "r"(NCOLS)
                 : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 oz_encode = nullptr;
std::once_flag oz_once;

void oz_encode_init() {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                       cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    fn = nullptr;
  oz_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
}

void oz_map(CUtensorMap* m, const __nv_bfloat16* base, int Kp, int rows, int s,
            int box_rows) {
  std::call_once(oz_once, oz_encode_init);
  if (!oz_encode) throw std::runtime_error("cuTensorMapEncodeTiled missing");
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)s};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * rows};
  cuuint32_t box[3] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows, 1};
  cuuint32_t est[3] = {1, 1, 1};
  CUresult r = oz_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base,
                         dims, strides, box, est,
                         CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw std::runtime_error("cuTensorMapEncodeTiled failed: " +
                             std::to_string((int)r));
}

bool oz_swap(const TcProb* p, int np) {
  int64_t sm = 0, sn = 0;
  for (int i = 0; i < np; ++i) {
    sm += p[i].M;
    sn += p[i].N;
  }
  return sn > sm;
}

}  // namespace

namespace {

// Split-K plan: when the output tiles of all products cannot fill the SMs,
// a product with at least four K chunks is cut into parts of whole chunks
// (at least two per part), as many as fill the SMs.  Depends only on the
// shapes and the SM count.
struct OzPlan {
  int ks[OZ_MAXPROB], cps[OZ_MAXPROB];
  int64_t scratch;   // doubles
};

OzPlan oz_plan(const TcProb* p, int np) {
  OzPlan pl;
  std::memset(&pl, 0, sizeof(pl));
  const bool swap = oz_swap(p, np);
  int64_t tiles = 0;
  for (int i = 0; i < np; ++i) {
    const int rows = swap ? p[i].b.rows : p[i].a.rows;
    const int cols = swap ? p[i].a.rows : p[i].b.rows;
    tiles += (int64_t)((rows + OZ_BM - 1) / OZ_BM) * ((cols + OZ_BN - 1) / OZ_BN);
  }
  const int sms = sm_count();
  for (int i = 0; i < np; ++i) {
    const int nkb = (p[i].K + OZ_BK - 1) / OZ_BK;
    const int nch = (nkb + OZ_KBLK_PER_CHUNK - 1) / OZ_KBLK_PER_CHUNK;
    int ks = 1;
    if (tiles > 0 && tiles < sms && nch >= 4) {
      ks = (int)std::min<int64_t>((sms + tiles - 1) / tiles, nch / 2);
      ks = std::max(1, std::min(ks, 64));
    }
    pl.cps[i] = ks > 1 ? (nch + ks - 1) / ks : std::max(nch, 1);
    pl.ks[i] = ks > 1 ? (nch + pl.cps[i] - 1) / pl.cps[i] : 1;
    if (pl.ks[i] > 1)
      pl.scratch += (int64_t)pl.ks[i] * p[i].M * p[i].N;
  }
  return pl;
}

}  // namespace

int64_t oz_sliced_scratch_doubles(const TcProb* p, int np) {
  if (np <= 0) return 0;
  if (np > OZ_MAXPROB) throw std::runtime_error("oz: too many blocks");
  return oz_plan(p, np).scratch;
}

int oz_gemm_sliced(const TcProb* p, int np, double alpha, double beta,
                   int nslice, double* scratch, unsigned int* d_err,
                   cudaStream_t st) {
  if (np <= 0) return 0;
  if (np > OZ_MAXPROB) throw std::runtime_error("oz: too many blocks");
  if (nslice < 2 || nslice > OZ_MAXS) throw std::runtime_error("oz: nslice");
  const bool swap = oz_swap(p, np);
  const OzPlan pl = oz_plan(p, np);
  if (pl.scratch > 0 && !scratch)
    throw std::runtime_error("oz: split-K scratch missing");
  OzLaunch* L = new OzLaunch;
  std::memset(L, 0, sizeof(OzLaunch));
  OzReduce R;
  std::memset(&R, 0, sizeof(R));
  int64_t poff = 0, relem = 0;
  int nr = 0;
  int tiles = 0;
  for (int i = 0; i < np; ++i) {
    const TcProb& g = p[i];
    const SlicedOp& rowop = swap ? g.b : g.a;
    const SlicedOp& colop = swap ? g.a : g.b;
    oz_map(&L->ta[i], (const __nv_bfloat16*)rowop.data, rowop.Kp, rowop.rows,
           nslice, OZ_BM);
    oz_map(&L->tb[i], (const __nv_bfloat16*)colop.data, colop.Kp, colop.rows,
           nslice, OZ_BN);
    L->erow[i] = rowop.exps;
    L->ecol[i] = colop.exps;
    L->C[i] = g.C;
    L->M[i] = g.M;
    L->N[i] = g.N;
    L->ldc[i] = g.ldc;
    L->nkb[i] = (g.K + OZ_BK - 1) / OZ_BK;
    L->tm[i] = (rowop.rows + OZ_BM - 1) / OZ_BM;
    L->tn[i] = (colop.rows + OZ_BN - 1) / OZ_BN;
    L->ks[i] = pl.ks[i];
    L->cps[i] = pl.cps[i];
    L->poff[i] = pl.ks[i] > 1 ? poff : 0;
    L->tile0[i] = tiles;
    tiles += L->tm[i] * L->tn[i] * L->ks[i];
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
  L->trans_out = swap ? 1 : 0;
  L->alpha = alpha;
  L->beta = beta;
  L->ap2 = pow2_of(alpha);
  L->scratch = scratch;
  L->err = d_err;
  const int stage = nslice * (OZ_BM * 128 + OZ_BN * 128);
  // stages, barriers, and one 32 x 16 double staging tile per drain warp
  const int smem = OZ_STAGES * stage + 1024 + 256 + OZ_DRAIN_WARPS * 32 * 16 * 8;
  // the attribute is shared by every thread and stream: set once, to the
  // largest launch (four slices), never lowered by a concurrent smaller one
  constexpr int OZ_SMEM_MAX = OZ_STAGES * OZ_MAXS * (OZ_BM * 128 + OZ_BN * 128) +
                              1024 + 256 + OZ_DRAIN_WARPS * 32 * 16 * 8;
  if (smem > OZ_SMEM_MAX) throw std::runtime_error("oz: shared memory plan");
  {
    static std::once_flag once[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    std::call_once(once[dev], [] {
      cudaFuncSetAttribute(oz_gemm_kernel,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           OZ_SMEM_MAX);
    });
  }
  // persistent: one CTA per SM (at most one fits), tiles strided over them
  const int grid = std::max(1, std::min(tiles, sm_count()));
  oz_gemm_kernel<<<grid, OZ_THREADS, smem, st>>>(*L);
  delete L;
  if (nr == 0) return 1;
  R.np = nr;
  R.elem0[nr] = relem;
  R.alpha = alpha;
  R.beta = beta;
  R.scratch = scratch;
  const int blocks = (int)std::min<int64_t>((relem + 255) / 256, 4096);
  oz_reduce_kernel<<<std::max(blocks, 1), 256, 0, st>>>(R);
  return 2;
}

}  // namespace cdcc
