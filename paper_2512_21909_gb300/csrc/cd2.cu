// cd2.cu -- symmetry-adapted two-step Cholesky decomposition of the ERI
// matrix (Sec. 3.2, Algorithm 1 and the second step, Eq. cv_2ndstep).
//
// The pair-integral matrix is block diagonal by the irrep of the basis
// pair; block G is given in factored form, (r|s) = B_G[r] . B_G[s]
// (B_G: npair(G) x naux(G), the integral source), and integral columns
// are evaluated from it with the FP64 GEMM.
//
// First step, per macro iteration: the host reads the current diagonals,
// keeps the list P (diagonal >= tau, not yet a pivot), and takes over all
// irreps the at most Q_max largest diagonals of P that reach
// sigma * D_max as candidates (ties: lower irrep, lower pair).  On the
// device, per irrep, the candidate columns minus the vectors found so far,
// Mt = B_Q B^T - L_Q^T L, come from two grouped FP64 GEMMs; then the micro
// iterations run as a fixed sequence of kernel pairs without host
// synchronisation: cd_pick (one CTA) takes the not-yet-pivoted candidate
// with the largest current diagonal, or ends the sequence once that is
// below tau_mic = max(tau, sigma * D_max); cd_update writes the new vector
// L^q_r = (Mt[q, r] - sum over this macro iteration's earlier vectors
// L^p_r L^p_q) / sqrt(D_q) for every pair r of q's irrep and
// D_r -= (L^q_r)^2.  The sums run in the same order as the oracle's.
//
// Second step, per irrep: the metric V = B_Q B_Q^T of the pivots is
// factored V = K K^T in place (df.cu) and the vectors are
// L = K^{-1} (B_Q B^T), one GEMM with (K^{-1})^T.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/cdcc.h"
#include "kernels.h"

namespace cdcc {

namespace {

constexpr int CD_MAXIRR = 8;

// rows of one irrep: D[r] = |B[r, :]|^2, a warp per row
__global__ void cd_diag_kernel(const double* __restrict__ B, int npair,
                               int naux, double* __restrict__ D) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // warps stride over the rows (the grid is capped at a few CTAs per SM)
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
       w < npair; w += nw) {
    const double* b = B + w * naux;
    double s = 0.0;
    for (int k = lane; k < naux; k += 32) s = fma(b[k], b[k], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) D[w] = s;
  }
}

// out[j, :] = B[idx[j], :]  (n rows of width w)
__global__ void cd_gather_rows_kernel(const double* __restrict__ B, int w,
                                      const int* __restrict__ idx, int n,
                                      double* __restrict__ out) {
  const int64_t total = (int64_t)n * w;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / w), k = (int)(e - (int64_t)j * w);
    out[e] = B[(int64_t)idx[j] * w + k];
  }
}

// out[p, j] = L[p, idx[j]]  (rows p < nrow of leading dimension ld)
__global__ void cd_gather_cols_kernel(const double* __restrict__ L,
                                      int64_t ld, int nrow,
                                      const int* __restrict__ idx, int n,
                                      double* __restrict__ out) {
  const int64_t total = (int64_t)nrow * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / n), j = (int)(e - (int64_t)p * n);
    out[e] = L[p * ld + idx[j]];
  }
}

// Per-irrep device state of one macro iteration.
struct CdIrrep {
  double* D[CD_MAXIRR];       // current diagonals
  unsigned char* taken[CD_MAXIRR];
  const double* Mt[CD_MAXIRR];  // [nq][npair]: candidate columns
  double* L[CD_MAXIRR];       // [capacity][npair]: vectors
  int npair[CD_MAXIRR];
  int ncv0[CD_MAXIRR];        // vectors before this macro iteration
};

// The pivot of one micro step (written by cd_pick, read by cd_update).
struct CdStep {
  int done;        // the micro iterations of this macro iteration ended
  int g, j, r, m;  // irrep, candidate index, pair, vector index in macro
  double dq;
  int count;       // pivots taken in this macro iteration
  int nmic[CD_MAXIRR];
};

constexpr int PICK_THREADS = 1024;

// One CTA: the not-yet-pivoted candidate with the largest diagonal (the
// first in candidate order on ties: candidates are sorted by irrep, then
// by their index in the irrep's candidate list), or the end of the
// sequence.  Records the pivot (irrep, pair) in piv_out.
__global__ void __launch_bounds__(PICK_THREADS)
    cd_pick_kernel(const __grid_constant__ CdIrrep S,
                   const int* __restrict__ cg, const int* __restrict__ cj,
                   const int* __restrict__ cr, int ncand, double tau_mic,
                   CdStep* st, int* __restrict__ piv_out) {
  if (st->done) return;
  __shared__ double bv[PICK_THREADS];
  __shared__ int bi[PICK_THREADS];
  const int t = threadIdx.x;
  double best = -1.0;
  int bidx = -1;
  for (int c = t; c < ncand; c += PICK_THREADS) {
    const int g = cg[c], r = cr[c];
    if (S.taken[g][r]) continue;
    const double d = S.D[g][r];
    if (bidx < 0 || d > best) {
      best = d;
      bidx = c;
    }
  }
  bv[t] = best;
  bi[t] = bidx;
  __syncthreads();
  for (int s = PICK_THREADS / 2; s > 0; s >>= 1) {
    if (t < s) {
      const int i2 = bi[t + s];
      // larger diagonal wins; equal diagonals: the earlier candidate
      if (i2 >= 0 && (bi[t] < 0 || bv[t + s] > bv[t] ||
                      (bv[t + s] == bv[t] && i2 < bi[t]))) {
        bv[t] = bv[t + s];
        bi[t] = i2;
      }
    }
    __syncthreads();
  }
  if (t == 0) {
    const int c = bi[0];
    if (c < 0 || bv[0] < tau_mic) {
      st->done = 1;
      return;
    }
    const int g = cg[c];
    st->g = g;
    st->j = cj[c];
    st->r = cr[c];
    st->m = st->nmic[g]++;
    st->dq = bv[0];
    S.taken[g][cr[c]] = 1;
    piv_out[2 * st->count] = g;
    piv_out[2 * st->count + 1] = cr[c];
    st->count += 1;
  }
}

// The new vector of the step's pivot for every pair of its irrep.
__global__ void cd_update_kernel(const __grid_constant__ CdIrrep S,
                                 const CdStep* __restrict__ st) {
  if (st->done) return;
  const int g = st->g;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = S.npair[g];
  if (r >= n) return;
  const int q = st->r, m = st->m;
  const double* Lb = S.L[g] + (int64_t)S.ncv0[g] * n;
  // product and difference rounded separately, as in the oracle
  double col = S.Mt[g][(int64_t)st->j * n + r];
  for (int p = 0; p < m; ++p)
    col = __dsub_rn(col, __dmul_rn(Lb[(int64_t)p * n + r],
                                   Lb[(int64_t)p * n + q]));
  const double l = col / sqrt(st->dq);
  S.L[g][((int64_t)S.ncv0[g] + m) * n + r] = l;
  S.D[g][r] = __dsub_rn(S.D[g][r], __dmul_rn(l, l));
}

struct CdError : std::runtime_error {
  cdcc_status status;
  CdError(cdcc_status s, const std::string& m)
      : std::runtime_error(m), status(s) {}
};

void cdk(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  (void)cudaGetLastError();
  if (e == cudaErrorMemoryAllocation)
    throw CdError(CDCC_ENOMEM, std::string(what) + ": out of device memory");
  throw CdError(CDCC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void launched(const char* what) { cdk(cudaGetLastError(), what); }

// Stream-ordered device buffers owned by one call (freed at its end).
class CdPool {
 public:
  explicit CdPool(cudaStream_t s) : st_(s) {}
  ~CdPool() {
    for (void* p : ptrs_) cudaFreeAsync(p, st_);
    cudaStreamSynchronize(st_);
  }
  template <class T>
  T* alloc(size_t n) {
    void* p = nullptr;
    cdk(cudaMallocAsync(&p, std::max<size_t>(n, 1) * sizeof(T), st_),
        "cudaMallocAsync");
    ptrs_.push_back(p);
    return (T*)p;
  }
  void release(void* p) {
    auto it = std::find(ptrs_.begin(), ptrs_.end(), p);
    if (it == ptrs_.end()) return;
    cudaFreeAsync(p, st_);
    ptrs_.erase(it);
  }

 private:
  cudaStream_t st_;
  std::vector<void*> ptrs_;
};

int grid_for(int64_t n, int threads) {
  return (int)std::max<int64_t>(
      1, std::min<int64_t>((n + threads - 1) / threads, 8 * (int64_t)sm_count()));
}

void gemm(std::vector<GemmProb>& probs, double alpha, double beta,
          CdPool& pool, cudaStream_t st) {
  for (size_t i = 0; i < probs.size(); i += GEMM_MAXPROB) {
    const int np = (int)std::min<size_t>(GEMM_MAXPROB, probs.size() - i);
    const int64_t ns = gemm_scratch_doubles(&probs[i], np);
    double* sk = ns > 0 ? pool.alloc<double>((size_t)ns) : nullptr;
    gemm64_grouped(&probs[i], np, alpha, beta, sk, st);
    launched("two-step CD GEMM");
    if (sk) pool.release(sk);
  }
}

struct CdResult {
  std::vector<std::vector<int>> piv;   // per irrep, in the order taken
  std::vector<double*> L;              // per irrep second-step vectors
  int macro = 0, micro = 0;
  double t_first = 0, t_second = 0;
};

// First step (Algorithm 1): the pivots of every irrep.
void first_step(int h, const std::vector<int>& npair,
                const std::vector<int>& naux,
                const std::vector<const double*>& B, double tau,
                double sigma, int qmax, cudaStream_t st, CdPool& pool,
                CdResult& res) {
  CdIrrep S;
  std::memset(&S, 0, sizeof(S));
  std::vector<std::vector<double>> Dh(h);
  std::vector<std::vector<char>> inP(h), taken(h);
  std::vector<int> ncv(h, 0), cap(h, 0);
  res.piv.assign(h, {});
  for (int g = 0; g < h; ++g) {
    const int n = npair[g];
    S.npair[g] = n;
    S.D[g] = pool.alloc<double>(n);
    S.taken[g] = pool.alloc<unsigned char>(n);
    cdk(cudaMemsetAsync(S.taken[g], 0, std::max(n, 1), st), "memset");
    if (n > 0) {
      cd_diag_kernel<<<grid_for((int64_t)n * 32, 256), 256, 0, st>>>(
          B[g], n, naux[g], S.D[g]);
      launched("cd_diag_kernel");
    }
    cap[g] = std::min(n, std::max(32, naux[g] + 8));
    S.L[g] = pool.alloc<double>((size_t)cap[g] * n);
    Dh[g].resize(n);
    inP[g].assign(n, 1);
    taken[g].assign(n, 0);
  }
  CdStep* d_step = pool.alloc<CdStep>(1);
  for (;;) {
    // current diagonals -> the list P and the candidates
    for (int g = 0; g < h; ++g)
      if (npair[g] > 0)
        cdk(cudaMemcpyAsync(Dh[g].data(), S.D[g], (size_t)npair[g] * 8,
                            cudaMemcpyDeviceToHost, st),
            "diagonal download");
    cdk(cudaStreamSynchronize(st), "sync");
    bool any = false;
    double dmax = 0.0;
    for (int g = 0; g < h; ++g)
      for (int r = 0; r < npair[g]; ++r) {
        inP[g][r] = inP[g][r] && !taken[g][r] && Dh[g][r] >= tau;
        if (inP[g][r]) {
          if (!std::isfinite(Dh[g][r]))
            throw CdError(CDCC_ENUMERIC, "two-step CD: non-finite diagonal");
          dmax = any ? std::max(dmax, Dh[g][r]) : Dh[g][r];
          any = true;
        }
      }
    if (!any) break;
    if (++res.macro > 100000)
      throw CdError(CDCC_ENUMERIC, "two-step CD: no progress");
    struct Cand {
      double d;
      int g, r;
    };
    std::vector<Cand> cand;
    for (int g = 0; g < h; ++g)
      for (int r = 0; r < npair[g]; ++r)
        if (inP[g][r] && Dh[g][r] >= sigma * dmax)
          cand.push_back({Dh[g][r], g, r});
    std::sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) {
      if (a.d != b.d) return a.d > b.d;
      if (a.g != b.g) return a.g < b.g;
      return a.r < b.r;
    });
    if ((int)cand.size() > qmax) cand.resize(qmax);
    std::vector<std::vector<int>> Q(h);
    for (const Cand& c : cand) Q[c.g].push_back(c.r);
    // candidate columns minus the vectors so far: Mt = B_Q B^T - L_Q^T L
    std::vector<double*> Mt(h, nullptr);
    std::vector<void*> tmp;
    std::vector<GemmProb> p1, p2;
    for (int g = 0; g < h; ++g) {
      const int nq = (int)Q[g].size(), n = npair[g];
      if (nq == 0) continue;
      if (ncv[g] + nq > cap[g]) {   // room for this macro's vectors
        const int nc = std::min(n, std::max(ncv[g] + nq, 2 * cap[g]));
        double* Ln = pool.alloc<double>((size_t)nc * n);
        if (ncv[g] > 0)
          cdk(cudaMemcpyAsync(Ln, S.L[g], (size_t)ncv[g] * n * 8,
                              cudaMemcpyDeviceToDevice, st),
              "vector copy");
        pool.release(S.L[g]);
        S.L[g] = Ln;
        cap[g] = nc;
      }
      int* d_idx = pool.alloc<int>(nq);
      tmp.push_back(d_idx);
      cdk(cudaMemcpyAsync(d_idx, Q[g].data(), (size_t)nq * 4,
                          cudaMemcpyHostToDevice, st),
          "candidate upload");
      double* Bq = pool.alloc<double>((size_t)nq * naux[g]);
      tmp.push_back(Bq);
      cd_gather_rows_kernel<<<grid_for((int64_t)nq * naux[g], 256), 256, 0,
                              st>>>(B[g], naux[g], d_idx, nq, Bq);
      launched("cd_gather_rows_kernel");
      Mt[g] = pool.alloc<double>((size_t)nq * n);
      tmp.push_back(Mt[g]);
      GemmProb a;
      std::memset(&a, 0, sizeof(a));
      a.A = Bq;
      a.lda = naux[g];
      a.B = B[g];
      a.tb = 1;
      a.ldb = naux[g];
      a.C = Mt[g];
      a.ldc = n;
      a.M = nq;
      a.N = n;
      a.K = naux[g];
      p1.push_back(a);
      if (ncv[g] > 0) {
        double* Lq = pool.alloc<double>((size_t)ncv[g] * nq);
        tmp.push_back(Lq);
        cd_gather_cols_kernel<<<grid_for((int64_t)ncv[g] * nq, 256), 256, 0,
                                st>>>(S.L[g], n, ncv[g], d_idx, nq, Lq);
        launched("cd_gather_cols_kernel");
        GemmProb b;
        std::memset(&b, 0, sizeof(b));
        b.A = Lq;
        b.ta = 1;
        b.lda = nq;
        b.B = S.L[g];
        b.ldb = n;
        b.C = Mt[g];
        b.ldc = n;
        b.M = nq;
        b.N = n;
        b.K = ncv[g];
        p2.push_back(b);
      }
    }
    gemm(p1, 1.0, 0.0, pool, st);
    gemm(p2, -1.0, 1.0, pool, st);
    // micro iterations: one (pick, update) pair per candidate, issued
    // without host synchronisation; the pairs after the end are no-ops
    std::vector<int> hc;
    int maxn = 1;
    for (int g = 0; g < h; ++g)
      for (int j = 0; j < (int)Q[g].size(); ++j) maxn = std::max(maxn, npair[g]);
    const int nc = (int)cand.size();
    for (int pass = 0; pass < 3; ++pass)
      for (int g = 0; g < h; ++g)
        for (int j = 0; j < (int)Q[g].size(); ++j)
          hc.push_back(pass == 0 ? g : pass == 1 ? j : Q[g][j]);
    int* d_c = pool.alloc<int>(3 * (size_t)nc);
    int* d_piv = pool.alloc<int>(2 * (size_t)nc);
    tmp.push_back(d_c);
    tmp.push_back(d_piv);
    cdk(cudaMemcpyAsync(d_c, hc.data(), hc.size() * 4, cudaMemcpyHostToDevice,
                        st),
        "candidate upload");
    for (int g = 0; g < h; ++g) {
      S.Mt[g] = Mt[g];
      S.ncv0[g] = ncv[g];
    }
    cdk(cudaMemsetAsync(d_step, 0, sizeof(CdStep), st), "memset");
    const double tau_mic = std::max(tau, sigma * dmax);
    for (int s = 0; s < nc; ++s) {
      cd_pick_kernel<<<1, PICK_THREADS, 0, st>>>(S, d_c, d_c + nc,
                                                 d_c + 2 * nc, nc, tau_mic,
                                                 d_step, d_piv);
      cd_update_kernel<<<(maxn + 255) / 256, 256, 0, st>>>(S, d_step);
    }
    launched("two-step CD micro iterations");
    CdStep hs;
    std::vector<int> hp(2 * (size_t)nc);
    cdk(cudaMemcpyAsync(&hs, d_step, sizeof(CdStep), cudaMemcpyDeviceToHost,
                        st),
        "step download");
    cdk(cudaMemcpyAsync(hp.data(), d_piv, hp.size() * 4,
                        cudaMemcpyDeviceToHost, st),
        "pivot download");
    cdk(cudaStreamSynchronize(st), "sync");
    if (hs.count <= 0 || hs.count > nc)
      throw CdError(CDCC_ENUMERIC, "two-step CD: a macro iteration took no "
                                   "pivot");
    for (int i = 0; i < hs.count; ++i) {
      const int g = hp[2 * i], r = hp[2 * i + 1];
      res.piv[g].push_back(r);
      taken[g][r] = 1;
    }
    for (int g = 0; g < h; ++g) ncv[g] += hs.nmic[g];
    res.micro += hs.count;
    for (void* p : tmp) pool.release(p);
  }
}

// Second step (Eq. cv_2ndstep): L = K^{-1} (B_Q B^T), V = B_Q B_Q^T = K K^T.
void second_step(int h, const std::vector<int>& npair,
                 const std::vector<int>& naux,
                 const std::vector<const double*>& B, cudaStream_t st,
                 CdPool& pool, CdResult& res) {
  res.L.assign(h, nullptr);
  MetricBlocks mb;
  std::memset(&mb, 0, sizeof(mb));
  std::vector<double*> Bq(h, nullptr);
  std::vector<GemmProb> pv, pc;
  std::vector<double*> C(h, nullptr);
  int64_t voff = 0;
  for (int g = 0; g < h; ++g) {
    mb.off[g] = voff;
    const int nq = (int)res.piv[g].size();
    mb.n[g] = nq;
    voff += (int64_t)nq * nq;
  }
  mb.nblk = h;
  double* V = pool.alloc<double>((size_t)std::max<int64_t>(voff, 1));
  double* Kit = pool.alloc<double>((size_t)std::max<int64_t>(voff, 1));
  for (int g = 0; g < h; ++g) {
    const int nq = (int)res.piv[g].size(), n = npair[g];
    res.L[g] = pool.alloc<double>((size_t)nq * n);
    if (nq == 0) continue;
    int* d_idx = pool.alloc<int>(nq);
    cdk(cudaMemcpyAsync(d_idx, res.piv[g].data(), (size_t)nq * 4,
                        cudaMemcpyHostToDevice, st),
        "pivot upload");
    Bq[g] = pool.alloc<double>((size_t)nq * naux[g]);
    cd_gather_rows_kernel<<<grid_for((int64_t)nq * naux[g], 256), 256, 0,
                            st>>>(B[g], naux[g], d_idx, nq, Bq[g]);
    launched("cd_gather_rows_kernel");
    GemmProb a;
    std::memset(&a, 0, sizeof(a));
    a.A = Bq[g];
    a.lda = naux[g];
    a.B = Bq[g];
    a.tb = 1;
    a.ldb = naux[g];
    a.C = V + mb.off[g];
    a.ldc = nq;
    a.M = nq;
    a.N = nq;
    a.K = naux[g];
    pv.push_back(a);
    C[g] = pool.alloc<double>((size_t)nq * n);
    GemmProb b = a;
    b.B = B[g];
    b.C = C[g];
    b.ldc = n;
    b.N = n;
    pc.push_back(b);
  }
  gemm(pv, 1.0, 0.0, pool, st);   // metric (Q|R)
  gemm(pc, 1.0, 0.0, pool, st);   // (Q|rs)
  unsigned int* d_err = pool.alloc<unsigned int>(1);
  cdk(cudaMemsetAsync(d_err, 0, 4, st), "memset");
  metric_factor(V, Kit, mb, d_err, st);
  launched("metric_factor");
  unsigned int herr = 0;
  cdk(cudaMemcpyAsync(&herr, d_err, 4, cudaMemcpyDeviceToHost, st),
      "status download");
  cdk(cudaStreamSynchronize(st), "sync");
  if (herr)
    throw CdError(CDCC_ENUMERIC,
                  "two-step CD: the pivots' metric is not positive definite");
  std::vector<GemmProb> pl;
  for (int g = 0; g < h; ++g) {
    const int nq = (int)res.piv[g].size(), n = npair[g];
    if (nq == 0) continue;
    GemmProb c;
    std::memset(&c, 0, sizeof(c));
    c.A = Kit + mb.off[g];   // (K^{-1})^T stored: op(A) = K^{-1}
    c.ta = 1;
    c.lda = nq;
    c.B = C[g];
    c.ldb = n;
    c.C = res.L[g];
    c.ldc = n;
    c.M = nq;
    c.N = n;
    c.K = nq;
    pl.push_back(c);
  }
  gemm(pl, 1.0, 0.0, pool, st);
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0)
      .count();
}

cdcc_status run_cd(int h, const int32_t* npair_in, const int32_t* naux_in,
                   const double* B_in, double tau, double sigma, int qmax,
                   int device, void* stream, int32_t* ncv_out,
                   int32_t* piv_out, int64_t piv_cap, double* L_out,
                   int64_t L_cap, double* stats) {
  if (h < 1 || h > CD_MAXIRR || !npair_in || !naux_in || !ncv_out)
    throw CdError(CDCC_EINVAL, "two-step CD: nirrep in 1..8 and the size "
                               "and count arrays are required");
  if (!(tau > 0.0) || !std::isfinite(tau) || !(sigma > 0.0) || sigma > 1.0 ||
      qmax < 1)
    throw CdError(CDCC_EINVAL, "two-step CD: tau > 0, 0 < sigma <= 1, "
                               "qmax >= 1");
  std::vector<int> npair(h), naux(h);
  int64_t nB = 0, nL = 0;
  for (int g = 0; g < h; ++g) {
    if (npair_in[g] < 0 || naux_in[g] < 0)
      throw CdError(CDCC_EINVAL, "two-step CD: negative size");
    npair[g] = npair_in[g];
    naux[g] = naux_in[g];
    nB += (int64_t)npair[g] * naux[g];
    nL += (int64_t)npair[g];
  }
  if (nB > 0 && !B_in)
    throw CdError(CDCC_EINVAL, "two-step CD: B is null");
  cdk(cudaSetDevice(device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  CdPool pool(st);
  const auto t0 = std::chrono::steady_clock::now();
  const double* dB = B_in;
  if (nB > 0 && !on_device(B_in)) {
    double* t = pool.alloc<double>((size_t)nB);
    cdk(cudaMemcpyAsync(t, B_in, (size_t)nB * 8, cudaMemcpyHostToDevice, st),
        "B upload");
    dB = t;
  }
  std::vector<const double*> B(h);
  int64_t off = 0;
  for (int g = 0; g < h; ++g) {
    B[g] = dB + off;
    off += (int64_t)npair[g] * naux[g];
  }
  CdResult res;
  first_step(h, npair, naux, B, tau, sigma, qmax, st, pool, res);
  cdk(cudaStreamSynchronize(st), "sync");
  res.t_first = seconds_since(t0);
  const auto t1 = std::chrono::steady_clock::now();
  second_step(h, npair, naux, B, st, pool, res);
  cdk(cudaStreamSynchronize(st), "sync");
  res.t_second = seconds_since(t1);
  int64_t npiv = 0, nvec = 0;
  for (int g = 0; g < h; ++g) {
    ncv_out[g] = (int32_t)res.piv[g].size();
    npiv += (int64_t)res.piv[g].size();
    nvec += (int64_t)res.piv[g].size() * npair[g];
  }
  if (stats) {
    stats[0] = res.macro;
    stats[1] = res.micro;
    stats[2] = res.t_first;
    stats[3] = res.t_second;
  }
  if (npiv > piv_cap || nvec > L_cap || (npiv > 0 && !piv_out) ||
      (nvec > 0 && !L_out))
    throw CdError(CDCC_ENOMEM, "two-step CD: output capacity too small (the "
                               "vector counts are in ncv)");
  // pivots (local pair indices), irrep blocks back to back
  std::vector<int32_t> hp;
  for (int g = 0; g < h; ++g)
    hp.insert(hp.end(), res.piv[g].begin(), res.piv[g].end());
  const bool pd = npiv > 0 && on_device(piv_out);
  const bool ld = nvec > 0 && on_device(L_out);
  if (npiv > 0)
    cdk(cudaMemcpyAsync(piv_out, hp.data(), (size_t)npiv * 4,
                        pd ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost,
                        st),
        "pivot copy");
  int64_t lo = 0;
  for (int g = 0; g < h; ++g) {
    const int64_t n = (int64_t)res.piv[g].size() * npair[g];
    if (n > 0)
      cdk(cudaMemcpyAsync(L_out + lo, res.L[g], (size_t)n * 8,
                          ld ? cudaMemcpyDeviceToDevice
                             : cudaMemcpyDeviceToHost,
                          st),
          "vector copy");
    lo += n;
  }
  cdk(cudaStreamSynchronize(st), "sync");
  (void)nL;
  return CDCC_OK;
}

}  // namespace

}  // namespace cdcc

extern "C" cdcc_status cdcc_cd_two_step(
    int nirrep, const int32_t* npair, const int32_t* naux, const double* B,
    double tau, double sigma, int qmax, int device, void* stream,
    int32_t* ncv, int32_t* piv, int64_t piv_cap, double* L, int64_t L_cap,
    double* stats, char* msg, int msg_len) {
  auto say = [&](const char* m) {
    if (msg && msg_len > 0) {
      std::strncpy(msg, m, (size_t)msg_len - 1);
      msg[msg_len - 1] = 0;
    }
  };
  say("");
  try {
    return cdcc::run_cd(nirrep, npair, naux, B, tau, sigma, qmax, device,
                        stream, ncv, piv, piv_cap, L, L_cap, stats);
  } catch (const cdcc::CdError& e) {
    say(e.what());
    return e.status;
  } catch (const std::bad_alloc&) {
    say("two-step CD: host allocation failed");
    return CDCC_ENOMEM;
  } catch (const std::exception& e) {
    say(e.what());
    return CDCC_EINVAL;
  }
}
