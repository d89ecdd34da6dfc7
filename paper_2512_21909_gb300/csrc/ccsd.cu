// ccsd.cu -- closed-shell CD-CCSD residual, Lambda and density on the GPU,
// and the C ABI of include/cdcc.h.
//
// Amplitude equations (T1-dressed form).  With t_ai = t1[i,a], the
// similarity-transformed Hamiltonian exp(-T1) H exp(T1) has Cholesky vectors
// Lhat^P = (1 - t) L^P (1 + t) (the t1-contracted intermediates t^P_ia,
// t^P_ai, t^P_ij, t^P_ab of App. A folded into one dressed vector) and
// one-electron part (1-t) h (1+t).  The residuals are the projections
//     R1[i,a]     = < Phi_{i alpha}^{a alpha} | exp(-T) H exp(T) | 0 >
//     R2[i,j,a,b] = < Phi_{i alpha j beta}^{a alpha b beta} | ... | 0 >
// written with Cholesky-built integrals (Sec. 2.1 Eq. 1); the particle-
// particle ladder (Sec. 2.3) uses (ac|bd) = sum_P Lhat^P_ac Lhat^P_bd.
//
// Lambda (Sec. 2.3): with Lag = E + l1.R1 + l2.R2 (Sec. 2.2), the Lambda
// equations dLag/dt = 0 are solved by Jacobi/DIIS; dLag/dt is the reverse
// (adjoint) sweep of the recorded residual, i.e. the transpose of every
// residual contraction, evaluated with the t-dependent intermediates stored
// once (they do not depend on lambda).
//
// Densities (Sec. 2.4, 2.6): Gamma^P_pq = dLag/dL^P_pq and D_pq = dLag/dh_pq
// are one more reverse sweep with respect to the Cholesky vectors and h; the
// vvvv part of the density is contracted on the fly with the Cholesky vectors
// (the adjoint of the ladder), never stored as Gamma_abcd.
// Gradient (Sec. 2.1 Eq. 2 + Sec. 2.6): g_x = sum_P sum_pq Gamma^P_pq dL_x^P_pq.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/cdcc.h"
#include "engine.h"
#include "kernels.h"

using namespace cdcc;

namespace {

struct HostDims {
  int h, nocc, nvir, n, nchol;
};

// dense index of local index l of irrep g in space s
inline int64_t dense_index(const Dims& d, int s, int g, int l, int nocc) {
  switch (s) {
    case SO:
    case SV:
    case SQ:
      return d.gstart[s][g] + l;
    default:  // SA: orbital index
      if (l < d.n[SO][g]) return d.gstart[SO][g] + l;
      return nocc + d.gstart[SV][g] + (l - d.n[SO][g]);
  }
}

inline int64_t dense_dim(const Dims& d, int s) {
  if (s == SA) return d.total(SO) + d.total(SV);
  return d.total(s);
}

// Visit every stored element of a DPD layout with its dense row-major index.
template <class F>
void visit_dense(const Layout& L, const Dims& d, F f) {
  const int nocc = d.total(SO);
  int64_t dd[MAXRANK];
  for (int q = 0; q < L.rank; ++q) dd[q] = dense_dim(d, L.sp[q]);
  for_each_tuple(d.h, L.rank, L.gtot, [&](const int* g) {
    SubBlock sb = sub_block(L, d, g);
    if (sb.empty) return;
    int64_t n = 1;
    for (int q = 0; q < L.rank; ++q) n *= sb.dim[q];
    for (int64_t e = 0; e < n; ++e) {
      int64_t r = e, off = sb.base, dense = 0;
      int l[MAXRANK];
      for (int q = L.rank - 1; q >= 0; --q) {
        l[q] = (int)(r % sb.dim[q]);
        r /= sb.dim[q];
        off += l[q] * sb.stride[q];
      }
      for (int q = 0; q < L.rank; ++q)
        dense = dense * dd[q] + dense_index(d, L.sp[q], g[q], l[q], nocc);
      f(off, dense);
    }
  });
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Separable denominators of an amplitude layout for the Jacobi step.
struct Denom2D {
  Block2D* blocks = nullptr;
  Chunk2D* chunks = nullptr;
  double *rv = nullptr, *cv = nullptr;
  int nblk = 0, nchunk = 0;
  int64_t nrv = 0, ncv = 0;
};

struct Diis {
  int dim = 0, count = 0, next = 0;
  int64_t n = 0;
  std::vector<Tensor*> x, e;
  std::vector<double> B;  // dim x dim
};

}  // namespace

struct cdcc_ctx {
  cdcc_options opt;
  Dims dims;
  HostDims hd;
  std::vector<int> orb_irrep, chol_irrep;
  std::vector<double> eps;
  cudaStream_t st = 0;
  std::unique_ptr<Engine> eng;
  std::string err;
  int state = 0;  // 1 init, 2 ccsd, 3 lambda, 4 density
  bool tape_ready = false;
  // the engine's intermediates hold an accurate residual evaluation at the
  // current amplitudes (set when CCSD converges), so recording the tape
  // needs no second evaluation
  bool fwd_fresh = false;
  // c->res holds the accurate residual at the converged amplitudes
  bool res_acc = false;
  double e_corr = 0, e_ref = 0;
  int64_t nnz0 = 0;
  double* d_eps = nullptr;
  unsigned long long* d_max = nullptr;
  double* d_dots = nullptr;
  double* d_partial = nullptr;
  int64_t partial_n = 0;
  double phase[4] = {0, 0, 0, 0};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // tensors
  Tensor *Lpk = nullptr, *Loo, *Lov, *Lvo, *Lvv;
  Tensor *hoo, *hov, *hvo, *hvv, *Ioo;
  Tensor *amp, *T1, *T2, *res, *R1, *R2, *err1, *lam, *L1, *L2, *E;
  Tensor *Gam = nullptr, *Gsym = nullptr, *D1a = nullptr, *D1s = nullptr;
  Tensor *Govov = nullptr, *Govvv = nullptr, *W0 = nullptr, *Xe = nullptr;
  Diis cc_diis, lam_diis;
  Denom2D den[2];   // T1, T2 layouts
  unsigned int* d_err = nullptr;
  int iters_mixed[2] = {0, 0}, iters_fp64[2] = {0, 0};
  bool otf = false;   // ladder assembled on the fly (no stored W0)
  int z_iters = 0;    // conjugate-gradient iterations of the Z-vector solve
};

namespace {

#define CK(x)                                                              \
  do {                                                                     \
    cudaError_t e_ = (x);                                                  \
    if (e_ != cudaSuccess)                                                 \
      throw EngineError(std::string("CUDA: ") + cudaGetErrorString(e_) +  \
                        " at " #x);                                        \
  } while (0)

struct StatusError : std::exception {
  cdcc_status s;
  std::string m;
  StatusError(cdcc_status s_, std::string m_) : s(s_), m(std::move(m_)) {}
};

void copy_in(cdcc_ctx* c, double* dst, const double* src, int64_t n) {
  if (n <= 0) return;
  CK(cudaMemcpyAsync(dst, src, (size_t)n * 8,
                     is_device_ptr(src) ? cudaMemcpyDeviceToDevice
                                        : cudaMemcpyHostToDevice,
                     c->st));
}

std::vector<double> to_host(cdcc_ctx* c, const Tensor* t) {
  std::vector<double> h((size_t)std::max<int64_t>(t->lay.size, 0));
  if (!h.empty())
    CK(cudaMemcpyAsync(h.data(), t->d, h.size() * 8, cudaMemcpyDeviceToHost,
                       c->st));
  CK(cudaStreamSynchronize(c->st));
  return h;
}

void upload_dense(cdcc_ctx* c, Tensor* t, const std::vector<double>& dense) {
  std::vector<double> p((size_t)t->lay.size, 0.0);
  visit_dense(t->lay, c->dims, [&](int64_t off, int64_t di) {
    p[off] = dense[di];
  });
  CK(cudaMemcpyAsync(t->d, p.data(), p.size() * 8, cudaMemcpyHostToDevice,
                     c->st));
  CK(cudaStreamSynchronize(c->st));
}

// ------------------------------------------------------------------ prepare
// Amplitude-independent integrals, built once per gradient (and recorded at
// the head of the tape so that the density sweep differentiates them):
//   (ia|jb), (mc|bd) and the undressed ladder integrals W0[a,b,c,d]=(ac|bd).
void prepare(cdcc_ctx* c) {
  Engine& e = *c->eng;
  c->Govov = e.tensor("Govov", {SO, SV, SO, SV}, 2);
  e.contract(1.0, c->Lov, "Pia", c->Lov, "Pjb", 0.0, c->Govov, "iajb");
  // (mc|bd) stored with rows (m,b) and columns (c,d): its products with
  // the amplitudes (sums over c,d or over m,b) are then direct GEMMs
  c->Govvv = e.tensor("Govvv", {SO, SV, SV, SV}, 2);
  e.contract(1.0, c->Lov, "Pmc", c->Lvv, "Pbd", 0.0, c->Govvv, "mbcd");
  c->Govov->symmetric = true;   // (ia|jb) is a symmetric matrix per block
  c->Govov->constant = c->Govvv->constant = true;
  // 2 (ia|jb) - (ib|ja) of the energy expression, also amplitude independent
  c->Xe = e.tensor("Xe", {SO, SV, SO, SV}, 2);
  e.axpy(2.0, c->Govov, "iajb", 0.0, c->Xe, "iajb");
  e.axpy(-1.0, c->Govov, "ibja", 1.0, c->Xe, "iajb");
  c->Xe->constant = true;
  if (c->otf) return;           // the ladder builds its integrals itself
  c->W0 = e.tensor("W0", {SV, SV, SV, SV}, 2);
  e.contract(1.0, c->Lvv, "Pac", c->Lvv, "Pbd", 0.0, c->W0, "abcd");
  // W0[(ab),(cd)] = (ac|bd) is a symmetric matrix per block
  c->W0->symmetric = true;
  c->W0->constant = true;
  c->W0->ladder = true;
}

// ------------------------------------------------------------------ residual
// Forward evaluation of E, R1, R2 at the amplitudes in c->amp.  Every line is
// one engine primitive so that the same code, recorded, yields the adjoints.
void residual(cdcc_ctx* c) {
  Engine& e = *c->eng;
  // intermediates: written only by the engine operations below, so their
  // permuted copies can be reused while they do not change
  auto T = [&](const char* n, std::vector<int> sp, int split) {
    Tensor* t = e.tensor(n, sp, split);
    t->cacheable = true;
    return t;
  };
  Tensor *T1 = c->T1, *T2 = c->T2;
  Tensor *Loo = c->Loo, *Lov = c->Lov, *Lvo = c->Lvo, *Lvv = c->Lvv;

  // symmetrised doubles  t2s = (t2 + t2^swap) / 2
  Tensor* t2s = T("t2s", {SO, SO, SV, SV}, 2);
  e.axpy(0.5, T2, "ijab", 0.0, t2s, "ijab");
  e.axpy(0.5, T2, "jiba", 1.0, t2s, "ijab");

  // T1 dressing of the Cholesky vectors and of h
  Tensor* Lhoo = T("Lhoo", {SQ, SO, SO}, 1);
  e.axpy(1.0, Loo, "Pij", 0.0, Lhoo, "Pij");
  e.contract(1.0, Lov, "Pia", T1, "ja", 1.0, Lhoo, "Pij");
  Tensor* Lhvv = T("Lhvv", {SQ, SV, SV}, 1);
  e.axpy(1.0, Lvv, "Pab", 0.0, Lhvv, "Pab");
  e.contract(-1.0, T1, "ia", Lov, "Pib", 1.0, Lhvv, "Pab");
  Tensor* Lhvo = T("Lhvo", {SQ, SV, SO}, 1);
  e.axpy(1.0, Lvo, "Pai", 0.0, Lhvo, "Pai");
  e.contract(1.0, Lvv, "Pab", T1, "ib", 1.0, Lhvo, "Pai");
  e.contract(-1.0, T1, "ja", Lhoo, "Pji", 1.0, Lhvo, "Pai");
  Tensor* hhoo = T("hhoo", {SO, SO}, 1);
  e.axpy(1.0, c->hoo, "ij", 0.0, hhoo, "ij");
  e.contract(1.0, c->hov, "ia", T1, "ja", 1.0, hhoo, "ij");
  Tensor* hhvv = T("hhvv", {SV, SV}, 1);
  e.axpy(1.0, c->hvv, "ab", 0.0, hhvv, "ab");
  e.contract(-1.0, T1, "ia", c->hov, "ib", 1.0, hhvv, "ab");
  Tensor* hhvo = T("hhvo", {SV, SO}, 1);
  e.axpy(1.0, c->hvo, "ai", 0.0, hhvo, "ai");
  e.contract(1.0, c->hvv, "ab", T1, "ib", 1.0, hhvo, "ai");
  e.contract(-1.0, T1, "ja", hhoo, "ji", 1.0, hhvo, "ai");

  // dressed Fock matrix F = hhat + 2 Lhat J - Lhat_pk Lhat_kq
  Tensor* J = T("J", {SQ}, 1);
  e.contract(1.0, Lhoo, "Pkl", c->Ioo, "kl", 0.0, J, "P");
  Tensor* Foo = T("Foo", {SO, SO}, 1);
  e.axpy(1.0, hhoo, "ij", 0.0, Foo, "ij");
  e.contract(2.0, Lhoo, "Pij", J, "P", 1.0, Foo, "ij");
  e.contract(-1.0, Lhoo, "Pik", Lhoo, "Pkj", 1.0, Foo, "ij");
  Tensor* Fov = T("Fov", {SO, SV}, 1);
  e.axpy(1.0, c->hov, "ia", 0.0, Fov, "ia");
  e.contract(2.0, Lov, "Pia", J, "P", 1.0, Fov, "ia");
  e.contract(-1.0, Lhoo, "Pik", Lov, "Pka", 1.0, Fov, "ia");
  Tensor* Fvo = T("Fvo", {SV, SO}, 1);
  e.axpy(1.0, hhvo, "ai", 0.0, Fvo, "ai");
  e.contract(2.0, Lhvo, "Pai", J, "P", 1.0, Fvo, "ai");
  e.contract(-1.0, Lhvo, "Pak", Lhoo, "Pki", 1.0, Fvo, "ai");
  Tensor* Fvv = T("Fvv", {SV, SV}, 1);
  e.axpy(1.0, hhvv, "ab", 0.0, Fvv, "ab");
  e.contract(2.0, Lhvv, "Pab", J, "P", 1.0, Fvv, "ab");
  e.contract(-1.0, Lhvo, "Pak", Lov, "Pkb", 1.0, Fvv, "ab");

  // Cholesky-built integrals (Eq. 1), Mulliken order; (ia|jb), (mc|bd) and
  // the undressed ladder integrals are amplitude independent (prepare()).
  Tensor* Govov = c->Govov;
  Tensor* Gvovo = T("Gvovo", {SV, SO, SV, SO}, 2);
  e.contract(1.0, Lhvo, "Pai", Lhvo, "Pbj", 0.0, Gvovo, "aibj");
  Tensor* Goooo = T("Goooo", {SO, SO, SO, SO}, 2);
  e.contract(1.0, Lhoo, "Pki", Lhoo, "Plj", 0.0, Goooo, "kilj");
  Tensor* Goovv = T("Goovv", {SO, SO, SV, SV}, 2);
  e.contract(1.0, Lhoo, "Pki", Lhvv, "Pac", 0.0, Goovv, "kiac");
  Tensor* Govvo = T("Govvo", {SO, SV, SV, SO}, 2);
  e.contract(1.0, Lov, "Pme", Lhvo, "Pbj", 0.0, Govvo, "mebj");

  Tensor* u = T("u", {SO, SO, SV, SV}, 2);
  e.axpy(2.0, t2s, "ijab", 0.0, u, "ijab");
  e.axpy(-1.0, t2s, "ijba", 1.0, u, "ijab");

  // ---- singles
  Tensor* R1 = c->R1;
  e.axpy(1.0, Fvo, "ai", 0.0, R1, "ia");
  Tensor* Yt = T("Yt", {SQ, SO, SV}, 1);
  e.contract(1.0, u, "kicd", Lov, "Pkc", 0.0, Yt, "Pid");
  e.contract(1.0, Lhvv, "Pad", Yt, "Pid", 1.0, R1, "ia");
  Tensor* Zt = T("Zt", {SQ, SO, SV}, 1);
  e.contract(1.0, u, "klac", Lov, "Plc", 0.0, Zt, "Pka");
  e.contract(-1.0, Lhoo, "Pki", Zt, "Pka", 1.0, R1, "ia");
  e.contract(1.0, u, "ikac", Fov, "kc", 1.0, R1, "ia");

  // ---- doubles
  Tensor* Rr = T("R2raw", {SO, SO, SV, SV}, 2);
  e.axpy(1.0, Gvovo, "aibj", 0.0, Rr, "ijab");
  // particle-particle ladder with the dressed (ac|bd)^ = sum_P Lhat_ac Lhat_bd,
  // Lhat_vv = L_vv - t1^T L_ov, expanded so that only the undressed W0 (built
  // once per gradient) enters the O(o^2 v^4) product:
  //   (ac|bd)^ = (ac|bd) - t_m^a (mc|bd) - t_n^b (ac|nd) + t_m^a t_n^b (mc|nd)
  if (c->otf)
    e.ladder(1.0, t2s, c->Lvv, Rr);                              // PPL
  else
    e.ladder_stored(1.0, t2s, c->W0, Rr);                        // PPL
  Tensor* Yl = T("Ylad", {SO, SO, SO, SV}, 2);
  e.contract(1.0, t2s, "ijcd", c->Govvv, "mbcd", 0.0, Yl, "ijmb");
  e.contract(-1.0, T1, "ma", Yl, "ijmb", 1.0, Rr, "ijab");
  e.contract(-1.0, T1, "nb", Yl, "jina", 1.0, Rr, "ijab");
  Tensor* Zl = T("Zlad", {SO, SO, SO, SO}, 2);
  e.contract(1.0, t2s, "ijcd", Govov, "mcnd", 0.0, Zl, "ijmn");
  Tensor* Xl = T("Xlad", {SO, SO, SV, SO}, 2);
  e.contract(1.0, T1, "ma", Zl, "ijmn", 0.0, Xl, "ijan");
  e.contract(1.0, T1, "nb", Xl, "ijan", 1.0, Rr, "ijab");
  Tensor* Wh = T("Whh", {SO, SO, SO, SO}, 2);
  e.axpy(1.0, Goooo, "kilj", 0.0, Wh, "kilj");
  e.contract(1.0, t2s, "ijcd", Govov, "kcld", 1.0, Wh, "kilj");
  e.contract(1.0, t2s, "klab", Wh, "kilj", 1.0, Rr, "ijab");     // hole-hole
  // rings: spin-integrated P(ij)P(ab) t_im^ae W_mbej, direct (WA) and
  // exchange (WC) spin patterns.  W_mbej is stored with rows (m,e) and
  // columns (j,b), and the ring sum Rg_ij^ab with rows (j,b) and columns
  // (i,a): the layouts in which the products below write and read them.
  Tensor* WA = T("WA", {SO, SV, SO, SV}, 2);
  e.axpy(1.0, Govvo, "mebj", 0.0, WA, "mejb");
  e.contract(0.5, u, "jnbf", Govov, "menf", 1.0, WA, "mejb");
  e.contract(-0.5, t2s, "jnbf", Govov, "mfne", 1.0, WA, "mejb");
  Tensor* WC = T("WC", {SO, SV, SO, SV}, 2);
  e.axpy(-1.0, Goovv, "mjbe", 0.0, WC, "mejb");
  e.contract(0.5, t2s, "jnfb", Govov, "mfne", 1.0, WC, "mejb");
  Tensor* Rg = T("Ring", {SO, SV, SO, SV}, 2);
  e.contract(1.0, WA, "mejb", u, "imae", 0.0, Rg, "jbia");
  e.contract(1.0, WC, "mejb", t2s, "imae", 1.0, Rg, "jbia");
  e.contract(1.0, WC, "meib", t2s, "mjae", 1.0, Rg, "jbia");
  e.axpy(1.0, Rg, "jbia", 1.0, Rr, "ijab");
  e.axpy(1.0, Rg, "iajb", 1.0, Rr, "ijab");
  // Fock-like terms
  Tensor* Fvv2 = T("Fvv2", {SV, SV}, 1);
  e.axpy(1.0, Fvv, "bc", 0.0, Fvv2, "bc");
  e.contract(-1.0, u, "klbd", Govov, "ldkc", 1.0, Fvv2, "bc");
  Tensor* Foo2 = T("Foo2", {SO, SO}, 1);
  e.axpy(1.0, Foo, "kj", 0.0, Foo2, "kj");
  e.contract(1.0, u, "ljcd", Govov, "kdlc", 1.0, Foo2, "kj");
  Tensor* E1 = T("E1", {SO, SO, SV, SV}, 2);
  e.contract(1.0, t2s, "ijac", Fvv2, "bc", 0.0, E1, "ijab");
  e.contract(-1.0, t2s, "ikab", Foo2, "kj", 1.0, E1, "ijab");
  e.axpy(1.0, E1, "ijab", 1.0, Rr, "ijab");
  e.axpy(1.0, E1, "jiba", 1.0, Rr, "ijab");
  // symmetrise
  e.axpy(0.5, Rr, "ijab", 0.0, c->R2, "ijab");
  e.axpy(0.5, Rr, "jiba", 1.0, c->R2, "ijab");

  // ---- energy <0|Hhat|0> + sum (2(ia|jb) - (ib|ja)) t_ij^ab
  Tensor* E = c->E;
  e.contract(1.0, hhoo, "kl", c->Ioo, "kl", 0.0, E, "");
  e.contract(1.0, Foo, "kl", c->Ioo, "kl", 1.0, E, "");
  e.contract(1.0, c->Xe, "iajb", t2s, "ijab", 1.0, E, "");
}

double scalar(cdcc_ctx* c, const Tensor* t) {
  double v = 0;
  CK(cudaMemcpyAsync(&v, t->d, 8, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return v;
}

// Row and column parts of D = sum (occupied eps) - sum (virtual eps) for a
// layout whose row group holds occupied and column group virtual indices
// (t1: {SO,SV}/1, t2: {SO,SO,SV,SV}/2), with the row-major tuple order of
// the DPD layout (dpd.h); rows are cut into chunks of ~16K elements.
void build_denom(cdcc_ctx* c, const Layout& L, Denom2D& D) {
  const Dims& d = c->dims;
  const int h = d.h, nocc = c->hd.nocc;
  const double* eps = c->eps.data();
  std::vector<Block2D> blocks;
  std::vector<Chunk2D> chunks;
  std::vector<double> rv, cv;
  auto group = [&](int q0, int m, int G, std::vector<double>& out) {
    // tuples of irreps with xor G (g_0 slowest), then local indices
    const int ncode = m >= 2 ? (m == 2 ? h : h * h) : 1;
    for (int code = 0; code < ncode; ++code) {
      int g[MAXRANK];
      int x = G, cc = code;
      for (int q = m - 2; q >= 0; --q) {
        g[q] = cc % h;
        cc /= h;
        x ^= g[q];
      }
      g[m - 1] = x;
      int64_t cnt = 1;
      for (int q = 0; q < m; ++q) cnt *= d.n[L.sp[q0 + q]][g[q]];
      for (int64_t e = 0; e < cnt; ++e) {
        int64_t r = e;
        double v = 0.0;
        for (int q = m - 1; q >= 0; --q) {
          const int sp = L.sp[q0 + q];
          const int n = d.n[sp][g[q]];
          const int l = (int)(r % n);
          r /= n;
          v += sp == SO ? eps[d.gstart[SO][g[q]] + l]
                        : -eps[nocc + d.gstart[SV][g[q]] + l];
        }
        out.push_back(v);
      }
    }
  };
  for (int G = 0; G < h; ++G) {
    Block2D b;
    b.off = L.blk_off[G];
    b.ncol = L.ncol[G];
    b.rv0 = (int64_t)rv.size();
    b.cv0 = (int64_t)cv.size();
    group(0, L.split, G, rv);
    group(L.split, L.rank - L.split, G ^ L.gtot, cv);
    if ((int64_t)rv.size() - b.rv0 != L.nrow[G] ||
        (int64_t)cv.size() - b.cv0 != L.ncol[G])
      throw StatusError(CDCC_EINVAL, "internal: denominator layout");
    const int blk = (int)blocks.size();
    blocks.push_back(b);
    if (L.nrow[G] == 0 || L.ncol[G] == 0) continue;
    const int step = (int)std::max<int64_t>(
        1, std::min<int64_t>(L.nrow[G], 16384 / std::max<int64_t>(1, L.ncol[G])));
    for (int r = 0; r < L.nrow[G]; r += step)
      chunks.push_back(
          {blk, r, (int)std::min<int64_t>(step, L.nrow[G] - r)});
  }
  Engine& e = *c->eng;
  D.nblk = (int)blocks.size();
  D.nchunk = (int)chunks.size();
  D.nrv = (int64_t)rv.size();
  D.ncv = (int64_t)cv.size();
  D.blocks = (Block2D*)e.al.alloc(blocks.size() * sizeof(Block2D));
  D.chunks = (Chunk2D*)e.al.alloc(std::max<size_t>(1, chunks.size()) *
                                  sizeof(Chunk2D));
  D.rv = (double*)e.al.alloc(std::max<int64_t>(1, D.nrv) * 8);
  D.cv = (double*)e.al.alloc(std::max<int64_t>(1, D.ncv) * 8);
  CK(cudaMemcpyAsync(D.blocks, blocks.data(), blocks.size() * sizeof(Block2D),
                     cudaMemcpyHostToDevice, c->st));
  if (!chunks.empty())
    CK(cudaMemcpyAsync(D.chunks, chunks.data(),
                       chunks.size() * sizeof(Chunk2D),
                       cudaMemcpyHostToDevice, c->st));
  if (D.nrv)
    CK(cudaMemcpyAsync(D.rv, rv.data(), D.nrv * 8, cudaMemcpyHostToDevice,
                       c->st));
  if (D.ncv)
    CK(cudaMemcpyAsync(D.cv, cv.data(), D.ncv * 8, cudaMemcpyHostToDevice,
                       c->st));
  CK(cudaStreamSynchronize(c->st));   // host vectors go out of scope
}

void free_denom(cdcc_ctx* c, Denom2D& D) {
  Engine& e = *c->eng;
  if (D.blocks) e.al.release(D.blocks, D.nblk * sizeof(Block2D));
  if (D.chunks)
    e.al.release(D.chunks, std::max(1, D.nchunk) * sizeof(Chunk2D));
  if (D.rv) e.al.release(D.rv, std::max<int64_t>(1, D.nrv) * 8);
  if (D.cv) e.al.release(D.cv, std::max<int64_t>(1, D.ncv) * 8);
  D = Denom2D();
}

// err = R / D over the amplitude vector layout; returns max |R/D|
double probe_step(cdcc_ctx* c, Tensor* R1, Tensor* R2, Tensor* e1) {
  Engine& e = *c->eng;
  CK(cudaMemsetAsync(c->d_max, 0, 8, c->st));
  if (!c->den[0].blocks) build_denom(c, c->T1->lay, c->den[0]);
  if (!c->den[1].blocks) build_denom(c, c->T2->lay, c->den[1]);
  const Denom2D &d1 = c->den[0], &d2 = c->den[1];
  const int64_t n1 = c->T1->lay.size;
  // bytes: read R, write the step
  const double ub = 16.0 * (c->T1->lay.size + c->T2->lay.size);
  e.timed(Engine::K_UPDATE, ub, [&] {
    return jacobi2d(d1.blocks, d1.chunks, d1.nchunk, d1.rv, d1.cv, R1->d,
                    nullptr, e1->d, c->d_max, c->st) +
           jacobi2d(d2.blocks, d2.chunks, d2.nchunk, d2.rv, d2.cv, R2->d,
                    nullptr, e1->d + n1, c->d_max, c->st);
  });
  unsigned long long bits = 0;
  CK(cudaMemcpyAsync(&bits, c->d_max, 8, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  double v;
  std::memcpy(&v, &bits, 8);
  return v;
}

void diis_init(cdcc_ctx* c, Diis& D, const std::string& tag, int64_t n) {
  D.dim = std::max(0, std::min(c->opt.diis_dim, 15));
  D.count = D.next = 0;
  D.n = n;
  D.x.clear();
  D.e.clear();
  D.B.assign((size_t)D.dim * D.dim, 0.0);
  for (int k = 0; k < D.dim; ++k) {
    D.x.push_back(c->eng->flat(tag + "_x" + std::to_string(k), n));
    D.e.push_back(c->eng->flat(tag + "_e" + std::to_string(k), n));
  }
}

// Push (x, err) and overwrite x with the DIIS extrapolation.
void diis_step(cdcc_ctx* c, Diis& D, Tensor* x, Tensor* err) {
  if (D.dim < 2) return;
  Engine& e = *c->eng;
  const int s = D.next;
  CK(cudaMemcpyAsync(D.x[s]->d, x->d, (size_t)D.n * 8,
                     cudaMemcpyDeviceToDevice, c->st));
  CK(cudaMemcpyAsync(D.e[s]->d, err->d, (size_t)D.n * 8,
                     cudaMemcpyDeviceToDevice, c->st));
  D.next = (D.next + 1) % D.dim;
  D.count = std::min(D.count + 1, D.dim);
  const int m = D.count;
  std::vector<const double*> xs(m);
  for (int k = 0; k < m; ++k) xs[k] = D.e[k]->d;
  e.timed(Engine::K_OTHER, 8.0 * (m + 1) * D.n, [&] {
    return multi_dot(xs.data(), m, D.e[s]->d, D.n, c->d_partial, c->d_dots,
                     c->st);
  });
  std::vector<double> dots(m);
  CK(cudaMemcpyAsync(dots.data(), c->d_dots, m * 8, cudaMemcpyDeviceToHost,
                     c->st));
  CK(cudaStreamSynchronize(c->st));
  for (int k = 0; k < m; ++k) {
    D.B[s * D.dim + k] = dots[k];
    D.B[k * D.dim + s] = dots[k];
  }
  if (m < 2) return;
  // solve [B -1; -1 0][c; l] = [0; -1] (scaled), Gaussian elimination
  const int N = m + 1;
  std::vector<double> A((size_t)N * N, 0.0), rhs(N, 0.0);
  double sc = 0;
  for (int i = 0; i < m; ++i) sc = std::max(sc, D.B[i * D.dim + i]);
  if (!(sc > 0)) sc = 1;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) A[i * N + j] = D.B[i * D.dim + j] / sc;
  for (int i = 0; i < m; ++i) {
    A[i * N + m] = -1.0;
    A[m * N + i] = -1.0;
  }
  rhs[m] = -1.0;
  std::vector<int> piv(N);
  for (int k = 0; k < N; ++k) {
    int p = k;
    for (int i = k + 1; i < N; ++i)
      if (std::fabs(A[i * N + k]) > std::fabs(A[p * N + k])) p = i;
    if (A[p * N + k] == 0.0) return;  // singular: skip extrapolation
    if (p != k) {
      for (int j = 0; j < N; ++j) std::swap(A[k * N + j], A[p * N + j]);
      std::swap(rhs[k], rhs[p]);
    }
    for (int i = k + 1; i < N; ++i) {
      const double f = A[i * N + k] / A[k * N + k];
      for (int j = k; j < N; ++j) A[i * N + j] -= f * A[k * N + j];
      rhs[i] -= f * rhs[k];
    }
  }
  std::vector<double> sol(N);
  for (int i = N - 1; i >= 0; --i) {
    double v = rhs[i];
    for (int j = i + 1; j < N; ++j) v -= A[i * N + j] * sol[j];
    sol[i] = v / A[i * N + i];
  }
  std::vector<const double*> px(m);
  for (int k = 0; k < m; ++k) px[k] = D.x[k]->d;
  e.timed(Engine::K_OTHER, 8.0 * (m + 1) * D.n, [&] {
    return lincomb(x->d, px.data(), sol.data(), m, D.n, c->st);
  });
}

struct PhaseTimer {
  cdcc_ctx* c;
  int idx;
  PhaseTimer(cdcc_ctx* c_, int i) : c(c_), idx(i) {
    CK(cudaEventRecord(c->ev0, c->st));
  }
  void stop() {
    CK(cudaEventRecord(c->ev1, c->st));
    CK(cudaEventSynchronize(c->ev1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    c->phase[idx] = ms * 1e-3;
  }
};

// Precision schedule (MIXED): the amplitude-independent integrals and the
// density sweep use 3-slice tensor-core products; the CCSD and Lambda
// iterations use 2-slice products until max|R/D| < switch_tol and FP64
// contractions afterwards, so the converged amplitudes satisfy the FP64
// equations.
int mixed(cdcc_ctx* c) {
  return c->opt.precision == CDCC_PREC_MIXED ||
         c->opt.precision == CDCC_PREC_TC;
}
// arithmetic of the accurate phases: FP64 DFMA, or (CDCC_PREC_TC) the
// exact-slice tensor-core products with 4 slices
int exact_prec(cdcc_ctx* c) {
  return c->opt.precision == CDCC_PREC_TC ? 14 : 0;
}
int early_prec(cdcc_ctx* c) { return mixed(c) ? 2 : exact_prec(c); }

// Leave the reduced-precision iterations once max|R/D| is below switch_tol,
// or once it has stopped improving (3 iterations without a 30% gain), which
// happens when the residual reaches the floor of the reduced precision.
struct SwitchRule {
  double tol, best = 1e300;
  int since = 0;
  explicit SwitchRule(double t) : tol(t) {}
  bool done(double r) {
    if (r < tol) return true;
    if (r < 0.7 * best) {
      best = r;
      since = 0;
    } else if (++since >= 3) {
      return true;
    }
    return false;
  }
};

void check_device_error(cdcc_ctx* c) {
  // launches outside Engine::timed report here at the latest
  CK(cudaGetLastError());
  unsigned int err = 0;
  CK(cudaMemcpyAsync(&err, c->d_err, 4, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (err)
    throw StatusError(CDCC_ETIMEOUT,
                      "a bounded device wait gave up (code " +
                          std::to_string(err) + ")");
}

// Linearised ladder in the accurate phase (MIXED and TC schedules, see
// Engine::ladder_lin): the anchor is evaluated accurately when the phase
// starts, later iterations correct it in BF16x3, and convergence is only
// accepted on an iteration whose ladder was a fresh accurate anchor, so the
// converged amplitudes solve the accurate equations.
bool linearised(cdcc_ctx* c) {
  return mixed(c) && c->opt.ladder_linearize != 0;
}

void run_ccsd(cdcc_ctx* c, double* e_corr, int* iters, double* resid) {
  Engine& e = *c->eng;
  PhaseTimer pt(c, 0);
  e.thaw();   // the forward tensors are written again
  {
    const double gb = c->opt.ladder_slices_gb;
    e.ladder_keep_slices(gb > 0 && std::isfinite(gb)
                             ? (int64_t)(std::min(gb, 1e6) * 1e9)
                             : 0);
  }
  c->fwd_fresh = false;
  c->res_acc = false;
  e.ladder_lin(0, 0);
  e.zero(c->amp);
  // the amplitude-independent integrals enter every later FP64 iteration, so
  // they are built with FP64-accurate products
  e.set_precision(exact_prec(c));
  prepare(c);
  e.set_precision(early_prec(c));
  bool early = mixed(c);
  SwitchRule sw(c->opt.switch_tol);
  c->tape_ready = false;
  c->iters_mixed[0] = c->iters_fp64[0] = 0;
  diis_init(c, c->cc_diis, "ccdiis", c->amp->lay.size);
  double e_old = 0, rmax = 0, E = 0;
  bool have_old = false;
  int it = 1;
  for (; it <= c->opt.max_iter; ++it) {
    residual(c);
    (early ? c->iters_mixed[0] : c->iters_fp64[0])++;
    E = scalar(c, c->E);
    rmax = probe_step(c, c->R1, c->R2, c->err1);
    if (!std::isfinite(rmax) || !std::isfinite(E))
      throw StatusError(CDCC_ENUMERIC, "non-finite CCSD residual");
    if (!early && rmax <= c->opt.conv_tol && have_old &&
        std::fabs(E - e_old) <= c->opt.energy_tol) {
      if (!linearised(c) || e.ladder_lin_anchored(0)) break;
      // converged around an older anchor: re-evaluate at the same
      // amplitudes with a fresh accurate anchor before accepting
      e.ladder_lin(0, 1);
      continue;
    }
    if (early && sw.done(rmax)) {
      early = false;        // re-evaluate at the same amplitudes, accurately
      e.set_precision(exact_prec(c));
      if (linearised(c)) e.ladder_lin(0, 1);
      have_old = false;
      continue;
    }
    e_old = E;
    have_old = true;
    e.timed(Engine::K_OTHER, 24.0 * c->amp->lay.size, [&] {
      return axpby(1.0, c->err1->d, 1.0, c->amp->d, c->amp->lay.size, c->st);
    });
    if (it >= 2) diis_step(c, c->cc_diis, c->amp, c->err1);
  }
  e.ladder_lin(0, 0);
  pt.stop();
  check_device_error(c);
  if (it > c->opt.max_iter)
    throw StatusError(CDCC_ENOCONV, "CCSD did not converge");
  // the last evaluation was accurate (and its ladder a fresh anchor) at the
  // converged amplitudes: the tape can be recorded without re-running it
  c->fwd_fresh = true;
  c->res_acc = true;
  c->e_corr = E - c->e_ref;
  if (e_corr) *e_corr = c->e_corr;
  if (iters) *iters = it;
  if (resid) *resid = rmax;
  c->state = 2;
}

void ensure_tape(cdcc_ctx* c) {
  if (c->tape_ready) return;
  Engine& e = *c->eng;
  e.clear_tape();
  e.record(true);
  e.record_only(true);   // the t-independent integrals are already built
  prepare(c);
  if (c->fwd_fresh) {
    // the intermediates of the last (accurate) CCSD evaluation are those
    // at the current amplitudes: record the residual without executing it
    residual(c);
    e.record_only(false);
  } else {
    e.record_only(false);
    const int prec = e.precision();
    e.set_precision(exact_prec(c));
    residual(c);
    e.set_precision(prec);
  }
  e.record(false);
  c->tape_ready = true;
}

void run_lambda(cdcc_ctx* c, int* iters, double* resid) {
  Engine& e = *c->eng;
  PhaseTimer pt(c, 1);
  ensure_tape(c);
  // every Lambda iteration (and the density sweep after it) reads the same
  // forward tensors: their permuted copies and slices are kept meanwhile
  e.freeze_tape_operands();
  e.zero(c->lam);
  e.set_precision(early_prec(c));
  bool early = mixed(c);
  SwitchRule sw(c->opt.switch_tol);
  c->iters_mixed[1] = c->iters_fp64[1] = 0;
  // the CCSD history is no longer needed: Lambda reuses its buffers
  diis_init(c, c->lam_diis, "ccdiis", c->lam->lay.size);
  Tensor* g1 = e.adjoint(c->T1);
  Tensor* g2 = e.adjoint(c->T2);
  e.ladder_lin(1, 0);
  double rmax = 0;
  int it = 1;
  for (; it <= c->opt.max_iter; ++it) {
    e.backward({{c->E, nullptr}, {c->R1, c->L1}, {c->R2, c->L2}}, TAG_AMP);
    (early ? c->iters_mixed[1] : c->iters_fp64[1])++;
    rmax = probe_step(c, g1, g2, c->err1);
    if (!std::isfinite(rmax))
      throw StatusError(CDCC_ENUMERIC, "non-finite Lambda residual");
    if (!early && rmax <= c->opt.conv_tol) {
      if (!linearised(c) || e.ladder_lin_anchored(1)) break;
      e.ladder_lin(1, 1);   // accept only on a fresh accurate anchor
      continue;
    }
    if (early && sw.done(rmax)) {
      early = false;
      e.set_precision(exact_prec(c));
      if (linearised(c)) e.ladder_lin(1, 1);
      continue;
    }
    e.timed(Engine::K_OTHER, 24.0 * c->lam->lay.size, [&] {
      return axpby(1.0, c->err1->d, 1.0, c->lam->d, c->lam->lay.size, c->st);
    });
    if (it >= 2) diis_step(c, c->lam_diis, c->lam, c->err1);
  }
  e.ladder_lin(1, 0);
  pt.stop();
  check_device_error(c);
  if (it > c->opt.max_iter)
    throw StatusError(CDCC_ENOCONV, "Lambda did not converge");
  if (iters) *iters = it;
  if (resid) *resid = rmax;
  c->state = 3;
}

void assemble_density(cdcc_ctx* c);
void frozen_fock_correction(cdcc_ctx* c);
void relax_density(cdcc_ctx* c);

void run_density(cdcc_ctx* c, double* D1) {
  Engine& e = *c->eng;
  PhaseTimer pt(c, 2);
  e.ladder_keep_slices(0);   // the sweep below builds its own batches
  ensure_tape(c);
  e.freeze_tape_operands();
  e.set_precision(c->opt.precision == CDCC_PREC_TC ? 14 : (mixed(c) ? 3 : 0));
  e.backward({{c->E, nullptr}, {c->R1, c->L1}, {c->R2, c->L2}},
             TAG_L | TAG_H);
  e.thaw();
  e.set_precision(0);
  assemble_density(c);
  if (c->opt.fock_model == CDCC_FROZEN_FOCK) frozen_fock_correction(c);
  if (c->opt.relaxed) relax_density(c);
  pt.stop();
  if (D1) {
    const int n = c->hd.n;
    std::vector<double> h = to_host(c, c->D1s);
    std::vector<double> dense((size_t)n * n, 0.0);
    visit_dense(c->D1s->lay, c->dims,
                [&](int64_t off, int64_t di) { dense[di] = h[off]; });
    std::memcpy(D1, dense.data(), dense.size() * 8);
  }
  c->state = 4;
}

// FROZEN_FOCK model: the Fock matrix stays diag(eps) under a displacement
// (h follows L as h = diag(eps) - G(L)) and E = E_corr, so
//     Gamma_FF = Gamma - d<M, G(L)>/dL,   M = D - 1_occ,
// with D the symmetrised one-particle density of the density sweep and
// G(L) = 2 L^P J_P - sum_k L^P_pk L^P_kq the two-electron Fock part (the
// 1_occ removes the reference energy sum_i (2 eps_i - G_ii)).  d<M,G>/dL
// comes from the engine's reverse sweep over a short recorded evaluation of
// <M, G(L)>; the recorded Lambda/density tape is replaced and rebuilt when
// next needed.
void frozen_fock_correction(cdcc_ctx* c) {
  Engine& e = *c->eng;
  Tensor *Loo = c->Loo, *Lov = c->Lov, *Lvo = c->Lvo, *Lvv = c->Lvv;
  Tensor* Moo = e.tensor("ff_Moo", {SO, SO}, 1);
  Tensor* Mov = e.tensor("ff_Mov", {SO, SV}, 1);
  Tensor* Mvo = e.tensor("ff_Mvo", {SV, SO}, 1);
  Tensor* Mvv = e.tensor("ff_Mvv", {SV, SV}, 1);
  e.axpy(1.0, c->D1s, "pq", 0.0, Moo, "pq");
  e.axpy(-1.0, c->Ioo, "ij", 1.0, Moo, "ij");
  e.axpy(1.0, c->D1s, "pq", 0.0, Mov, "pq");
  e.axpy(1.0, c->D1s, "pq", 0.0, Mvo, "pq");
  e.axpy(1.0, c->D1s, "pq", 0.0, Mvv, "pq");
  e.clear_tape();
  c->tape_ready = false;
  e.record(true);
  Tensor* J = e.tensor("ff_J", {SQ}, 1);
  e.contract(1.0, Loo, "Pkl", c->Ioo, "kl", 0.0, J, "P");
  Tensor* Goo = e.tensor("ff_Goo", {SO, SO}, 1);
  e.contract(2.0, Loo, "Pij", J, "P", 0.0, Goo, "ij");
  e.contract(-1.0, Loo, "Pik", Loo, "Pkj", 1.0, Goo, "ij");
  Tensor* Gov = e.tensor("ff_Gov", {SO, SV}, 1);
  e.contract(2.0, Lov, "Pia", J, "P", 0.0, Gov, "ia");
  e.contract(-1.0, Loo, "Pik", Lov, "Pka", 1.0, Gov, "ia");
  Tensor* Gvo = e.tensor("ff_Gvo", {SV, SO}, 1);
  e.contract(2.0, Lvo, "Pai", J, "P", 0.0, Gvo, "ai");
  e.contract(-1.0, Lvo, "Pak", Loo, "Pki", 1.0, Gvo, "ai");
  Tensor* Gvv = e.tensor("ff_Gvv", {SV, SV}, 1);
  e.contract(2.0, Lvv, "Pab", J, "P", 0.0, Gvv, "ab");
  e.contract(-1.0, Lvo, "Pak", Lov, "Pkb", 1.0, Gvv, "ab");
  Tensor* EG = e.tensor("ff_EG", {}, 0);
  e.contract(1.0, Moo, "ij", Goo, "ij", 0.0, EG, "");
  e.contract(1.0, Mov, "ia", Gov, "ia", 1.0, EG, "");
  e.contract(1.0, Mvo, "ai", Gvo, "ai", 1.0, EG, "");
  e.contract(1.0, Mvv, "ab", Gvv, "ab", 1.0, EG, "");
  e.record(false);
  e.backward({{EG, nullptr}}, TAG_L);
  e.clear_tape();
  // Gsym -= sym(d<M,G>/dL), assembled like Gamma^P
  Tensor* Dg = e.tensor("ff_dG", {SQ, SA, SA}, 1);
  e.zero(Dg);
  e.axpy(1.0, e.adjoint(Loo), "Pij", 1.0, Dg, "Pij");
  e.axpy(1.0, e.adjoint(Lov), "Pia", 1.0, Dg, "Pia");
  e.axpy(1.0, e.adjoint(Lvo), "Pai", 1.0, Dg, "Pai");
  e.axpy(1.0, e.adjoint(Lvv), "Pab", 1.0, Dg, "Pab");
  e.axpy(-0.5, Dg, "Ppq", 1.0, c->Gsym, "Ppq");
  e.axpy(-0.5, Dg, "Pqp", 1.0, c->Gsym, "Ppq");
}

// Orbital relaxation (Sec. 2.5, Eq. z_vector) of the relaxed model: the
// orbitals follow the closed-shell SCF condition f_ai = 0 at every
// displacement, so the gradient gains sum_ai Z_ai df_ai/dx with Z the
// solution of the Z-vector equations
//     sum_em A_ai,em Z_em = -2 W_ai,   W = [h, D] + sum_P [L^P, Gamma^P],
//     A_ai,em = f_ae d_im - f_mi d_ae + 4 (ai|em) - (ae|im) - (am|ie)
// (A is the bracket of Eq. z_vector written with the Fock blocks; it is
// symmetric, so conjugate gradients solve the system with one Hessian
// product per iteration through the Cholesky vectors).  Then
//     Gamma^P += sym d/dL^P sum_ai Z_ai f_ai(L)
// (one reverse sweep of a recorded evaluation, as in the frozen-Fock
// correction).  D is left as the unrelaxed dLag/dh.
void relax_density(cdcc_ctx* c) {
  Engine& e = *c->eng;
  Tensor *Loo = c->Loo, *Lov = c->Lov, *Lvo = c->Lvo, *Lvv = c->Lvv;
  // blocks of the symmetric D and Gamma^P
  Tensor* Doo = e.tensor("rx_Doo", {SO, SO}, 1);
  Tensor* Dvo = e.tensor("rx_Dvo", {SV, SO}, 1);
  Tensor* Dvv = e.tensor("rx_Dvv", {SV, SV}, 1);
  e.axpy(1.0, c->D1s, "pq", 0.0, Doo, "pq");
  e.axpy(1.0, c->D1s, "pq", 0.0, Dvo, "pq");
  e.axpy(1.0, c->D1s, "pq", 0.0, Dvv, "pq");
  Tensor* Goo = e.tensor("rx_Goo", {SQ, SO, SO}, 1);
  Tensor* Gvo = e.tensor("rx_Gvo", {SQ, SV, SO}, 1);
  Tensor* Gvv = e.tensor("rx_Gvv", {SQ, SV, SV}, 1);
  e.axpy(1.0, c->Gsym, "Ppq", 0.0, Goo, "Ppq");
  e.axpy(1.0, c->Gsym, "Ppq", 0.0, Gvo, "Ppq");
  e.axpy(1.0, c->Gsym, "Ppq", 0.0, Gvv, "Ppq");
  // W_ai = [h, D]_ai + sum_P [L^P, Gamma^P]_ai
  Tensor* W = e.tensor("rx_W", {SV, SO}, 1);
  e.contract(1.0, c->hvv, "ab", Dvo, "bi", 0.0, W, "ai");
  e.contract(1.0, c->hvo, "aj", Doo, "ji", 1.0, W, "ai");
  e.contract(-1.0, Dvv, "ab", c->hvo, "bi", 1.0, W, "ai");
  e.contract(-1.0, Dvo, "aj", c->hoo, "ji", 1.0, W, "ai");
  e.contract(1.0, Lvv, "Pab", Gvo, "Pbi", 1.0, W, "ai");
  e.contract(1.0, Lvo, "Paj", Goo, "Pji", 1.0, W, "ai");
  e.contract(-1.0, Gvv, "Pab", Lvo, "Pbi", 1.0, W, "ai");
  e.contract(-1.0, Gvo, "Paj", Loo, "Pji", 1.0, W, "ai");
  // Fock blocks f = h + G(L) (diag(eps) at the reference of the model)
  Tensor* J = e.tensor("rx_J", {SQ}, 1);
  e.contract(1.0, Loo, "Pkl", c->Ioo, "kl", 0.0, J, "P");
  Tensor* Foo = e.tensor("rx_Foo", {SO, SO}, 1);
  e.axpy(1.0, c->hoo, "ij", 0.0, Foo, "ij");
  e.contract(2.0, Loo, "Pij", J, "P", 1.0, Foo, "ij");
  e.contract(-1.0, Loo, "Pik", Loo, "Pkj", 1.0, Foo, "ij");
  Tensor* Fvv = e.tensor("rx_Fvv", {SV, SV}, 1);
  e.axpy(1.0, c->hvv, "ab", 0.0, Fvv, "ab");
  e.contract(2.0, Lvv, "Pab", J, "P", 1.0, Fvv, "ab");
  e.contract(-1.0, Lvo, "Pak", Lov, "Pkb", 1.0, Fvv, "ab");
  // A p through the Cholesky vectors
  Tensor* X = e.tensor("rx_X", {SQ}, 1);
  Tensor* Y = e.tensor("rx_Y", {SQ, SO, SV}, 1);
  Tensor* Q = e.tensor("rx_Q", {SQ, SO, SO}, 1);
  auto hess = [&](Tensor* p, Tensor* Ap) {
    e.contract(1.0, Fvv, "ae", p, "ei", 0.0, Ap, "ai");
    e.contract(-1.0, p, "am", Foo, "mi", 1.0, Ap, "ai");
    e.contract(1.0, Lvo, "Pem", p, "em", 0.0, X, "P");
    e.contract(4.0, Lvo, "Pai", X, "P", 1.0, Ap, "ai");
    e.contract(1.0, Loo, "Pim", p, "em", 0.0, Y, "Pie");
    e.contract(-1.0, Lvv, "Pae", Y, "Pie", 1.0, Ap, "ai");
    e.contract(1.0, Lov, "Pie", p, "em", 0.0, Q, "Pim");
    e.contract(-1.0, Lvo, "Pam", Q, "Pim", 1.0, Ap, "ai");
  };
  Tensor* S = e.tensor("rx_S", {}, 0);
  auto dot = [&](Tensor* a, Tensor* b) {
    e.contract(1.0, a, "ai", b, "ai", 0.0, S, "");
    return scalar(c, S);
  };
  Tensor* Z = e.tensor("rx_Z", {SV, SO}, 1);
  Tensor* r = e.tensor("rx_r", {SV, SO}, 1);
  Tensor* p = e.tensor("rx_p", {SV, SO}, 1);
  Tensor* Ap = e.tensor("rx_Ap", {SV, SO}, 1);
  e.zero(Z);
  e.axpy(-2.0, W, "ai", 0.0, r, "ai");      // r = b - A*0, b = -2W
  e.axpy(1.0, r, "ai", 0.0, p, "ai");
  double rr = dot(r, r);
  const double bb = rr;
  const double tol2 = 1e-26 * std::max(bb, 1e-300);
  int it = 0;
  while (rr > tol2) {
    if (++it > 500)
      throw StatusError(CDCC_ENOCONV, "Z-vector equations did not converge");
    hess(p, Ap);
    const double pAp = dot(p, Ap);
    if (!(pAp > 0) || !std::isfinite(pAp))
      throw StatusError(CDCC_ENUMERIC,
                        "Z-vector: the orbital Hessian is not positive");
    const double alpha = rr / pAp;
    e.axpy(alpha, p, "ai", 1.0, Z, "ai");
    e.axpy(-alpha, Ap, "ai", 1.0, r, "ai");
    const double rn = dot(r, r);
    e.axpy(1.0, r, "ai", rn / rr, p, "ai");
    rr = rn;
  }
  // Gamma^P += sym d/dL^P <Z, f_vo(L)>, f_vo = h_vo + 2 L_vo J - L_vk L_ko
  e.clear_tape();
  c->tape_ready = false;
  e.record(true);
  Tensor* Jr = e.tensor("rx_Jr", {SQ}, 1);
  e.contract(1.0, Loo, "Pkl", c->Ioo, "kl", 0.0, Jr, "P");
  Tensor* Gf = e.tensor("rx_Gf", {SV, SO}, 1);
  e.contract(2.0, Lvo, "Pai", Jr, "P", 0.0, Gf, "ai");
  e.contract(-1.0, Lvo, "Pak", Loo, "Pki", 1.0, Gf, "ai");
  Tensor* EZ = e.tensor("rx_EZ", {}, 0);
  e.contract(1.0, Z, "ai", Gf, "ai", 0.0, EZ, "");
  e.record(false);
  e.backward({{EZ, nullptr}}, TAG_L);
  e.clear_tape();
  Tensor* Dg = e.tensor("rx_dG", {SQ, SA, SA}, 1);
  e.zero(Dg);
  e.axpy(1.0, e.adjoint(Loo), "Pij", 1.0, Dg, "Pij");
  e.axpy(1.0, e.adjoint(Lov), "Pia", 1.0, Dg, "Pia");
  e.axpy(1.0, e.adjoint(Lvo), "Pai", 1.0, Dg, "Pai");
  e.axpy(1.0, e.adjoint(Lvv), "Pab", 1.0, Dg, "Pab");
  e.axpy(0.5, Dg, "Ppq", 1.0, c->Gsym, "Ppq");
  e.axpy(0.5, Dg, "Pqp", 1.0, c->Gsym, "Ppq");
  c->z_iters = it;
}

// Gamma^P and D from the adjoints left by the density sweep.
void assemble_density(cdcc_ctx* c) {
  Engine& e = *c->eng;
  // Gamma^P_pq: embed the block adjoints into the packed pattern, symmetrise
  e.zero(c->Gam);
  e.axpy(1.0, e.adjoint(c->Loo), "Pij", 1.0, c->Gam, "Pij");
  e.axpy(1.0, e.adjoint(c->Lov), "Pia", 1.0, c->Gam, "Pia");
  e.axpy(1.0, e.adjoint(c->Lvo), "Pai", 1.0, c->Gam, "Pai");
  e.axpy(1.0, e.adjoint(c->Lvv), "Pab", 1.0, c->Gam, "Pab");
  e.axpy(0.5, c->Gam, "Ppq", 0.0, c->Gsym, "Ppq");
  e.axpy(0.5, c->Gam, "Pqp", 1.0, c->Gsym, "Ppq");
  // one-particle density
  e.zero(c->D1a);
  e.axpy(1.0, e.adjoint(c->hoo), "ij", 1.0, c->D1a, "ij");
  e.axpy(1.0, e.adjoint(c->hov), "ia", 1.0, c->D1a, "ia");
  e.axpy(1.0, e.adjoint(c->hvo), "ai", 1.0, c->D1a, "ai");
  e.axpy(1.0, e.adjoint(c->hvv), "ab", 1.0, c->D1a, "ab");
  e.axpy(0.5, c->D1a, "pq", 0.0, c->D1s, "pq");
  e.axpy(0.5, c->D1a, "qp", 1.0, c->D1s, "pq");
}

size_t packed_size_g(const cdcc_ctx* c, int gx) {
  size_t s = 0;
  for (int gP = 0; gP < c->hd.h; ++gP) {
    size_t pairs = 0;
    for (int gp = 0; gp < c->hd.h; ++gp)
      pairs += (size_t)c->dims.n[SA][gp] * c->dims.n[SA][gp ^ gP ^ gx];
    s += (size_t)c->dims.n[SQ][gP] * pairs;
  }
  return s;
}

void run_contract(cdcc_ctx* c, int nx, const int32_t* x_irrep,
                  const double* dL, double* g) {
  Engine& e = *c->eng;
  PhaseTimer pt(c, 3);
  const int64_t nnz = c->Gsym->lay.size;
  const bool dev = is_device_ptr(dL);
  std::vector<double> out(nx, 0.0);
  // group consecutive totally symmetric displacements
  const int XB = 8;
  double* stage = nullptr;
  if (!dev) stage = e.scratch((int64_t)XB * nnz);
  double* d_g = e.scratch(std::max(nx, 1));
  const int64_t need = batched_dot_partial_doubles(nnz, XB);
  double* part = e.scratch(need);
  std::vector<double> gtmp(XB);
  int64_t off = 0;
  int x = 0;
  while (x < nx) {
    const int gx = x_irrep ? x_irrep[x] : 0;
    if (gx < 0 || gx >= c->hd.h)
      throw StatusError(CDCC_EINVAL, "displacement irrep out of range");
    if (gx != 0) {
      off += (int64_t)packed_size_g(c, gx);
      out[x++] = 0.0;
      continue;
    }
    int cnt = 0;
    while (x + cnt < nx && cnt < XB && (x_irrep ? x_irrep[x + cnt] : 0) == 0)
      ++cnt;
    const double* src = dL + off;
    if (!dev) {
      CK(cudaMemcpyAsync(stage, src, (size_t)cnt * nnz * 8,
                         cudaMemcpyHostToDevice, c->st));
      src = stage;
    }
    // algorithmic bytes: each dL_x once plus Gamma once
    e.timed(Engine::K_DOT, 8.0 * (cnt + 1) * nnz, [&] {
      return batched_dot(c->Gsym->d, src, cnt, nnz, part, d_g, c->st);
    });
    CK(cudaMemcpyAsync(gtmp.data(), d_g, cnt * 8, cudaMemcpyDeviceToHost,
                       c->st));
    CK(cudaStreamSynchronize(c->st));
    for (int k = 0; k < cnt; ++k) out[x + k] = gtmp[k];
    off += (int64_t)cnt * nnz;
    x += cnt;
  }
  e.release_scratch();
  pt.stop();
  std::memcpy(g, out.data(), nx * 8);
}

// sum_e A[e] X_x[e] for nx vectors X_x of n doubles back to back (host or
// device memory), 8 at a time through the batched dot kernel.
void dots_with(cdcc_ctx* c, const double* A, const double* X, int nx,
               int64_t n, double* out) {
  Engine& e = *c->eng;
  if (nx <= 0) return;
  if (n == 0) {
    for (int x = 0; x < nx; ++x) out[x] = 0.0;
    return;
  }
  const bool dev = is_device_ptr(X);
  const int XB = 8;
  double* stage = dev ? nullptr : e.scratch((int64_t)XB * n);
  double* d_g = e.scratch(XB);
  double* part = e.scratch(batched_dot_partial_doubles(n, XB));
  std::vector<double> tmp(XB);
  for (int x = 0; x < nx; x += XB) {
    const int cnt = std::min(XB, nx - x);
    const double* src = X + (int64_t)x * n;
    if (!dev) {
      CK(cudaMemcpyAsync(stage, src, (size_t)cnt * n * 8,
                         cudaMemcpyHostToDevice, c->st));
      src = stage;
    }
    e.timed(Engine::K_DOT, 8.0 * (cnt + 1) * n, [&] {
      return batched_dot(A, src, cnt, n, part, d_g, c->st);
    });
    CK(cudaMemcpyAsync(tmp.data(), d_g, cnt * 8, cudaMemcpyDeviceToHost,
                       c->st));
    CK(cudaStreamSynchronize(c->st));
    for (int k = 0; k < cnt; ++k) out[x + k] = tmp[k];
  }
  e.release_scratch();
}

// Three-term gradient of the density-fitting / Cholesky form (Sec. 2.1
// Eqs. dfcd, cv_2ndstep, eri_cddf_der; Sec. 2.6 Eq. 2el_grad_cont): with
// L = K^{-1} B and M = K K^T,
//   g_x = sum_P <Jt^P, dB_x^P> - sum_PQ W_PQ dM_x,PQ,
//   Jt = K^{-T} Gamma,  Ltilde = K^{-T} L,  W = 1/2 Ltilde Jt^T,
// in the accurate arithmetic of the schedule.
void run_contract_df(cdcc_ctx* c, const double* metric, int nx,
                     const double* dB, const double* dM, double* g) {
  Engine& e = *c->eng;
  PhaseTimer pt(c, 3);
  Tensor* Mt = e.tensor("df_M", {SQ, SQ}, 1);
  Tensor* Kt = e.tensor("df_KinvT", {SQ, SQ}, 1);
  MetricBlocks mb;
  std::memset(&mb, 0, sizeof(mb));
  int64_t off = 0;
  for (int G = 0; G < c->hd.h; ++G) {
    if (Mt->lay.blk_off[G] != off)
      throw StatusError(CDCC_EINVAL, "internal: metric layout");
    mb.off[G] = off;
    mb.n[G] = c->dims.n[SQ][G];
    off += (int64_t)mb.n[G] * mb.n[G];
  }
  mb.nblk = c->hd.h;
  if (off != Mt->lay.size)
    throw StatusError(CDCC_EINVAL, "internal: metric size");
  copy_in(c, Mt->d, metric, off);
  CK(cudaMemsetAsync(c->d_err + 1, 0, 4, c->st));
  e.timed(Engine::K_OTHER, 16.0 * off, [&] {
    return metric_factor(Mt->d, Kt->d, mb, c->d_err + 1, c->st);
  });
  unsigned int bad = 0;
  CK(cudaMemcpyAsync(&bad, c->d_err + 1, 4, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (bad)
    throw StatusError(CDCC_EINVAL, "metric is not positive definite");
  ++Mt->ver;
  ++Kt->ver;
  const int prec = e.precision();
  e.set_precision(exact_prec(c));
  Tensor* Jt = e.tensor("df_Jt", {SQ, SA, SA}, 1);
  Tensor* Lt = e.tensor("df_Lt", {SQ, SA, SA}, 1);
  Tensor* W = e.tensor("df_W", {SQ, SQ}, 1);
  e.contract(1.0, Kt, "PQ", c->Gsym, "Qpq", 0.0, Jt, "Ppq");
  e.contract(1.0, Kt, "PQ", c->Lpk, "Qpq", 0.0, Lt, "Ppq");
  e.contract(0.5, Lt, "Ppq", Jt, "Qpq", 0.0, W, "PQ");
  e.set_precision(prec);
  std::vector<double> gb(std::max(nx, 1)), gm(std::max(nx, 1));
  dots_with(c, Jt->d, dB, nx, Jt->lay.size, gb.data());
  dots_with(c, W->d, dM, nx, W->lay.size, gm.data());
  pt.stop();
  check_device_error(c);
  for (int x = 0; x < nx; ++x) g[x] = gb[x] - gm[x];
}

// What the reduced-precision arithmetic of the schedule changed, measured
// against FP64 DFMA arithmetic at the same converged (t, lambda):
//   dE   = |E64(t) - E(t)| + |<lambda, R64(t)>|: the FP64 equations leave a
//          residual R64 at the schedule's amplitudes, and to first order the
//          FP64 energy at its own solution differs by -<lambda, R64>;
//   dg_x = |<Gamma64 - Gamma, dL_x>| from an FP64 density sweep.
// Gamma^P and D of the context are restored afterwards.
void run_error_estimate(cdcc_ctx* c, int nx, const int32_t* x_irrep,
                        const double* dL, double* dE, double* dg) {
  Engine& e = *c->eng;
  std::vector<double> g0(std::max(nx, 1)), g64(std::max(nx, 1));
  if (nx > 0) run_contract(c, nx, x_irrep, dL, g0.data());
  const int64_t ng = c->Gsym->lay.size, nd = c->D1s->lay.size;
  Tensor* keepG = e.flat("errest_G", ng);
  Tensor* keepD = e.flat("errest_D", nd);
  CK(cudaMemcpyAsync(keepG->d, c->Gsym->d, (size_t)ng * 8,
                     cudaMemcpyDeviceToDevice, c->st));
  CK(cudaMemcpyAsync(keepD->d, c->D1s->d, (size_t)nd * 8,
                     cudaMemcpyDeviceToDevice, c->st));
  e.thaw();
  ensure_tape(c);
  const int prec = e.precision();
  e.set_precision(0);
  residual(c);                       // FP64 E, R and tape intermediates at t
  c->res_acc = false;
  const double E64 = scalar(c, c->E) - c->e_ref;
  const double* lam = c->lam->d;
  e.timed(Engine::K_OTHER, 16.0 * c->lam->lay.size, [&] {
    return multi_dot(&lam, 1, c->res->d, c->lam->lay.size, c->d_partial,
                     c->d_dots, c->st);
  });
  double lr = 0;
  CK(cudaMemcpyAsync(&lr, c->d_dots, 8, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  *dE = std::fabs(E64 - c->e_corr) + std::fabs(lr);
  e.backward({{c->E, nullptr}, {c->R1, c->L1}, {c->R2, c->L2}},
             TAG_L | TAG_H);
  assemble_density(c);
  if (c->opt.fock_model == CDCC_FROZEN_FOCK) frozen_fock_correction(c);
  if (c->opt.relaxed) relax_density(c);
  if (nx > 0) run_contract(c, nx, x_irrep, dL, g64.data());
  for (int x = 0; x < nx; ++x) dg[x] = std::fabs(g64[x] - g0[x]);
  CK(cudaMemcpyAsync(c->Gsym->d, keepG->d, (size_t)ng * 8,
                     cudaMemcpyDeviceToDevice, c->st));
  CK(cudaMemcpyAsync(c->D1s->d, keepD->d, (size_t)nd * 8,
                     cudaMemcpyDeviceToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  e.set_precision(prec);
  check_device_error(c);
}

double lam_dot_res(cdcc_ctx* c) {
  Engine& e = *c->eng;
  const double* lam = c->lam->d;
  e.timed(Engine::K_OTHER, 16.0 * c->lam->lay.size, [&] {
    return multi_dot(&lam, 1, c->res->d, c->lam->lay.size, c->d_partial,
                     c->d_dots, c->st);
  });
  double v = 0;
  CK(cudaMemcpyAsync(&v, c->d_dots, 8, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return v;
}

// Error report of E_corr (cdcc_energy_error): the convergence term
// <lambda, R(t)> and, for the exact-slice schedule, the change of the energy
// functional E + <lambda, R> between 3 and 4 exact slices, divided by 2^7
// (each slice keeps 7 more bits of every operand).
void run_energy_error(cdcc_ctx* c, double* dE) {
  Engine& e = *c->eng;
  e.thaw();
  if (!c->res_acc) {
    // the accurate residual at t is needed again
    const int prec = e.precision();
    e.set_precision(exact_prec(c));
    residual(c);
    e.set_precision(prec);
    c->res_acc = true;
  }
  const double conv = lam_dot_res(c);
  double out = std::fabs(conv);
  if (c->opt.precision == CDCC_PREC_TC) {
    const double E4 = c->e_corr + c->e_ref;
    const int prec = e.precision();
    e.set_precision(13);
    residual(c);
    e.set_precision(prec);
    const double E3 = scalar(c, c->E);
    const double conv3 = lam_dot_res(c);
    out += (std::fabs(E3 - E4) + std::fabs(conv3 - conv)) / 128.0;
    // c->res and the recorded intermediates now hold the 3-slice values
    c->res_acc = false;
    c->fwd_fresh = false;
    c->tape_ready = false;
  }
  check_device_error(c);
  *dE = out;
}

void init_ctx(cdcc_ctx* c, int nirrep, int nocc, int nvir, int nchol,
              const int32_t* orb_irrep, const double* eps,
              const int32_t* chol_irrep, const double* L) {
  if (!(nirrep == 1 || nirrep == 2 || nirrep == 4 || nirrep == 8))
    throw StatusError(CDCC_EINVAL, "nirrep must be 1, 2, 4 or 8");
  if (nocc < 1 || nvir < 1 || nchol < 1)
    throw StatusError(CDCC_EINVAL, "nocc, nvir, nchol must be >= 1");
  if (!orb_irrep || !eps || !chol_irrep || !L)
    throw StatusError(CDCC_EINVAL, "null input pointer");
  const int n = nocc + nvir;
  c->hd = {nirrep, nocc, nvir, n, nchol};
  c->orb_irrep.assign(orb_irrep, orb_irrep + n);
  c->chol_irrep.assign(chol_irrep, chol_irrep + nchol);
  c->eps.assign(eps, eps + n);
  Dims& d = c->dims;
  d.h = nirrep;
  for (int p = 0; p < n; ++p) {
    const int g = orb_irrep[p];
    if (g < 0 || g >= nirrep)
      throw StatusError(CDCC_EINVAL, "orbital irrep out of range");
    if (p > 0 && p != nocc && orb_irrep[p - 1] > g)
      throw StatusError(CDCC_EINVAL,
                        "orbitals must be sorted by irrep within occ / vir");
    d.n[p < nocc ? SO : SV][g]++;
  }
  for (int P = 0; P < nchol; ++P) {
    const int g = chol_irrep[P];
    if (g < 0 || g >= nirrep)
      throw StatusError(CDCC_EINVAL, "Cholesky irrep out of range");
    if (P > 0 && chol_irrep[P - 1] > g)
      throw StatusError(CDCC_EINVAL, "Cholesky vectors must be sorted");
    d.n[SQ][g]++;
  }
  double emax_o = -1e300, emin_v = 1e300;
  for (int p = 0; p < n; ++p) {
    if (!std::isfinite(eps[p]))
      throw StatusError(CDCC_EINVAL, "non-finite orbital energy");
    if (p < nocc)
      emax_o = std::max(emax_o, eps[p]);
    else
      emin_v = std::min(emin_v, eps[p]);
  }
  if (!(emax_o < emin_v))
    throw StatusError(CDCC_EINVAL, "occupied and virtual energies overlap");
  int so = 0, sv = 0, sq = 0;
  for (int g = 0; g < nirrep; ++g) {
    d.n[SA][g] = d.n[SO][g] + d.n[SV][g];
    d.off_all[SO][g] = 0;
    d.off_all[SV][g] = d.n[SO][g];
    d.gstart[SO][g] = so;
    d.gstart[SV][g] = sv;
    d.gstart[SQ][g] = sq;
    so += d.n[SO][g];
    sv += d.n[SV][g];
    sq += d.n[SQ][g];
  }

  CK(cudaSetDevice(c->opt.device));
  c->st = (cudaStream_t)c->opt.stream;
  DevAlloc al;
  al.fa = c->opt.dev_alloc;
  al.ff = c->opt.dev_free;
  al.user = c->opt.alloc_user;
  c->eng = std::make_unique<Engine>(d, c->st, al);
  {
    const double pc = c->opt.perm_cache_gb;
    c->eng->set_perm_cache_bytes(pc > 0 && std::isfinite(pc)
                                     ? (int64_t)(std::min(pc, 1e6) * 1e9)
                                     : 0);
  }
  Engine& e = *c->eng;
  CK(cudaEventCreate(&c->ev0));
  CK(cudaEventCreate(&c->ev1));

  c->Lpk = e.tensor("Lpk", {SQ, SA, SA}, 1);
  c->nnz0 = c->Lpk->lay.size;
  if ((size_t)c->nnz0 != packed_size_g(c, 0))
    throw StatusError(CDCC_EINVAL, "internal: packed size mismatch");
  if (!is_device_ptr(L)) {
    // symmetry L^P_pq = L^P_qp inside the stored pattern
    std::vector<double> dense;
    const Layout& lay = c->Lpk->lay;
    double maxasym = 0;
    for (int gP = 0; gP < nirrep; ++gP) {
      const int64_t base = lay.blk_off[gP];
      const int64_t ncol = lay.ncol[gP];
      for (int64_t k = 0; k < lay.nrow[gP]; ++k) {
        const double* row = L + base + k * ncol;
        int64_t coff = 0;
        std::vector<int64_t> offs(nirrep);
        for (int gp = 0; gp < nirrep; ++gp) {
          offs[gp] = coff;
          coff += (int64_t)d.n[SA][gp] * d.n[SA][gp ^ gP];
        }
        for (int gp = 0; gp < nirrep; ++gp) {
          const int gq = gp ^ gP;
          const int np_ = d.n[SA][gp], nq = d.n[SA][gq];
          for (int p = 0; p < np_; ++p)
            for (int q = 0; q < nq; ++q) {
              const double a = row[offs[gp] + (int64_t)p * nq + q];
              const double b = row[offs[gq] + (int64_t)q * np_ + p];
              if (!std::isfinite(a))
                throw StatusError(CDCC_EINVAL, "non-finite Cholesky vector");
              maxasym = std::max(maxasym, std::fabs(a - b));
            }
        }
      }
    }
    if (maxasym > 1e-12)
      throw StatusError(CDCC_EINVAL, "L^P_pq is not symmetric in pq");
  }
  copy_in(c, c->Lpk->d, L, c->nnz0);
  // blocks of L (leaves of the tape)
  c->Loo = e.tensor("Loo", {SQ, SO, SO}, 1);
  c->Lov = e.tensor("Lov", {SQ, SO, SV}, 1);
  c->Lvo = e.tensor("Lvo", {SQ, SV, SO}, 1);
  c->Lvv = e.tensor("Lvv", {SQ, SV, SV}, 1);
  e.axpy(1.0, c->Lpk, "Ppq", 0.0, c->Loo, "Ppq");
  e.axpy(1.0, c->Lpk, "Ppq", 0.0, c->Lov, "Ppq");
  e.axpy(1.0, c->Lpk, "Ppq", 0.0, c->Lvo, "Ppq");
  e.axpy(1.0, c->Lpk, "Ppq", 0.0, c->Lvv, "Ppq");
  c->Loo->tag = c->Lov->tag = c->Lvo->tag = c->Lvv->tag = TAG_L;
  c->Loo->constant = c->Lov->constant = c->Lvo->constant =
      c->Lvv->constant = true;

  // identity on the occupied space
  c->Ioo = e.tensor("Ioo", {SO, SO}, 1);
  {
    std::vector<double> I((size_t)nocc * nocc, 0.0);
    for (int i = 0; i < nocc; ++i) I[(size_t)i * nocc + i] = 1.0;
    upload_dense(c, c->Ioo, I);
  }
  // core Hamiltonian h = diag(eps) - G(L), G = 2 L J - L_pk L_kq
  c->hoo = e.tensor("hoo", {SO, SO}, 1);
  c->hov = e.tensor("hov", {SO, SV}, 1);
  c->hvo = e.tensor("hvo", {SV, SO}, 1);
  c->hvv = e.tensor("hvv", {SV, SV}, 1);
  {
    std::vector<double> Eo((size_t)nocc * nocc, 0.0),
        Ev((size_t)nvir * nvir, 0.0);
    for (int i = 0; i < nocc; ++i) Eo[(size_t)i * nocc + i] = eps[i];
    for (int a = 0; a < nvir; ++a) Ev[(size_t)a * nvir + a] = eps[nocc + a];
    upload_dense(c, c->hoo, Eo);
    upload_dense(c, c->hvv, Ev);
    Tensor* J0 = e.tensor("J0", {SQ}, 1);
    e.contract(1.0, c->Loo, "Pkl", c->Ioo, "kl", 0.0, J0, "P");
    e.contract(-2.0, c->Loo, "Pij", J0, "P", 1.0, c->hoo, "ij");
    e.contract(1.0, c->Loo, "Pik", c->Loo, "Pkj", 1.0, c->hoo, "ij");
    e.contract(-2.0, c->Lov, "Pia", J0, "P", 0.0, c->hov, "ia");
    e.contract(1.0, c->Loo, "Pik", c->Lov, "Pka", 1.0, c->hov, "ia");
    e.contract(-2.0, c->Lvo, "Pai", J0, "P", 0.0, c->hvo, "ai");
    e.contract(1.0, c->Lvo, "Pak", c->Loo, "Pki", 1.0, c->hvo, "ai");
    e.contract(-2.0, c->Lvv, "Pab", J0, "P", 1.0, c->hvv, "ab");
    e.contract(1.0, c->Lvo, "Pak", c->Lov, "Pkb", 1.0, c->hvv, "ab");
  }
  c->hoo->tag = c->hov->tag = c->hvo->tag = c->hvv->tag = TAG_H;
  // ladder mode: the stored (ab|cd) integrals cost 8 bytes per element, the
  // density sweep adds their adjoint, and the tensor-core schedules cache
  // slices of both (factors below); on the fly only two row batches live
  {
    const Layout lw = e.layout({SV, SV, SV, SV}, 2);
    const double k = c->opt.precision == CDCC_PREC_TC      ? 4.5
                     : c->opt.precision == CDCC_PREC_MIXED ? 3.5
                                                           : 2.0;
    const double stored = 8.0 * (double)lw.size * k;
    size_t fre = 0, tot = 0;
    CK(cudaMemGetInfo(&fre, &tot));
    if (c->opt.ladder == CDCC_LADDER_STORED)
      c->otf = false;
    else if (c->opt.ladder == CDCC_LADDER_OTF)
      c->otf = true;
    else  // with an FP64 finish the on-the-fly build is FP64 DFMA work as
          // large as the ladder itself, so stored is kept up to 75 %
      c->otf = stored > (c->opt.precision == CDCC_PREC_TC ? 0.4 : 0.75) *
                            (double)fre;
    const double gb = c->opt.ladder_batch_gb > 0 ? c->opt.ladder_batch_gb
                                                 : 2.0;
    e.ladder_batch_bytes = (int64_t)(gb * 1e9);
    e.set_ladder_pm(c->opt.ladder_pm != 0);
  }
  {
    std::vector<double> h = to_host(c, c->hoo);
    double tr = 0;
    // trace over the diagonal blocks (rows == cols inside each irrep)
    visit_dense(c->hoo->lay, c->dims, [&](int64_t off, int64_t di) {
      if (di / nocc == di % nocc) tr += h[off];
    });
    double se = 0;
    for (int i = 0; i < nocc; ++i) se += eps[i];
    c->e_ref = tr + se;
  }
  // amplitude, residual and multiplier vectors [x1 | x2]
  const Layout l1 = e.layout({SO, SV}, 1);
  const Layout l2 = e.layout({SO, SO, SV, SV}, 2);
  const int64_t na = l1.size + l2.size;
  c->amp = e.flat("amp", na);
  c->T1 = e.view("T1", c->amp, 0, {SO, SV}, 1);
  c->T2 = e.view("T2", c->amp, l1.size, {SO, SO, SV, SV}, 2);
  c->amp->tag = TAG_AMP;
  c->T1->tag = c->T2->tag = TAG_AMP;
  c->res = e.flat("res", na);
  c->R1 = e.view("R1", c->res, 0, {SO, SV}, 1);
  c->R2 = e.view("R2", c->res, l1.size, {SO, SO, SV, SV}, 2);
  c->lam = e.flat("lam", na);
  c->L1 = e.view("L1", c->lam, 0, {SO, SV}, 1);
  c->L2 = e.view("L2", c->lam, l1.size, {SO, SO, SV, SV}, 2);
  c->err1 = e.flat("err", na);
  c->E = e.tensor("E", {}, 0);
  c->Gam = e.tensor("Gam", {SQ, SA, SA}, 1);
  c->Gsym = e.tensor("Gsym", {SQ, SA, SA}, 1);
  c->D1a = e.tensor("D1a", {SA, SA}, 1);
  c->D1s = e.tensor("D1s", {SA, SA}, 1);
  // small device scalars
  c->d_eps = (double*)e.al.alloc((size_t)n * 8);
  CK(cudaMemcpyAsync(c->d_eps, eps, (size_t)n * 8, cudaMemcpyHostToDevice,
                     c->st));
  c->d_max = (unsigned long long*)e.al.alloc(8);
  c->d_dots = (double*)e.al.alloc(16 * 8);
  c->partial_n = multi_dot_partial_doubles(na, 16);
  c->d_partial = (double*)e.al.alloc((size_t)c->partial_n * 8);
  c->d_err = (unsigned int*)e.al.alloc(16);
  CK(cudaMemsetAsync(c->d_err, 0, 16, c->st));
  e.d_err = c->d_err;
  CK(cudaStreamSynchronize(c->st));
  c->state = 1;
}

template <class F>
cdcc_status guarded(cdcc_ctx* c, F f) {
  try {
    f();
    return CDCC_OK;
  } catch (const StatusError& s) {
    if (c) c->err = s.m;
    return s.s;
  } catch (const EngineError& e) {
    if (c) c->err = e.msg;
    const std::string& m = e.msg;
    if (m.find("alloc") != std::string::npos ||
        m.find("out of memory") != std::string::npos)
      return CDCC_ENOMEM;
    if (m.rfind("CUDA", 0) == 0) return CDCC_ECUDA;
    return CDCC_EINVAL;
  } catch (const std::bad_alloc&) {
    if (c) c->err = "host allocation failed";
    return CDCC_ENOMEM;
  } catch (const std::exception& e) {
    if (c) c->err = e.what();
    return CDCC_EINVAL;
  }
}

void free_ctx(cdcc_ctx* c) {
  if (!c) return;
  if (c->eng) {
    Engine& e = *c->eng;
    e.al.release(c->d_eps, (size_t)c->hd.n * 8);
    e.al.release(c->d_max, 8);
    e.al.release(c->d_dots, 16 * 8);
    e.al.release(c->d_partial, (size_t)c->partial_n * 8);
    e.al.release(c->d_err, 16);
    free_denom(c, c->den[0]);
    free_denom(c, c->den[1]);
    // optional per-contraction trace of the profiled work of this context
    if (const char* f = std::getenv("CDCC_TRACE")) e.write_trace(f);
    cudaStreamSynchronize(c->st);
    c->eng.reset();
  }
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  cudaStreamSynchronize(c->st);
  delete c;
}

}  // namespace

extern "C" {

cdcc_status cdcc_ladder_pm_tables(int nirrep, const int32_t* nocc_irrep,
                                  const int32_t* nvir_irrep, double batch_gb,
                                  int32_t* out, int64_t cap, int64_t* len) {
  if (!nocc_irrep || !nvir_irrep || !len || !(batch_gb > 0) ||
      !std::isfinite(batch_gb))
    return CDCC_EINVAL;
  if (nirrep != 1 && nirrep != 2 && nirrep != 4 && nirrep != 8)
    return CDCC_EINVAL;
  try {
    Dims d;
    d.h = nirrep;
    for (int g = 0; g < nirrep; ++g) {
      if (nocc_irrep[g] < 0 || nvir_irrep[g] < 0 || nocc_irrep[g] > 4096 ||
          nvir_irrep[g] > 4096)
        return CDCC_EINVAL;
      d.n[SO][g] = nocc_irrep[g];
      d.n[SV][g] = nvir_irrep[g];
    }
    Layout TL;
    TL.rank = 4;
    TL.sp[0] = SO;
    TL.sp[1] = SO;
    TL.sp[2] = SV;
    TL.sp[3] = SV;
    TL.split = 2;
    TL.gtot = 0;
    TL.build(d);
    PmPlan P;
    std::vector<int> tab;
    pm_host_tables(TL, d, (int64_t)std::min(batch_gb * 1e9, 1e15), P, tab);
    std::vector<int32_t> o;
    for (int G = 0; G < nirrep; ++G) {
      if (P.uo[G] == 0 || P.uv[G] == 0) continue;
      int nb = 0;
      for (const PmBatch& pb : P.batches) nb += pb.b.G == G;
      o.insert(o.end(), {G, P.uo[G], P.uv[G], nb, (int32_t)TL.nrow[G],
                         (int32_t)TL.ncol[G]});
      o.insert(o.end(), tab.begin() + P.orow[G],
               tab.begin() + P.orow[G] + 2 * P.uo[G]);
      o.insert(o.end(), tab.begin() + P.vcol[G],
               tab.begin() + P.vcol[G] + 2 * P.uv[G]);
      for (const PmBatch& pb : P.batches) {
        if (pb.b.G != G) continue;
        o.insert(o.end(), {pb.b.ga, pb.b.a0, pb.b.a1, pb.nv});
        o.insert(o.end(), tab.begin() + pb.vrow,
                 tab.begin() + pb.vrow + 3 * pb.nv);
      }
    }
    *len = (int64_t)o.size();
    if (out) {
      if (cap < (int64_t)o.size()) return CDCC_ENOMEM;
      std::memcpy(out, o.data(), o.size() * sizeof(int32_t));
    }
    return CDCC_OK;
  } catch (const EngineError&) {
    return CDCC_EINVAL;
  } catch (const std::bad_alloc&) {
    return CDCC_ENOMEM;
  }
}

void cdcc_default_options(cdcc_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->conv_tol = 1e-10;
  o->energy_tol = 1e-12;
  o->max_iter = 100;
  o->diis_dim = 8;
  o->precision = CDCC_PREC_FP64;
  o->switch_tol = 1e-6;
  o->device = 0;
  o->stream = nullptr;
  o->ladder = CDCC_LADDER_AUTO;
  o->ladder_batch_gb = 2.0;
  o->fock_model = CDCC_FIXED_CORE;
  o->ladder_linearize = 1;
  o->perm_cache_gb = 32.0;
  o->ladder_slices_gb = 48.0;
  o->ladder_pm = 1;
  o->relaxed = 0;
}

cdcc_status cd_ccsd_init(cdcc_ctx** out, int nirrep, int nocc, int nvir,
                         int nchol, const int32_t* orb_irrep,
                         const double* eps, const int32_t* chol_irrep,
                         const double* L, const cdcc_options* opt) {
  if (!out) return CDCC_EINVAL;
  *out = nullptr;
  cdcc_ctx* c = new (std::nothrow) cdcc_ctx();
  if (!c) return CDCC_ENOMEM;
  if (opt)
    c->opt = *opt;
  else
    cdcc_default_options(&c->opt);
  if (c->opt.max_iter <= 0) c->opt.max_iter = 100;
  cdcc_status s = guarded(c, [&] {
    if (c->opt.precision < CDCC_PREC_FP64 || c->opt.precision > CDCC_PREC_TC ||
        c->opt.ladder < CDCC_LADDER_AUTO || c->opt.ladder > CDCC_LADDER_OTF ||
        c->opt.fock_model < CDCC_FIXED_CORE ||
        c->opt.fock_model > CDCC_FROZEN_FOCK)
      throw StatusError(CDCC_EINVAL,
                        "unknown precision, ladder mode or Fock model");
    if (c->opt.relaxed != 0 &&
        (c->opt.relaxed != 1 || c->opt.fock_model != CDCC_FIXED_CORE))
      throw StatusError(CDCC_EINVAL,
                        "orbital relaxation is defined for the fixed-core "
                        "model only (relaxed = 0 or 1)");
    init_ctx(c, nirrep, nocc, nvir, nchol, orb_irrep, eps, chol_irrep, L);
  });
  *out = c;  // also on error, so that cdcc_last_error can be read
  return s;
}

size_t cdcc_packed_size(const cdcc_ctx* c, int gx) {
  if (!c || c->state < 1 || gx < 0 || gx >= c->hd.h) return 0;
  return packed_size_g(c, gx);
}

cdcc_status ccsd_solve(cdcc_ctx* c, double* e_corr, int* iters,
                       double* resid) {
  if (!c || c->state < 1) return CDCC_ESTATE;
  return guarded(c, [&] { run_ccsd(c, e_corr, iters, resid); });
}

cdcc_status lambda_solve(cdcc_ctx* c, int* iters, double* resid) {
  if (!c) return CDCC_EINVAL;
  if (c->state < 2) {
    c->err = "lambda_solve before ccsd_solve";
    return CDCC_ESTATE;
  }
  return guarded(c, [&] { run_lambda(c, iters, resid); });
}

cdcc_status build_density(cdcc_ctx* c, double* D1) {
  if (!c) return CDCC_EINVAL;
  if (c->state < 3) {
    c->err = "build_density before lambda_solve";
    return CDCC_ESTATE;
  }
  return guarded(c, [&] { run_density(c, D1); });
}

cdcc_status cdcc_get_gamma(cdcc_ctx* c, double* gamma) {
  if (!c || !gamma) return CDCC_EINVAL;
  if (c->state < 4) return CDCC_ESTATE;
  return guarded(c, [&] {
    CK(cudaMemcpyAsync(gamma, c->Gsym->d, (size_t)c->nnz0 * 8,
                       cudaMemcpyDefault, c->st));
    CK(cudaStreamSynchronize(c->st));
  });
}

cdcc_status contract_dL(cdcc_ctx* c, int nx, const int32_t* x_irrep,
                        const double* dL, double* g) {
  if (!c) return CDCC_EINVAL;
  if (c->state < 4) {
    c->err = "contract_dL before build_density";
    return CDCC_ESTATE;
  }
  if (nx < 0 || (nx > 0 && (!dL || !g))) return CDCC_EINVAL;
  if (nx == 0) return CDCC_OK;
  return guarded(c, [&] { run_contract(c, nx, x_irrep, dL, g); });
}

cdcc_status cdcc_error_estimate(cdcc_ctx* c, int nx, const int32_t* x_irrep,
                                const double* dL, double* dE, double* dg) {
  if (!c || !dE) return CDCC_EINVAL;
  if (c->state < 4) {
    c->err = "cdcc_error_estimate before build_density";
    return CDCC_ESTATE;
  }
  if (nx < 0 || (nx > 0 && (!dL || !dg))) return CDCC_EINVAL;
  return guarded(c, [&] { run_error_estimate(c, nx, x_irrep, dL, dE, dg); });
}

size_t cdcc_metric_size(const cdcc_ctx* c) {
  if (!c || c->state < 1) return 0;
  size_t s = 0;
  for (int G = 0; G < c->hd.h; ++G)
    s += (size_t)c->dims.n[SQ][G] * c->dims.n[SQ][G];
  return s;
}

cdcc_status contract_df(cdcc_ctx* c, const double* metric, int nx,
                        const double* dB, const double* dM, double* g) {
  if (!c || !metric) return CDCC_EINVAL;
  if (c->state < 4) {
    c->err = "contract_df before build_density";
    return CDCC_ESTATE;
  }
  if (nx < 0 || (nx > 0 && (!dB || !dM || !g))) return CDCC_EINVAL;
  return guarded(c, [&] { run_contract_df(c, metric, nx, dB, dM, g); });
}

cdcc_status cdcc_energy_error(cdcc_ctx* c, double* dE) {
  if (!c || !dE) return CDCC_EINVAL;
  if (c->state < 3) {
    c->err = "cdcc_energy_error before lambda_solve";
    return CDCC_ESTATE;
  }
  return guarded(c, [&] { run_energy_error(c, dE); });
}

cdcc_status gradient(cdcc_ctx* c, int nx, const int32_t* x_irrep,
                     const double* dL, double* e_corr, double* g) {
  if (!c || c->state < 1) return CDCC_ESTATE;
  cdcc_status s = CDCC_OK;
  if (c->state < 2) s = ccsd_solve(c, e_corr, nullptr, nullptr);
  if (s != CDCC_OK) return s;
  if (e_corr) *e_corr = c->e_corr;
  if (c->state < 3) s = lambda_solve(c, nullptr, nullptr);
  if (s != CDCC_OK) return s;
  if (c->state < 4) s = build_density(c, nullptr);
  if (s != CDCC_OK) return s;
  return contract_dL(c, nx, x_irrep, dL, g);
}

cdcc_status cdcc_get_amplitudes(cdcc_ctx* c, int which, double* out) {
  if (!c || !out || which < 0 || which > 3) return CDCC_EINVAL;
  if ((which < 2 && c->state < 2) || (which >= 2 && c->state < 3))
    return CDCC_ESTATE;
  return guarded(c, [&] {
    Tensor* t = which == 0 ? c->T1 : which == 1 ? c->T2
              : which == 2 ? c->L1 : c->L2;
    std::vector<double> h = to_host(c, t);
    const int o = c->hd.nocc, v = c->hd.nvir;
    const size_t n = which % 2 == 0 ? (size_t)o * v : (size_t)o * o * v * v;
    std::memset(out, 0, n * 8);
    visit_dense(t->lay, c->dims,
                [&](int64_t off, int64_t di) { out[di] = h[off]; });
  });
}

cdcc_status cdcc_phase_times(cdcc_ctx* c, double* t4) {
  if (!c || !t4) return CDCC_EINVAL;
  for (int i = 0; i < 4; ++i) t4[i] = c->phase[i];
  return CDCC_OK;
}

cdcc_status cdcc_profile(cdcc_ctx* c, int enable) {
  if (!c || !c->eng) return CDCC_EINVAL;
  return guarded(c, [&] {
    c->eng->prof_collect();
    c->eng->profile(enable != 0);
  });
}

cdcc_status cdcc_kernel_stats(cdcc_ctx* c, int kind, double* seconds,
                              long long* launches, double* work) {
  if (!c || !c->eng || kind < 0 || kind >= Engine::K_NKIND)
    return CDCC_EINVAL;
  return guarded(c, [&] {
    c->eng->prof_collect();
    if (seconds) *seconds = c->eng->prof_sec[kind];
    if (launches) *launches = (long long)c->eng->prof_n[kind];
    if (work) *work = c->eng->prof_work[kind];
  });
}

cdcc_status cdcc_ladder_stats(cdcc_ctx* c, double* seconds, double* flops,
                              long long* calls) {
  if (!c || !c->eng || !seconds || !flops || !calls) return CDCC_EINVAL;
  return guarded(c, [&] {
    int64_t n = 0;
    c->eng->ladder_stats(seconds, flops, &n);
    *calls = (long long)n;
  });
}

cdcc_status cdcc_ladder_mode(cdcc_ctx* c, int* mode) {
  if (!c || !mode) return CDCC_EINVAL;
  *mode = c->otf ? CDCC_LADDER_OTF : CDCC_LADDER_STORED;
  return CDCC_OK;
}

cdcc_status cdcc_solver_info(cdcc_ctx* c, int* info) {
  if (!c || !info) return CDCC_EINVAL;
  info[0] = c->iters_mixed[0];
  info[1] = c->iters_fp64[0];
  info[2] = c->iters_mixed[1];
  info[3] = c->iters_fp64[1];
  return CDCC_OK;
}

cdcc_status cdcc_dgemm(int transA, int transB, int M, int N, int K,
                       double alpha, const double* A, int lda,
                       const double* B, int ldb, double beta, double* C,
                       int ldc, int mode, void* stream) {
  if (M < 0 || N < 0 || K < 0 || mode < 0 || (mode > 3 && mode < 12) ||
      mode > 14)
    return CDCC_EINVAL;
  if (M == 0 || N == 0) return CDCC_OK;
  if (!A || !B || !C) return CDCC_EINVAL;
  if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(C))
    return CDCC_EINVAL;
  const int rowsA = transA ? K : M, colsA = transA ? M : K;
  const int rowsB = transB ? N : K, colsB = transB ? K : N;
  if (lda < std::max(1, colsA) || ldb < std::max(1, colsB) || ldc < N)
    return CDCC_EINVAL;
  (void)rowsA;
  (void)rowsB;
  cudaStream_t st = (cudaStream_t)stream;
  GemmProb g;
  std::memset(&g, 0, sizeof(g));
  g.A = A;
  g.B = B;
  g.C = C;
  g.M = M;
  g.N = N;
  g.K = K;
  g.lda = lda;
  g.ldb = ldb;
  g.ldc = ldc;
  g.ta = transA ? 1 : 0;
  g.tb = transB ? 1 : 0;
  void* ws = nullptr;
  double* sk = nullptr;
  unsigned int* err = nullptr;
  cdcc_status s = CDCC_OK;
  try {
    if (mode == 0) {
      const int64_t n = gemm_scratch_doubles(&g, 1);
      if (n > 0) CK(cudaMallocAsync((void**)&sk, (size_t)n * 8, st));
      gemm64_grouped(&g, 1, alpha, beta, sk, st);
    } else if (mode >= 12) {
      const int64_t wb = oz_workspace_bytes(&g, 1, mode - 10);
      CK(cudaMallocAsync(&ws, (size_t)wb, st));
      CK(cudaMallocAsync((void**)&err, 16, st));
      CK(cudaMemsetAsync(err, 0, 16, st));
      oz_gemm_grouped(&g, 1, alpha, beta, mode - 10, ws, err, st);
    } else {
      const int64_t wb = tc_workspace_bytes(&g, 1, mode);
      const int64_t n = tc_scratch_doubles(&g, 1, mode);
      CK(cudaMallocAsync(&ws, (size_t)wb, st));
      if (n > 0) CK(cudaMallocAsync((void**)&sk, (size_t)n * 8, st));
      CK(cudaMallocAsync((void**)&err, 16, st));
      CK(cudaMemsetAsync(err, 0, 16, st));
      tc_gemm_grouped(&g, 1, alpha, beta, mode, ws, sk, err, st);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    if (err) {
      unsigned int h = 0;
      CK(cudaMemcpy(&h, err, 4, cudaMemcpyDeviceToHost));
      if (h) s = CDCC_ETIMEOUT;
    }
  } catch (const std::exception&) {
    s = CDCC_ECUDA;
  }
  if (ws) cudaFreeAsync(ws, st);
  if (sk) cudaFreeAsync(sk, st);
  if (err) cudaFreeAsync(err, st);
  cudaStreamSynchronize(st);
  return s;
}

long long cdcc_kernel_launches(const cdcc_ctx* c) {
  return c && c->eng ? (long long)c->eng->launches : 0;
}

const char* cdcc_last_error(const cdcc_ctx* c) {
  return c ? c->err.c_str() : "null context";
}

void cd_ccsd_free(cdcc_ctx* c) { free_ctx(c); }

}  // extern "C"
