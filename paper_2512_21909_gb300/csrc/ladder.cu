// ladder.cu -- particle-particle ladder with the (ab|cd) integrals assembled
// on the fly from the virtual-virtual Cholesky vectors (Sec. 2.3).
//
// For the pair irrep G the ladder is the product R_G[(ij),(ab)] +=
// T_G[(ij),(cd)] W_G[(ab),(cd)]^T with W[a,b,c,d] = (ac|bd) =
// sum_P L[P,a,c] L[P,b,d].  W_G is symmetric (every L^P is), so it is built
// one row batch at a time: the rows (a,b) with a in [a0,a1) of irrep ga and
// b of irrep gb = ga^G.  For each irrep gc of c (gd = gc^G, the Cholesky
// irrep is Gp = ga^gc) one GEMM over P gives
//     X_gc[(a,c),(b,d)] = sum_P L_Gp[P,(a,c)] L_Gp[P,(b,d)],
// all gc in one grouped launch; a permutation writes the batch rows
// W[(a,b),(c,d)], and one GEMM applies them.  Peak memory is two batches
// instead of sum_G N_vv(G)^2 doubles.
//
// Adjoint (Lambda iterations and the density sweep), with dR the adjoint of R:
//   dT_G[(ij),(cd) in batch] += dR_G[(ij),(ab)] W[(ab),(cd) in batch]
//        = dR_G W_batch^T                      (W symmetric: same as forward)
//   dW_batch[(ab),(cd)] = sum_ij dR_G[ij,(ab) in batch] T_G[ij,(cd)]
//   dL[P,a,c] += sum_bd dW[a,b,c,d] L[P,b,d],  dL[P,b,d] += sum_ac dW[a,b,c,d]
//        L[P,a,c]                              (two launches: their targets
//                                               overlap when ga == gb)
#include <algorithm>
#include <cstring>
#include <sstream>

#include "engine.h"

namespace cdcc {

#define LCK(x)                                                            \
  do {                                                                    \
    cudaError_t e_ = (x);                                                 \
    if (e_ != cudaSuccess)                                                \
      throw EngineError(std::string("CUDA: ") + cudaGetErrorString(e_) + \
                        " at " #x);                                       \
  } while (0)

namespace {

bool is_doubles(const Layout& L) {
  return L.rank == 4 && L.split == 2 && L.gtot == 0 && L.sp[0] == SO &&
         L.sp[1] == SO && L.sp[2] == SV && L.sp[3] == SV;
}

bool is_lvv(const Layout& L) {
  return L.rank == 3 && L.split == 1 && L.gtot == 0 && L.sp[0] == SQ &&
         L.sp[1] == SV && L.sp[2] == SV;
}

void check_block(const GemmProb& g, const double* a0, int64_t asz,
                 const double* b0, int64_t bsz, const double* c0,
                 int64_t csz) {
  // last element touched by each operand (row-major blocks with leading
  // dimensions lda/ldb/ldc; ta/tb swap the stored shape)
  const int64_t ar = g.ta ? g.K : g.M, ac = g.ta ? g.M : g.K;
  const int64_t br = g.tb ? g.N : g.K, bc = g.tb ? g.K : g.N;
  const int64_t ea = (g.A - a0) + (ar - 1) * g.lda + ac;
  const int64_t eb = (g.B - b0) + (br - 1) * g.ldb + bc;
  const int64_t ec = (g.C - c0) + (int64_t)(g.M - 1) * g.ldc + g.N;
  if (g.A < a0 || g.B < b0 || g.C < c0 || ea > asz || eb > bsz || ec > csz ||
      ac > g.lda || bc > g.ldb || g.N > g.ldc)
    throw EngineError("internal: ladder GEMM block out of bounds");
}

}  // namespace

std::vector<LadBatch> Engine::ladder_batches(const Layout& TL) {
  return ladder_batch_list(TL, dims_, ladder_batch_bytes);
}

std::vector<LadBatch> ladder_batch_list(const Layout& TL, const Dims& dims_,
                                        int64_t ladder_batch_bytes) {
  std::vector<LadBatch> out;
  const int h = dims_.h;
  for (int G = 0; G < h; ++G) {
    const int64_t ncol = TL.ncol[G];
    if (ncol == 0 || TL.nrow[G] == 0) continue;
    const int64_t max_rows =
        std::max<int64_t>(1, ladder_batch_bytes / (8 * ncol));
    for (int ga = 0; ga < h; ++ga) {
      const int gb = ga ^ G;
      const int na = dims_.n[SV][ga], nb = dims_.n[SV][gb];
      if (na == 0 || nb == 0) continue;
      const int step = (int)std::max<int64_t>(
          1, std::min<int64_t>(na, max_rows / nb));
      for (int a0 = 0; a0 < na; a0 += step) {
        const int a1 = std::min(na, a0 + step);
        out.push_back({G, ga, a0, a1, (int64_t)(a1 - a0) * nb});
      }
    }
  }
  return out;
}

void Engine::ladder_reserve(int64_t n) {
  if (n <= lad_n_) return;
  if (lad_x_) al.release(lad_x_, (size_t)lad_n_ * 8);
  if (lad_w_) al.release(lad_w_, (size_t)lad_n_ * 8);
  lad_x_ = lad_w_ = nullptr;
  lad_n_ = 0;
  lad_x_ = (double*)al.alloc((size_t)n * 8);
  lad_w_ = (double*)al.alloc((size_t)n * 8);
  lad_n_ = n;
}

// X_gc blocks of one batch: [a][c][b][d] for gc = 0..h-1, back to back.
// forward: lad_x_ -> W rows [(a,b)][(c,d)] (leading dimension N_vv(G));
// inverse: the same elements read from W and written to X.
// One CTA per (a,c) row of an X_gc block: it reads (or writes) that row
// contiguously and writes (reads) nb contiguous segments of nd elements,
// one per W row (a,b).
void Engine::ladder_perm(const LadBatch& b, bool inverse, const double* src,
                         double* dst) {
  const int h = dims_.h, G = b.G, gb = b.ga ^ G;
  LadPerm P;
  std::memset(&P, 0, sizeof(P));
  P.na = b.a1 - b.a0;
  P.nb = dims_.n[SV][gb];
  int64_t ncol = 0, xoff = 0;
  int rows = 0;
  for (int gc = 0; gc < h; ++gc) {
    const int nc = dims_.n[SV][gc], nd = dims_.n[SV][gc ^ G];
    P.coff[gc] = ncol;
    P.xoff[gc] = xoff;
    P.nc[gc] = nc;
    P.nd[gc] = nd;
    P.row0[gc] = rows;
    rows += P.na * nc * (nd > 0 && P.nb > 0 ? 1 : 0);
    ncol += (int64_t)nc * nd;
    xoff += (int64_t)P.na * nc * P.nb * nd;
  }
  P.row0[h] = rows;
  P.h = h;
  P.ncol = ncol;
  if (xoff != b.rows * ncol || b.rows * ncol > lad_n_)
    throw EngineError("internal: ladder batch size mismatch");
  if (rows == 0) return;
  timed(K_PERM, 16.0 * (double)b.rows * ncol, [&] {
    return ladder_permute(P, inverse, src, dst, rows, st_);
  });
}

// W rows of batch b into lad_w_ (via lad_x_); returns the GEMM flops.
double Engine::ladder_build(const LadBatch& b, Tensor* L) {
  const int h = dims_.h, G = b.G, ga = b.ga, gb = ga ^ G;
  const int na = b.a1 - b.a0, nb = dims_.n[SV][gb];
  const Layout& LL = L->lay;
  GemmProb probs[GEMM_MAXPROB];
  int np = 0;
  int64_t xoff = 0;
  bool holes = false;
  for (int gc = 0; gc < h; ++gc) {
    const int gd = gc ^ G, Gp = ga ^ gc;
    const int nc = dims_.n[SV][gc], nd = dims_.n[SV][gd];
    const int64_t M = (int64_t)na * nc, N = (int64_t)nb * nd;
    const int64_t K = LL.nrow[Gp];
    if (M * N == 0) continue;
    if (K == 0) {
      holes = true;          // (ac|bd) = 0 for an empty Cholesky irrep
      xoff += M * N;
      continue;
    }
    const int64_t ld = LL.ncol[Gp];
    GemmProb g;
    std::memset(&g, 0, sizeof(g));
    g.A = L->d + LL.blk_off[Gp] + LL.csub[Gp * LL.ncode_c + ga] +
          (int64_t)b.a0 * nc;
    g.ta = 1;
    g.lda = (int)ld;
    g.B = L->d + LL.blk_off[Gp] + LL.csub[Gp * LL.ncode_c + gb];
    g.tb = 0;
    g.ldb = (int)ld;
    g.C = lad_x_ + xoff;
    g.ldc = (int)N;
    g.M = (int)M;
    g.N = (int)N;
    g.K = (int)K;
    check_block(g, L->d, LL.size, L->d, LL.size, lad_x_, lad_n_);
    probs[np++] = g;
    xoff += M * N;
  }
  if (holes) LCK(cudaMemsetAsync(lad_x_, 0, (size_t)xoff * 8, st_));
  double fl = 0;
  if (np > 0) {
    const Mat ml{L->d, &LL, false, L};
    run_gemms(probs, np, ml, ml, 1.0, 0.0);
    for (int i = 0; i < np; ++i)
      fl += 2.0 * probs[i].M * (double)probs[i].N * probs[i].K;
  }
  ladder_perm(b, false, lad_x_, lad_w_);
  return fl;
}

namespace {
bool tc_shape(int64_t M, int64_t N, int64_t K) {
  return std::min(M, N) >= 32 && std::max(M, N) >= 64 && K >= 32;
}
}  // namespace

bool Engine::ladder_fusable(const LadBatch& b, const Layout& TL,
                            const Layout& LL) {
  const int prec = active_precision();
  if (prec < 1 || prec > 3 || !d_err) return false;
  const int G = b.G, ga = b.ga, gb = ga ^ G;
  if (!tc_shape(TL.nrow[G], b.rows, TL.ncol[G])) return false;
  const int na = b.a1 - b.a0, nb = dims_.n[SV][gb];
  for (int gc = 0; gc < dims_.h; ++gc) {
    const int gd = gc ^ G, Gp = ga ^ gc;
    const int64_t M = (int64_t)na * dims_.n[SV][gc];
    const int64_t N = (int64_t)nb * dims_.n[SV][gd];
    const int64_t K = LL.nrow[Gp];
    if (M * N == 0 || K == 0) continue;
    if (!tc_shape(M, N, K)) return false;
  }
  return true;
}

// Batch rows of (ab|cd) as ns BF16 slices [ns][rows][Kp] (lad_ws_), written
// by the epilogue of the build GEMM; returns its flops.
double Engine::ladder_build_sliced(const LadBatch& b, Tensor* L, int ns,
                                   void* dst) {
  const int h = dims_.h, G = b.G, ga = b.ga, gb = ga ^ G;
  const int na = b.a1 - b.a0, nb = dims_.n[SV][gb];
  const Layout& LL = L->lay;
  int64_t ncol = 0;
  for (int gc = 0; gc < h; ++gc)
    ncol += (int64_t)dims_.n[SV][gc] * dims_.n[SV][gc ^ G];
  const int64_t Kp = slice_kp((int)ncol);
  const size_t need = (size_t)ns * b.rows * Kp * 2;
  if ((int64_t)ns * b.rows * Kp >= ((int64_t)1 << 31))
    throw EngineError("ladder batch too large for 32-bit slice offsets");
  if (!dst && need > lad_ws_bytes_) {
    if (lad_ws_) al.release(lad_ws_, lad_ws_bytes_);
    lad_ws_ = al.alloc(need);
    lad_ws_bytes_ = need;
  }
  void* W = dst ? dst : lad_ws_;
  // zero padding columns [ncol, Kp) and, for an irrep without Cholesky
  // vectors, the whole batch ((ac|bd) = 0 there)
  bool holes = false;
  for (int gc = 0; gc < h; ++gc) {
    const int64_t M = (int64_t)na * dims_.n[SV][gc];
    const int64_t N = (int64_t)nb * dims_.n[SV][gc ^ G];
    if (M * N > 0 && LL.nrow[ga ^ gc] == 0) holes = true;
  }
  if (holes)
    LCK(cudaMemsetAsync(W, 0, need, st_));
  else if (Kp > ncol)
    LCK(cudaMemset2DAsync((uint8_t*)W + ncol * 2, (size_t)Kp * 2, 0,
                          (size_t)(Kp - ncol) * 2, (size_t)ns * b.rows, st_));
  TcProb tp[GEMM_MAXPROB];
  TcLadEpi ep[GEMM_MAXPROB];
  int np = 0;
  int64_t coff = 0, wsb = 1024;
  for (int gc = 0; gc < h; ++gc) {
    const int gd = gc ^ G, Gp = ga ^ gc;
    const int nc = dims_.n[SV][gc], nd = dims_.n[SV][gd];
    const int64_t M = (int64_t)na * nc, N = (int64_t)nb * nd;
    if (M * N > 0 && LL.nrow[Gp] > 0)
      wsb += (int64_t)ns * (M + N) * slice_kp((int)LL.nrow[Gp]) * 2 + 8192;
  }
  uint8_t* cur = (uint8_t*)scratch((wsb + 7) / 8);
  double fl = 0;
  for (int gc = 0; gc < h; ++gc) {
    const int gd = gc ^ G, Gp = ga ^ gc;
    const int nc = dims_.n[SV][gc], nd = dims_.n[SV][gd];
    const int64_t M = (int64_t)na * nc, N = (int64_t)nb * nd;
    const int64_t K = LL.nrow[Gp];
    const int64_t c0 = coff;
    coff += (int64_t)nc * nd;
    if (M * N == 0 || K == 0) continue;
    const int64_t ld = LL.ncol[Gp];
    const double* A = L->d + LL.blk_off[Gp] + LL.csub[Gp * LL.ncode_c + ga] +
                      (int64_t)b.a0 * nc;
    const double* B = L->d + LL.blk_off[Gp] + LL.csub[Gp * LL.ncode_c + gb];
    // both operands are K x (rows) blocks of L with leading dimension ld
    if (M > ld || N > ld || (A - L->d) + (K - 1) * ld + M > LL.size ||
        (B - L->d) + (K - 1) * ld + N > LL.size)
      throw EngineError("internal: ladder build block out of bounds");
    // op(A) rows (a,c) = columns of L (K-major slices of L^T), op(B)^T rows
    // (b,d) likewise; both cached with L
    TcProb& t = tp[np];
    std::memset(&t, 0, sizeof(t));
    t.a = slice_side(L, A, (int)M, (int)K, ld, 1, ns, false, &cur);
    t.b = slice_side(L, B, (int)N, (int)K, ld, 1, ns, false, &cur);
    t.M = (int)M;
    t.N = (int)N;
    t.K = (int)K;
    t.ldc = (int)N;
    TcLadEpi& e = ep[np];
    e.W = W;
    e.rows = b.rows;
    e.Kp = Kp;
    e.coff = c0;
    e.nc = nc;
    e.nd = nd;
    e.nb = nb;
    e.ns = ns;
    ++np;
    fl += 2.0 * M * (double)N * K;
  }
  if (coff != ncol) throw EngineError("internal: ladder column count");
  if (np > 0) {
    tc_flops += (int64_t)fl;
    timed(K_TC, fl, [&] {
      return tc_gemm_ladder(tp, np, ns, ep, d_err, st_);
    });
  }
  return fl;
}

// Y_G[(ij), (ab) in batch] += alpha * X_G[(ij),(cd)] W_batch^T with the
// batch rows already in slices (lad_ws_)
void Engine::ladder_apply_sliced(const LadBatch& b, double alpha, Tensor* X,
                                 Tensor* Y, int ns, const void* W) {
  const Layout& XL = X->lay;
  const int G = b.G;
  const int64_t M = XL.nrow[G], K = XL.ncol[G];
  if (M == 0) return;
  const int gb = b.ga ^ G;
  const double* A = X->d + XL.blk_off[G];
  double* C = Y->d + Y->lay.blk_off[G] + Y->lay.csub[G * Y->lay.ncode_c + b.ga] +
              (int64_t)b.a0 * dims_.n[SV][gb];
  {
    GemmProb g;
    std::memset(&g, 0, sizeof(g));
    g.A = A;
    g.lda = (int)K;
    g.B = nullptr;
    g.C = C;
    g.ldc = (int)K;
    g.M = (int)M;
    g.N = (int)b.rows;
    g.K = (int)K;
    // A and C inside their tensors (B is the slice buffer)
    const int64_t ea = (A - X->d) + (M - 1) * K + K;
    const int64_t ec = (C - Y->d) + (M - 1) * K + b.rows;
    if (ea > XL.size || ec > Y->lay.size)
      throw EngineError("internal: ladder apply out of bounds");
  }
  const int64_t Kp = slice_kp((int)K);
  uint8_t* cur = (uint8_t*)scratch(
      ((int64_t)ns * M * Kp * 2 + M * 4 + 8192 + 7) / 8);
  TcProb t;
  std::memset(&t, 0, sizeof(t));
  t.a = slice_side(X, A, (int)M, (int)K, K, 0, ns, false, &cur);
  t.b = {W ? W : lad_ws_, nullptr, (int)b.rows, (int)Kp};
  t.C = C;
  t.M = (int)M;
  t.N = (int)b.rows;
  t.K = (int)K;
  t.ldc = (int)K;
  const double fl = 2.0 * M * (double)b.rows * K;
  tc_flops += (int64_t)fl;
  const int64_t sk = tc_sliced_scratch_doubles(&t, 1, ns);
  double* skb = sk > 0 ? scratch(sk) : nullptr;
  timed(K_TC, fl, [&] {
    return tc_gemm_sliced(&t, 1, alpha, 1.0, ns, skb, d_err, st_);
  });
}

// Y_G[(ij), (ab) in batch] += alpha * X_G[(ij),(cd)] W_batch^T
void Engine::ladder_apply_batch(const LadBatch& b, double alpha, Tensor* X,
                                Tensor* Y) {
  const Layout& XL = X->lay;
  const int G = b.G;
  const int64_t M = XL.nrow[G], K = XL.ncol[G];
  if (M == 0) return;
  const int gb = b.ga ^ G;
  GemmProb g;
  std::memset(&g, 0, sizeof(g));
  g.A = X->d + XL.blk_off[G];
  g.lda = (int)K;
  g.B = lad_w_;
  g.tb = 1;
  g.ldb = (int)K;
  g.C = Y->d + Y->lay.blk_off[G] + Y->lay.csub[G * Y->lay.ncode_c + b.ga] +
        (int64_t)b.a0 * dims_.n[SV][gb];
  g.ldc = (int)K;
  g.M = (int)M;
  g.N = (int)b.rows;
  g.K = (int)K;
  check_block(g, X->d, XL.size, lad_w_, lad_n_, Y->d, Y->lay.size);
  const Mat mx{X->d, &XL, false, X};
  const Mat mw{lad_w_, nullptr, false, nullptr};
  run_gemms(&g, 1, mx, mw, alpha, 1.0);
}

void Engine::ladder(double alpha, Tensor* T, Tensor* L, Tensor* R) {
  if (!is_doubles(T->lay) || !is_doubles(R->lay) || !is_lvv(L->lay))
    throw EngineError("ladder: layouts must be {SO,SO,SV,SV}/2 and "
                      "{SQ,SV,SV}/1");
  if (recording_)
    tape_.push_back({2, alpha, 1.0, T, L, R, "ijcd", "Pac", "ijab"});
  if (record_only_) return;
  ladder_lin_apply(0, alpha, T, L, false, R);
}

void Engine::ladder_stored(double alpha, Tensor* T, Tensor* W, Tensor* R) {
  if (!is_doubles(T->lay) || !is_doubles(R->lay))
    throw EngineError("ladder_stored: amplitude layouts must be "
                      "{SO,SO,SV,SV}/2");
  if (recording_)
    tape_.push_back({3, alpha, 1.0, T, W, R, "ijcd", "abcd", "ijab"});
  if (record_only_) return;
  ladder_lin_apply(0, alpha, T, W, true, R);
}

void Engine::ladder_lin(int which, int mode, int prec) {
  LadderLin& st = lin_[which];
  st.mode = mode;
  st.prec = prec;
  st.anchored = false;
}

// Y += alpha * Lad(X), linearised around the anchor of lin_[which] (see
// engine.h); with the mode off (or while a tape is recorded) the plain map.
void Engine::ladder_lin_apply(int which, double alpha, Tensor* X, Tensor* LW,
                              bool stored, Tensor* Y) {
  LadderLin& st = lin_[which];
  if (st.mode == 0 || recording_) {
    ladder_map(alpha, X, LW, stored, Y);
    return;
  }
  const std::string tag = which == 0 ? "ladlin_f_" : "ladlin_a_";
  std::vector<int> sp(X->lay.sp, X->lay.sp + X->lay.rank);
  st.in = tensor(tag + "in", sp, X->lay.split, X->lay.gtot);
  st.out = tensor(tag + "out", sp, X->lay.split, X->lay.gtot);
  if (st.mode == 1) {
    // new anchor: X0 = X, out = Lad_acc(X0)
    axpy_raw(1.0, X->lay, X->d, "ijab", 0.0, st.in->lay, st.in->d, "ijab");
    zero(st.out);
    ladder_map(1.0, X, LW, stored, st.out);
    st.mode = 2;
    st.anchored = true;
  } else {
    // Y += alpha * Lad_delta(X - X0)
    st.d = tensor(tag + "d", sp, X->lay.split, X->lay.gtot);
    axpy_raw(1.0, X->lay, X->d, "ijab", 0.0, st.d->lay, st.d->d, "ijab");
    axpy_raw(-1.0, st.in->lay, st.in->d, "ijab", 1.0, st.d->lay, st.d->d,
             "ijab");
    ++st.d->ver;
    const int keep = tc_override_;
    tc_override_ = st.prec;
    try {
      ladder_map(alpha, st.d, LW, stored, Y);
    } catch (...) {
      tc_override_ = keep;
      throw;
    }
    tc_override_ = keep;
    st.anchored = false;
  }
  axpy_raw(alpha, st.out->lay, st.out->d, "ijab", 1.0, Y->lay, Y->d, "ijab");
  ++Y->ver;
}

void Engine::ladder_keep_slices(int64_t bytes) {
  lad_cache_cap_ = std::max<int64_t>(0, bytes);
  if (bytes > 0) return;
  if (lad_cache_.empty()) return;
  for (auto& kv : lad_cache_) al.release(kv.second.data, kv.second.bytes);
  lad_cache_.clear();
  lad_cache_bytes_ = 0;
}

void Engine::ladder_map(double alpha, Tensor* X, Tensor* LW, bool stored,
                        Tensor* Y) {
  if (stored) {
    contract(alpha, X, "ijcd", LW, "abcd", 1.0, Y, "ijab");
    return;
  }
  if (ladder_pm_) {
    ladder_map_pm(alpha, X, LW, Y);
    return;
  }
  Tensor* T = X;
  Tensor* L = LW;
  Tensor* R = Y;
  ++R->ver;
  SigScope sig(this, "ladder on the fly");
  cudaEvent_t tr_a = nullptr;
  if (prof_on_) {
    tr_a = get_event();
    cudaEventRecord(tr_a, st_);
  }
  const std::vector<LadBatch> bs = ladder_batches(T->lay);
  int64_t need = 0;
  for (const LadBatch& b : bs)
    need = std::max(need, b.rows * T->lay.ncol[b.G]);
  ladder_reserve(need);
  double fl = 0;
  const int ns = active_precision();
  for (const LadBatch& b : bs) {
    if (ladder_fusable(b, T->lay, L->lay)) {
      // profiling: build and apply traced apart (keys outside "ladder*")
      // (every trace record owns its two events: prof_collect returns
      // both to the pool)
      cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr, e3 = nullptr;
      if (prof_on_) {
        e0 = get_event();
        cudaEventRecord(e0, st_);
      }
      // slices kept from an earlier application (same L version), or built
      // now: into a kept buffer while the budget lasts, else the batch
      // buffer
      const void* W = nullptr;
      double fb = 0;
      if (lad_cache_cap_ > 0) {
        std::ostringstream key;
        key << b.G << ',' << b.ga << ',' << b.a0 << ',' << b.a1 << ',' << ns;
        auto it = lad_cache_.find(key.str());
        if (it != lad_cache_.end() && it->second.L == L &&
            it->second.lver == L->ver) {
          W = it->second.data;
        } else {
          int64_t ncol = 0;
          for (int gc = 0; gc < dims_.h; ++gc)
            ncol += (int64_t)dims_.n[SV][gc] * dims_.n[SV][gc ^ b.G];
          const size_t bytes =
              (size_t)ns * b.rows * slice_kp((int)ncol) * 2;
          void* dst = nullptr;
          if (it != lad_cache_.end() && it->second.bytes == bytes) {
            dst = it->second.data;   // stale (new L): rebuilt in place
          } else if (it == lad_cache_.end() &&
                     lad_cache_bytes_ + (int64_t)bytes <= lad_cache_cap_ &&
                     device_free_above(bytes, (size_t)8 << 30)) {
            // (kept or rebuilt slices hold the same values, so the choice
            // may depend on the free memory of the moment)
            dst = al.alloc(bytes);
            lad_cache_[key.str()] = {dst, bytes, 0, L};
            lad_cache_bytes_ += (int64_t)bytes;
            it = lad_cache_.find(key.str());
          }
          fb = ladder_build_sliced(b, L, ns, dst);
          if (dst) {
            it->second.lver = L->ver;
            it->second.L = L;
            W = dst;
          }
        }
      } else {
        fb = ladder_build_sliced(b, L, ns);
      }
      if (prof_on_) {
        e1 = get_event();
        e2 = get_event();
        cudaEventRecord(e1, st_);
        cudaEventRecord(e2, st_);
      }
      ladder_apply_sliced(b, alpha, T, R, ns, W);
      if (prof_on_) {
        e3 = get_event();
        cudaEventRecord(e3, st_);
        const double fa =
            2.0 * (double)b.rows * T->lay.ncol[b.G] * T->lay.nrow[b.G];
        trace_pending_.push_back({"part: fused ladder build [split]", e0, e1,
                                  fb});
        trace_pending_.push_back({"part: ladder apply [split]", e2, e3, fa});
      }
      fl += fb;
    } else {
      fl += ladder_build(b, L);
      ladder_apply_batch(b, alpha, T, R);
    }
    fl += 2.0 * (double)b.rows * T->lay.ncol[b.G] * T->lay.nrow[b.G];
    release_scratch();   // stream order: the next batch may reuse it
  }
  if (tr_a) {
    cudaEvent_t tr_b = get_event();
    cudaEventRecord(tr_b, st_);
    const int pr = active_precision();
    trace_pending_.push_back(
        {std::string("ladder on the fly (ijcd,Pac,Pbd->ijab) [") +
             (pr >= 12 ? "exact" : pr > 0 ? "split" : "fp64") + "]",
         tr_a, tr_b, fl});
  }
  release_scratch();
}

void Engine::ladder_adjoint(double alpha, Tensor* dR, Tensor* T, Tensor* L,
                            Tensor* dT, Tensor* dL) {
  if (!dT && !dL) return;
  SigScope sig(this, "ladder on the fly, adjoint");
  cudaEvent_t tr_a = nullptr;
  if (prof_on_) {
    tr_a = get_event();
    cudaEventRecord(tr_a, st_);
  }
  double fl = 0;
  const std::vector<LadBatch> bs = ladder_batches(T->lay);
  int64_t need = 0;
  for (const LadBatch& b : bs)
    need = std::max(need, b.rows * T->lay.ncol[b.G]);
  ladder_reserve(need);
  const int h = dims_.h;
  const Layout& LL = L->lay;
  // dL alone (the density sweep): with pair-symmetric dR and T, dW is
  // invariant under the joint swap (ab,cd) -> (ba,dc) and both give the same
  // dL terms, so only the batches with ga >= gb run, those with ga > gb at
  // twice the weight (the +/- ladder's symmetry assumption)
  const bool half = ladder_pm_ && !dT;
  for (const LadBatch& b : bs) {
    const int gbb = b.ga ^ b.G;
    if (half && b.ga < gbb) continue;
    const double wgt = half && b.ga > gbb ? 2.0 : 1.0;
    release_scratch();   // stream order: the previous batch is queued
    const double fapply =
        2.0 * (double)b.rows * T->lay.ncol[b.G] * T->lay.nrow[b.G];
    if (dT) {
      // the (ab|cd) rows are needed for dT only
      fl += ladder_build(b, L);
      ladder_apply_batch(b, alpha, dR, dT);
      fl += fapply;
    }
    if (!dL) continue;
    fl += 2.0 * fapply;   // dW and the two dL products (nominal)
    const int G = b.G, ga = b.ga, gb = ga ^ G;
    const int na = b.a1 - b.a0, nb = dims_.n[SV][gb];
    const Layout& RL = dR->lay;
    const int64_t K = RL.nrow[G], ncol = RL.ncol[G];
    if (K == 0) continue;
    // dW_batch = alpha * dR_G[:, batch]^T T_G  -> lad_w_
    {
      GemmProb g;
      std::memset(&g, 0, sizeof(g));
      g.A = dR->d + RL.blk_off[G] + RL.csub[G * RL.ncode_c + ga] +
            (int64_t)b.a0 * nb;
      g.ta = 1;
      g.lda = (int)ncol;
      g.B = T->d + T->lay.blk_off[G];
      g.ldb = (int)ncol;
      g.C = lad_w_;
      g.ldc = (int)ncol;
      g.M = (int)b.rows;
      g.N = (int)ncol;
      g.K = (int)K;
      check_block(g, dR->d, RL.size, T->d, T->lay.size, lad_w_, lad_n_);
      const Mat ma{dR->d, &RL, false, dR};
      const Mat mb{T->d, &T->lay, false, T};
      run_gemms(&g, 1, ma, mb, alpha * wgt, 0.0);
    }
    ladder_perm(b, true, lad_w_, lad_x_);        // dX_gc[(a,c),(b,d)]
    GemmProb p1[GEMM_MAXPROB], p2[GEMM_MAXPROB];
    int n1 = 0, n2 = 0;
    int64_t xoff = 0;
    for (int gc = 0; gc < h; ++gc) {
      const int gd = gc ^ G, Gp = ga ^ gc;
      const int nc = dims_.n[SV][gc], nd = dims_.n[SV][gd];
      const int64_t MA = (int64_t)na * nc, NB = (int64_t)nb * nd;
      const int64_t P = LL.nrow[Gp], ld = LL.ncol[Gp];
      if (MA * NB == 0) continue;
      if (P == 0) {
        xoff += MA * NB;
        continue;
      }
      double* LA = L->d + LL.blk_off[Gp] + LL.csub[Gp * LL.ncode_c + ga] +
                   (int64_t)b.a0 * nc;
      double* LB = L->d + LL.blk_off[Gp] + LL.csub[Gp * LL.ncode_c + gb];
      const int64_t oA = LA - L->d, oB = LB - L->d;
      // dL_A[P,(ac)] += L_B[P,(bd)] dX[(ac),(bd)]^T
      GemmProb g1;
      std::memset(&g1, 0, sizeof(g1));
      g1.A = LB;
      g1.lda = (int)ld;
      g1.B = lad_x_ + xoff;
      g1.tb = 1;
      g1.ldb = (int)NB;
      g1.C = dL->d + oA;
      g1.ldc = (int)ld;
      g1.M = (int)P;
      g1.N = (int)MA;
      g1.K = (int)NB;
      check_block(g1, L->d, LL.size, lad_x_, lad_n_, dL->d, dL->lay.size);
      p1[n1++] = g1;
      // dL_B[P,(bd)] += L_A[P,(ac)] dX[(ac),(bd)]
      GemmProb g2;
      std::memset(&g2, 0, sizeof(g2));
      g2.A = LA;
      g2.lda = (int)ld;
      g2.B = lad_x_ + xoff;
      g2.tb = 0;
      g2.ldb = (int)NB;
      g2.C = dL->d + oB;
      g2.ldc = (int)ld;
      g2.M = (int)P;
      g2.N = (int)NB;
      g2.K = (int)MA;
      check_block(g2, L->d, LL.size, lad_x_, lad_n_, dL->d, dL->lay.size);
      p2[n2++] = g2;
      xoff += MA * NB;
    }
    const Mat ml{L->d, &LL, false, L};
    const Mat mx{lad_x_, nullptr, false, nullptr};
    if (n1) run_gemms(p1, n1, ml, mx, 1.0, 1.0);
    if (n2) run_gemms(p2, n2, ml, mx, 1.0, 1.0);
  }
  if (dT) ++dT->ver;
  if (dL) ++dL->ver;
  if (tr_a) {
    cudaEvent_t tr_b = get_event();
    cudaEventRecord(tr_b, st_);
    trace_pending_.push_back({"ladder on the fly, adjoint", tr_a, tr_b, fl});
  }
  release_scratch();
}


// ---------------------------------------------------------------------------
// +/- packed on-the-fly ladder (Sec. 2.3; arithmetic in ladder_pm.cu).
// Canonical pairs (p,q) of an index pair: irrep(p) > irrep(q), or the same
// irrep and p >= q.  For the pair irrep G the canonical (a,b) rows are the
// row batches with ga > gb (all rows) and, for G = 0 (ga == gb), the rows
// with b <= a of each batch; batches with ga < gb are not built at all.
// Per batch: the (ab|cd) rows W as in the plain map, then
//   W+- = W[.,(cd)] +- W[.,(dc)]   (pm_pack_w)
//   S+- = A+- W+-^T                 (two GEMMs: canonical ij x ab x cd)
//   Y  += the signed combinations of S+ and S- (pm_unpack)
// with A+- packed once per pair irrep from X (pm_pack_x).  With float
// slices the BF16 slices of W+- are kept across applications (they depend
// on L only), within the budget of ladder_keep_slices.

void pm_host_tables(const Layout& TL, const Dims& dims_,
                    int64_t batch_bytes, PmPlan& P, std::vector<int>& tab) {
  P = PmPlan();
  tab.clear();
  const int h = dims_.h;
  auto off32 = [](int64_t v) {
    if (v < 0 || v > INT32_MAX)
      throw EngineError("ladder +/-: block offset beyond 32 bits");
    return (int)v;
  };
  for (int G = 0; G < h; ++G) {
    if (TL.nrow[G] == 0 || TL.ncol[G] == 0) continue;
    // canonical occupied pairs: rows (i,j) and (j,i)
    std::vector<int> r1, r2;
    for (int gi = 0; gi < h; ++gi) {
      const int gj = gi ^ G;
      if (gi < gj) continue;
      const int ni = dims_.n[SO][gi], nj = dims_.n[SO][gj];
      const int64_t o1 = TL.rsub[G * TL.ncode_r + gi];
      const int64_t o2 = TL.rsub[G * TL.ncode_r + gj];
      for (int i = 0; i < ni; ++i)
        for (int j = 0; j < (gi == gj ? i + 1 : nj); ++j) {
          r1.push_back(off32(o1 + (int64_t)i * nj + j));
          r2.push_back(off32(o2 + (int64_t)j * ni + i));
        }
    }
    // canonical virtual pairs: columns (c,d) and (d,c)
    std::vector<int> c1, c2;
    for (int gc = 0; gc < h; ++gc) {
      const int gd = gc ^ G;
      if (gc < gd) continue;
      const int nc = dims_.n[SV][gc], nd = dims_.n[SV][gd];
      const int64_t o1 = TL.csub[G * TL.ncode_c + gc];
      const int64_t o2 = TL.csub[G * TL.ncode_c + gd];
      for (int c = 0; c < nc; ++c)
        for (int d = 0; d < (gc == gd ? c + 1 : nd); ++d) {
          c1.push_back(off32(o1 + (int64_t)c * nd + d));
          c2.push_back(off32(o2 + (int64_t)d * nc + c));
        }
    }
    P.uo[G] = (int)r1.size();
    P.uv[G] = (int)c1.size();
    P.orow[G] = (int64_t)tab.size();
    tab.insert(tab.end(), r1.begin(), r1.end());
    tab.insert(tab.end(), r2.begin(), r2.end());
    P.vcol[G] = (int64_t)tab.size();
    tab.insert(tab.end(), c1.begin(), c1.end());
    tab.insert(tab.end(), c2.begin(), c2.end());
    P.max_a = std::max<int64_t>(P.max_a,
                                2 * (int64_t)r1.size() * (int64_t)c1.size());
  }
  for (const LadBatch& b : ladder_batch_list(TL, dims_, batch_bytes)) {
    const int G = b.G, ga = b.ga, gb = ga ^ G;
    if (ga < gb || P.uo[G] == 0 || P.uv[G] == 0) continue;
    const int na = dims_.n[SV][ga], nb = dims_.n[SV][gb];
    const int64_t oab = TL.csub[G * TL.ncode_c + ga];
    const int64_t oba = TL.csub[G * TL.ncode_c + gb];
    std::vector<int> lr, y1, y2;
    for (int a = b.a0; a < b.a1; ++a)
      for (int bb = 0; bb < (ga == gb ? a + 1 : nb); ++bb) {
        lr.push_back(off32((int64_t)(a - b.a0) * nb + bb));
        y1.push_back(off32(oab + (int64_t)a * nb + bb));
        y2.push_back(ga == gb && a == bb
                         ? -1
                         : off32(oba + (int64_t)bb * na + a));
      }
    if (lr.empty()) continue;
    PmBatch pb;
    pb.b = b;
    pb.nv = (int)lr.size();
    pb.vrow = (int64_t)tab.size();
    tab.insert(tab.end(), lr.begin(), lr.end());
    tab.insert(tab.end(), y1.begin(), y1.end());
    tab.insert(tab.end(), y2.begin(), y2.end());
    P.batches.push_back(pb);
    P.max_w = std::max<int64_t>(P.max_w, 2 * (int64_t)pb.nv * P.uv[G]);
  }
}

const PmPlan& Engine::pm_plan(const Layout& TL) {
  std::ostringstream ks;
  ks << TL.key() << '/' << ladder_batch_bytes;
  if (pm_.d_tab && pm_.key == ks.str()) return pm_;
  if (pm_.d_tab) al.release(pm_.d_tab, pm_.bytes);
  pm_ = PmPlan();
  std::vector<int> tab;
  pm_host_tables(TL, dims_, ladder_batch_bytes, pm_, tab);
  if (!tab.empty()) {
    pm_.bytes = tab.size() * sizeof(int);
    pm_.d_tab = (int*)al.alloc(pm_.bytes);
    // pageable source: the copy is complete (staged) when the call returns
    LCK(cudaMemcpyAsync(pm_.d_tab, tab.data(), pm_.bytes,
                        cudaMemcpyHostToDevice, st_));
  }
  pm_.key = ks.str();
  return pm_;
}

void Engine::ladder_map_pm(double alpha, Tensor* T, Tensor* L, Tensor* R) {
  ++R->ver;
  SigScope sig(this, "ladder on the fly");
  cudaEvent_t tr_a = nullptr;
  if (prof_on_) {
    tr_a = get_event();
    cudaEventRecord(tr_a, st_);
  }
  const PmPlan& P = pm_plan(T->lay);
  int64_t need = 0;
  for (const PmBatch& pb : P.batches)
    need = std::max(need, pb.b.rows * T->lay.ncol[pb.b.G]);
  ladder_reserve(need);
  if (P.max_a > pm_a_n_) {
    if (pm_a_) al.release(pm_a_, (size_t)pm_a_n_ * 8);
    pm_a_ = nullptr;
    pm_a_n_ = 0;
    pm_a_ = (double*)al.alloc((size_t)P.max_a * 8);
    pm_a_n_ = P.max_a;
  }
  if (P.max_w > pm_w_n_) {
    if (pm_w_) al.release(pm_w_, (size_t)pm_w_n_ * 8);
    pm_w_ = nullptr;
    pm_w_n_ = 0;
    pm_w_ = (double*)al.alloc((size_t)P.max_w * 8);
    pm_w_n_ = P.max_w;
  }
  const int prec = active_precision();
  const bool split = prec >= 1 && prec <= 3 && d_err != nullptr;
  const int ns = prec;
  double fl = 0;
  int curG = -1;
  bool a_sliced = false;
  for (const PmBatch& pb : P.batches) {
    const LadBatch& b = pb.b;
    const int G = b.G;
    const int uo = P.uo[G], uv = P.uv[G], nv = pb.nv;
    const int64_t ncol = T->lay.ncol[G];
    if (ncol != R->lay.ncol[G] || T->lay.nrow[G] != R->lay.nrow[G])
      throw EngineError("internal: ladder +/- layouts differ");
    const int* orow = P.d_tab + P.orow[G];
    const int* vcol = P.d_tab + P.vcol[G];
    const int* vrow = P.d_tab + pb.vrow;
    double* Ap = pm_a_;
    double* Am = pm_a_ + (int64_t)uo * uv;
    if (G != curG) {
      curG = G;
      a_sliced = false;
      const double* X = T->d + T->lay.blk_off[G];
      timed(K_PERM, 48.0 * uo * (double)uv, [&] {
        return pm_pack_x(X, ncol, orow, uo, vcol, uv, Ap, Am, st_);
      });
    }
    const int64_t Kp = slice_kp(uv);
    // kept BF16 slices of W+ | W- (float slices), or a buffer for them
    const bool tcs = split && tc_shape(uo, nv, uv);
    const void* Ws = nullptr;
    void* dst = nullptr;
    if (tcs && lad_cache_cap_ > 0) {
      std::ostringstream key;
      key << "pm," << G << ',' << b.ga << ',' << b.a0 << ',' << b.a1 << ','
          << ns;
      const size_t bytes = (size_t)2 * ns * nv * Kp * 2;
      auto it = lad_cache_.find(key.str());
      if (it != lad_cache_.end() && it->second.L == L &&
          it->second.lver == L->ver && it->second.bytes == bytes) {
        Ws = it->second.data;
      } else if (it != lad_cache_.end() && it->second.bytes == bytes) {
        dst = it->second.data;   // stale (new L): rebuilt in place
        it->second.lver = L->ver;
        it->second.L = L;
      } else if (it == lad_cache_.end() &&
                 lad_cache_bytes_ + (int64_t)bytes <= lad_cache_cap_ &&
                 device_free_above(bytes, (size_t)8 << 30)) {
        dst = al.alloc(bytes);
        lad_cache_[key.str()] = {dst, bytes, L->ver, L};
        lad_cache_bytes_ += (int64_t)bytes;
      }
    }
    double* Wp = pm_w_;
    double* Wm = pm_w_ + (int64_t)nv * uv;
    if (!Ws) {
      fl += ladder_build(b, L);   // (ab|cd) rows of the batch -> lad_w_
      timed(K_PERM, 32.0 * nv * (double)uv, [&] {
        return pm_pack_w(lad_w_, ncol, vrow, nv, vcol, uv, Wp, Wm, st_);
      });
      if (dst) {
        uint8_t* d8 = (uint8_t*)dst;
        timed(K_OTHER, 32.0 * nv * (double)uv, [&] {
          return split_float(Wp, nv, uv, uv, 0, ns, d8, st_) +
                 split_float(Wm, nv, uv, uv, 0, ns,
                             d8 + (size_t)ns * nv * Kp * 2, st_);
        });
        Ws = dst;
      }
    }
    double* S = scratch(2 * (int64_t)uo * nv);
    double* Sp = S;
    double* Sm = S + (int64_t)uo * nv;
    const double fa = 4.0 * uo * (double)nv * uv;
    if (Ws) {
      // both products on pre-sliced operands, one grouped launch
      const size_t abytes = (size_t)2 * ns * uo * Kp * 2;
      if (!a_sliced) {
        if (abytes > pm_as_bytes_) {
          if (pm_as_) al.release(pm_as_, pm_as_bytes_);
          pm_as_ = nullptr;
          pm_as_bytes_ = 0;
          pm_as_ = al.alloc(abytes);
          pm_as_bytes_ = abytes;
        }
        uint8_t* a8 = (uint8_t*)pm_as_;
        timed(K_OTHER, 32.0 * uo * (double)uv, [&] {
          return split_float(Ap, uo, uv, uv, 0, ns, a8, st_) +
                 split_float(Am, uo, uv, uv, 0, ns,
                             a8 + (size_t)ns * uo * Kp * 2, st_);
        });
        a_sliced = true;
      }
      TcProb t[2];
      std::memset(t, 0, sizeof(t));
      for (int q = 0; q < 2; ++q) {
        t[q].a = {(const uint8_t*)pm_as_ + (size_t)q * ns * uo * Kp * 2,
                  nullptr, uo, (int)Kp};
        t[q].b = {(const uint8_t*)Ws + (size_t)q * ns * nv * Kp * 2, nullptr,
                  nv, (int)Kp};
        t[q].C = q == 0 ? Sp : Sm;
        t[q].M = uo;
        t[q].N = nv;
        t[q].K = uv;
        t[q].ldc = nv;
      }
      tc_flops += (int64_t)fa;
      const int64_t sk = tc_sliced_scratch_doubles(t, 2, ns);
      double* skb = sk > 0 ? scratch(sk) : nullptr;
      timed(K_TC, fa, [&] {
        return tc_gemm_sliced(t, 2, 1.0, 0.0, ns, skb, d_err, st_);
      });
    } else {
      GemmProb g[2];
      std::memset(g, 0, sizeof(g));
      for (int q = 0; q < 2; ++q) {
        g[q].A = q == 0 ? Ap : Am;
        g[q].lda = uv;
        g[q].B = q == 0 ? Wp : Wm;
        g[q].tb = 1;
        g[q].ldb = uv;
        g[q].C = q == 0 ? Sp : Sm;
        g[q].ldc = nv;
        g[q].M = uo;
        g[q].N = nv;
        g[q].K = uv;
      }
      const Mat ma{pm_a_, nullptr, false, nullptr};
      const Mat mw{pm_w_, nullptr, false, nullptr};
      run_gemms(g, 2, ma, mw, 1.0, 0.0);
    }
    fl += fa;
    double* Y = R->d + R->lay.blk_off[G];
    timed(K_PERM, 80.0 * uo * (double)nv, [&] {
      return pm_unpack(Sp, Sm, uo, nv, orow, vrow, alpha, Y, ncol, st_);
    });
    release_scratch();   // stream order: the next batch may reuse it
  }
  if (tr_a) {
    cudaEvent_t tr_b = get_event();
    cudaEventRecord(tr_b, st_);
    trace_pending_.push_back(
        {std::string("ladder on the fly (ijcd,Pac,Pbd->ijab) [") +
             (prec >= 12 ? "exact" : prec > 0 ? "split" : "fp64") + ", +/-]",
         tr_a, tr_b, fl});
  }
  release_scratch();
}

}  // namespace cdcc
