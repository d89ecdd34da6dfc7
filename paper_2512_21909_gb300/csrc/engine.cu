// engine.cu -- contraction planner, permutation tasks and reverse-mode tape.
#include "engine.h"

#include <algorithm>
#include <cstring>
#include <cstdio>
#include <sstream>

namespace cdcc {

#define ECK(x)                                                            \
  do {                                                                    \
    cudaError_t e_ = (x);                                                 \
    if (e_ != cudaSuccess)                                                \
      throw EngineError(std::string("CUDA: ") + cudaGetErrorString(e_) + \
                        " at " #x);                                       \
  } while (0)

void* DevAlloc::alloc(size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (fa) {
    p = fa(bytes, (void*)st, user);
    if (!p) throw EngineError("device allocation callback failed");
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      throw EngineError(std::string("cudaMallocAsync: ") +
                        cudaGetErrorString(e));
    }
  }
  return p;
}

void DevAlloc::release(void* p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 256;
  if (ff)
    ff(p, bytes, (void*)st, user);
  else
    cudaFreeAsync(p, st);
}

bool device_free_above(size_t need, size_t reserve) {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return fr > need + reserve;
}

Engine::Engine(const Dims& d, cudaStream_t st, DevAlloc a)
    : al(a), dims_(d), st_(st) {
  al.st = st;
}

Engine::~Engine() {
  for (auto& kv : tensors_) {
    Tensor* t = kv.second.get();
    if (t->owns && t->d) al.release(t->d, (size_t)t->lay.size * 8);
  }
  for (auto& kv : task_cache_) {
    al.release(kv.second.tasks, kv.second.ntask * sizeof(PermTask));
    al.release(kv.second.chunks, kv.second.nchunk * sizeof(Chunk));
  }
  for (auto& b : pool_) al.release(b.d, (size_t)b.n * 8);
  if (lad_x_) al.release(lad_x_, (size_t)lad_n_ * 8);
  if (lad_w_) al.release(lad_w_, (size_t)lad_n_ * 8);
  if (lad_ws_) al.release(lad_ws_, lad_ws_bytes_);
  if (pm_.d_tab) al.release(pm_.d_tab, pm_.bytes);
  if (pm_a_) al.release(pm_a_, (size_t)pm_a_n_ * 8);
  if (pm_w_) al.release(pm_w_, (size_t)pm_w_n_ * 8);
  if (pm_as_) al.release(pm_as_, pm_as_bytes_);
  for (auto& kv : lad_cache_) al.release(kv.second.data, kv.second.bytes);
  for (auto& kv : slice_cache_) {
    al.release(kv.second.data, kv.second.bytes);
    if (kv.second.exps) al.release(kv.second.exps, kv.second.ebytes);
  }
  cudaStreamSynchronize(st_);
  for (auto& r : pending_) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ev_pool_) cudaEventDestroy(e);
}

Layout Engine::make_layout(const std::vector<int>& spaces, int split,
                           int gtot) {
  Layout L;
  L.rank = (int)spaces.size();
  if (L.rank > MAXRANK) throw EngineError("rank > 4");
  for (int q = 0; q < L.rank; ++q) L.sp[q] = spaces[q];
  L.split = split;
  L.gtot = gtot;
  L.build(dims_);
  return L;
}

Tensor* Engine::new_tensor(const std::string& name, std::vector<int> spaces,
                           int split, int gtot) {
  auto t = std::make_unique<Tensor>();
  t->name = name;
  t->lay = make_layout(spaces, split, gtot);
  t->d = (double*)al.alloc((size_t)std::max<int64_t>(t->lay.size, 1) * 8);
  ECK(cudaMemsetAsync(t->d, 0, (size_t)std::max<int64_t>(t->lay.size, 1) * 8,
                      st_));
  Tensor* r = t.get();
  tensors_[name] = std::move(t);
  return r;
}

Tensor* Engine::tensor(const std::string& name, std::vector<int> spaces,
                       int split, int gtot) {
  auto it = tensors_.find(name);
  if (it != tensors_.end()) {
    Layout L = make_layout(spaces, split, gtot);
    if (!L.same(it->second->lay))
      throw EngineError("tensor '" + name + "' re-declared with new layout");
    return it->second.get();
  }
  return new_tensor(name, spaces, split, gtot);
}

Tensor* Engine::flat(const std::string& name, int64_t n) {
  auto it = tensors_.find(name);
  if (it != tensors_.end()) {
    if (it->second->lay.size != n)
      throw EngineError("flat '" + name + "' re-declared with new size");
    return it->second.get();
  }
  auto t = std::make_unique<Tensor>();
  t->name = name;
  t->lay.rank = -1;
  t->lay.size = n;
  t->d = (double*)al.alloc((size_t)std::max<int64_t>(n, 1) * 8);
  ECK(cudaMemsetAsync(t->d, 0, (size_t)std::max<int64_t>(n, 1) * 8, st_));
  Tensor* r = t.get();
  tensors_[name] = std::move(t);
  return r;
}

Tensor* Engine::view(const std::string& name, Tensor* parent, int64_t offset,
                     std::vector<int> spaces, int split, int gtot) {
  auto it = tensors_.find(name);
  if (it != tensors_.end()) return it->second.get();
  auto t = std::make_unique<Tensor>();
  t->name = name;
  t->lay = make_layout(spaces, split, gtot);
  if (offset + t->lay.size > parent->lay.size)
    throw EngineError("view '" + name + "' exceeds its parent");
  t->d = parent->d + offset;
  t->owns = false;
  t->parent = parent;
  t->offset = offset;
  Tensor* r = t.get();
  tensors_[name] = std::move(t);
  return r;
}

Tensor* Engine::find(const std::string& name) {
  auto it = tensors_.find(name);
  return it == tensors_.end() ? nullptr : it->second.get();
}

Tensor* Engine::adjoint(Tensor* t) {
  if (t->adj) return t->adj;
  if (t->parent) {
    Tensor* pa = adjoint(t->parent);
    std::vector<int> sp(t->lay.sp, t->lay.sp + t->lay.rank);
    t->adj = view(t->name + "~", pa, t->offset, sp, t->lay.split,
                  t->lay.gtot);
  } else if (t->lay.rank < 0) {
    t->adj = flat(t->name + "~", t->lay.size);
  } else {
    std::vector<int> sp(t->lay.sp, t->lay.sp + t->lay.rank);
    t->adj = tensor(t->name + "~", sp, t->lay.split, t->lay.gtot);
  }
  t->adj->ladder = t->ladder;
  return t->adj;
}

cudaEvent_t Engine::get_event() {
  if (!ev_pool_.empty()) {
    cudaEvent_t e = ev_pool_.back();
    ev_pool_.pop_back();
    return e;
  }
  cudaEvent_t e;
  ECK(cudaEventCreate(&e));
  return e;
}

// Copy of constant tensor T (index string tl) in the matrix layout rows r,
// columns c; null when the cache budget does not allow it.  With create =
// false only reports whether the copy exists or would be made.
Tensor* Engine::permuted_constant(Tensor* T, const std::string& tl,
                                  const std::string& r, const std::string& c,
                                  bool create) {
  const std::string rc = r + c;
  if ((int)rc.size() != T->lay.rank || (int)tl.size() != T->lay.rank)
    return nullptr;
  // the permutation as positions of the target letters in tl (letters are
  // labels: "mcnd" -> "cdmn" and "kcld" -> "cdkl" are the same copy)
  std::string key = T->name + '|';
  std::vector<int> sp;
  for (char x : rc) {
    const size_t p = tl.find(x);
    if (p == std::string::npos) return nullptr;
    key += (char)('0' + (int)p);
    sp.push_back(T->lay.sp[p]);
  }
  key += ':' + std::to_string(r.size());
  auto it = perm_const_.find(key);
  if (it != perm_const_.end()) {
    if (create && it->second.src_ver != T->ver) {
      Tensor* P = it->second.t;
      axpy_raw(1.0, T->lay, T->d, tl, 0.0, P->lay, P->d, rc);
      ++P->ver;
      it->second.src_ver = T->ver;
    }
    return it->second.t;
  }
  const Layout L = make_layout(sp, (int)r.size(), T->lay.gtot);
  const int64_t bytes = std::max<int64_t>(L.size, 1) * 8;
  if (perm_const_cap_ <= 0 || perm_const_bytes_ + bytes > perm_const_cap_)
    return nullptr;
  if (!create) return T;   // would be made: any non-null answer
  // a kept copy holds the same values as a per-call permutation, so it may
  // depend on the free memory of the moment (8 GB stay free for the rest)
  if (!device_free_above((size_t)bytes, (size_t)8 << 30)) return nullptr;
  Tensor* P = new_tensor("perm:" + key, sp, (int)r.size(), T->lay.gtot);
  P->constant = true;
  // slices of a copy of a frozen or changing tensor count against the
  // bounded budget (and the free-memory guard)
  P->frozen = T->frozen || !T->constant;
  P->ladder = T->ladder;
  axpy_raw(1.0, T->lay, T->d, tl, 0.0, P->lay, P->d, rc);
  P->ver = 1;
  perm_const_[key] = {P, T->ver, T};
  perm_const_bytes_ += bytes;
  return P;
}

// The kept copy of T in layout (r, c) exists and is of T's current version.
bool Engine::permuted_current(Tensor* T, const std::string& tl,
                              const std::string& r, const std::string& c) {
  const std::string rc = r + c;
  if ((int)rc.size() != T->lay.rank || (int)tl.size() != T->lay.rank)
    return false;
  std::string key = T->name + '|';
  for (char x : rc) {
    const size_t p = tl.find(x);
    if (p == std::string::npos) return false;
    key += (char)('0' + (int)p);
  }
  key += ':' + std::to_string(r.size());
  auto it = perm_const_.find(key);
  return it != perm_const_.end() && it->second.src_ver == T->ver;
}

int Engine::sig_of(const std::string& s) {
  auto it = sig_id_.find(s);
  if (it != sig_id_.end()) return it->second;
  const int id = (int)sig_name_.size();
  sig_id_.emplace(s, id);
  sig_name_.push_back(s);
  sig_sec_.push_back({});
  return id;
}

void Engine::prof_collect() {
  if (pending_.empty() && trace_pending_.empty()) return;
  ECK(cudaStreamSynchronize(st_));
  for (auto& r : pending_) {
    float ms = 0;
    ECK(cudaEventElapsedTime(&ms, r.a, r.b));
    prof_sec[r.kind] += ms * 1e-3;
    if (r.sig >= 0 && r.sig < (int)sig_sec_.size() && r.kind < 8)
      sig_sec_[r.sig][r.kind] += ms * 1e-3;
    prof_work[r.kind] += r.work;
    prof_n[r.kind] += r.n;
    ev_pool_.push_back(r.a);
    ev_pool_.push_back(r.b);
  }
  pending_.clear();
  for (auto& r : trace_pending_) {
    float ms = 0;
    ECK(cudaEventElapsedTime(&ms, r.a, r.b));
    TraceAgg& a = trace_[r.key];
    a.sec += ms * 1e-3;
    a.flops += r.flops;
    a.calls += 1;
    ev_pool_.push_back(r.a);
    ev_pool_.push_back(r.b);
  }
  trace_pending_.clear();
}

void Engine::zero(Tensor* t) {
  ++t->ver;
  if (t->lay.size > 0)
    ECK(cudaMemsetAsync(t->d, 0, (size_t)t->lay.size * 8, st_));
}

void Engine::set_precision(int slices) {
  if (slices == tc_slices_) return;
  tc_slices_ = slices;
  for (auto& kv : slice_cache_) {
    al.release(kv.second.data, kv.second.bytes);
    if (kv.second.exps) al.release(kv.second.exps, kv.second.ebytes);
  }
  slice_cache_.clear();
  frozen_slice_bytes_ = 0;
}

void Engine::freeze_tape_operands() {
  for (const Op& op : tape_) {
    for (Tensor* T : {op.A, op.B}) {
      if (!T || T->constant || T->frozen) continue;
      T->constant = true;
      T->frozen = true;
      frozen_.push_back(T);
    }
  }
}

void Engine::thaw() {
  if (frozen_.empty()) return;
  // drop the permuted copies of frozen tensors (and their slices)
  std::set<const Tensor*> gone(frozen_.begin(), frozen_.end());
  std::set<const Tensor*> copies;
  for (auto it = perm_const_.begin(); it != perm_const_.end();) {
    if (!gone.count(it->second.src)) {
      ++it;
      continue;
    }
    Tensor* P = it->second.t;
    copies.insert(P);
    perm_const_bytes_ -= std::max<int64_t>(P->lay.size, 1) * 8;
    it = perm_const_.erase(it);
  }
  gone.insert(copies.begin(), copies.end());
  ECK(cudaStreamSynchronize(st_));   // nothing in flight reads them
  for (auto it = slice_cache_.begin(); it != slice_cache_.end();) {
    if (!gone.count(it->second.owner)) {
      ++it;
      continue;
    }
    al.release(it->second.data, it->second.bytes);
    if (it->second.exps) al.release(it->second.exps, it->second.ebytes);
    it = slice_cache_.erase(it);
  }
  frozen_slice_bytes_ = 0;
  for (auto it = tensors_.begin(); it != tensors_.end();) {
    Tensor* t = it->second.get();
    if (copies.count(t)) {
      if (t->owns && t->d) al.release(t->d, (size_t)t->lay.size * 8);
      it = tensors_.erase(it);
    } else {
      ++it;
    }
  }
  for (Tensor* T : frozen_) {
    T->constant = false;
    T->frozen = false;
  }
  frozen_.clear();
}

double* Engine::scratch(int64_t n) {
  n = std::max<int64_t>(n, 1);
  int best = -1;
  for (int i = 0; i < (int)pool_.size(); ++i)
    if (!pool_[i].busy && pool_[i].n >= n &&
        (best < 0 || pool_[i].n < pool_[best].n))
      best = i;
  if (best < 0) {
    // idle buffers too small for this request go back to the allocator, so
    // the pool stays near the largest simultaneous need
    std::vector<Buf> keep;
    for (auto& b : pool_) {
      if (!b.busy)
        al.release(b.d, (size_t)b.n * 8);
      else
        keep.push_back(b);
    }
    pool_.swap(keep);
    Buf b;
    b.n = n;
    b.d = (double*)al.alloc((size_t)n * 8);
    b.busy = false;
    pool_.push_back(b);
    best = (int)pool_.size() - 1;
  }
  pool_[best].busy = true;
  return pool_[best].d;
}

void Engine::release_scratch() {
  for (auto& b : pool_) b.busy = false;
}

const DevTasks& Engine::perm_tasks(const Layout& Y, const Layout& X,
                                   const int* xq, bool eps) {
  std::ostringstream key;
  key << Y.key() << '<' << X.key() << ':';
  for (int q = 0; q < Y.rank; ++q) key << xq[q];
  if (eps) key << 'e';
  auto it = task_cache_.find(key.str());
  if (it != task_cache_.end()) return it->second;

  const int nocc = dims_.total(SO);
  std::vector<PermTask> tasks;
  bool embed = false;
  for_each_tuple(dims_.h, Y.rank, Y.gtot, [&](const int* gy) {
    int gx[MAXRANK] = {0, 0, 0, 0};
    for (int q = 0; q < Y.rank; ++q) gx[xq[q]] = gy[q];
    SubBlock SY = sub_block(Y, dims_, gy);
    SubBlock SX = sub_block(X, dims_, gx);
    PermTask t;
    std::memset(&t, 0, sizeof(t));
    t.rank = Y.rank;
    t.ybase = SY.base;
    t.xbase = SX.base;
    int64_t n = 1;
    for (int q = 0; q < Y.rank; ++q) {
      const int ys = Y.sp[q], xs = X.sp[xq[q]], g = gy[q];
      int dim;
      if (ys == xs) {
        dim = dims_.n[ys][g];
      } else if (xs == SA && (ys == SO || ys == SV)) {
        dim = dims_.n[ys][g];
        t.xbase += (int64_t)dims_.off_all[ys][g] * SX.stride[xq[q]];
      } else if (ys == SA && (xs == SO || xs == SV)) {
        dim = dims_.n[xs][g];
        t.ybase += (int64_t)dims_.off_all[xs][g] * SY.stride[q];
        embed = true;
      } else {
        throw EngineError("axpy: incompatible index spaces");
      }
      t.dim[q] = dim;
      t.ys[q] = SY.stride[q];
      t.xs[q] = SX.stride[xq[q]];
      if (eps) {
        const int s = ys;
        if (s == SO) {
          t.gidx[q] = dims_.gstart[SO][g];
          t.sgn[q] = 1;
        } else if (s == SV) {
          t.gidx[q] = nocc + dims_.gstart[SV][g];
          t.sgn[q] = -1;
        }
      }
      n *= dim;
    }
    t.n = n;
    if (n > 0) {
      // every access of the box must stay inside both buffers
      int64_t ymax = t.ybase, xmax = t.xbase;
      for (int q = 0; q < Y.rank; ++q) {
        ymax += (int64_t)(t.dim[q] - 1) * t.ys[q];
        xmax += (int64_t)(t.dim[q] - 1) * t.xs[q];
      }
      if (t.ybase < 0 || t.xbase < 0 || ymax >= Y.size || xmax >= X.size)
        throw EngineError("internal: permutation task out of bounds");
      if (!eps) merge_box_dims(t);
      set_division_magic(t);
      tasks.push_back(t);
    }
  });
  if (Y.rank == 0 && Y.gtot == 0 && tasks.empty()) {
    // scalar copy
    PermTask t;
    std::memset(&t, 0, sizeof(t));
    t.n = 1;
    set_division_magic(t);
    tasks.push_back(t);
  }
  std::vector<Chunk> chunks;
  // chunk length: about four CTAs per SM over all tasks (small tensors are
  // latency bound), between 512 elements and chunk_elems()
  int64_t total = 0;
  for (const PermTask& t : tasks) total += t.n;
  int CH = chunk_elems();
  while (CH > 512 && total / CH < 4 * (int64_t)sm_count()) CH /= 2;
  for (int i = 0; i < (int)tasks.size(); ++i)
    for (int64_t s = 0; s < tasks[i].n; s += CH)
      chunks.push_back({i, (int)std::min<int64_t>(CH, tasks[i].n - s), s});
  DevTasks dt;
  dt.ntask = (int)tasks.size();
  dt.nchunk = (int)chunks.size();
  dt.embed = embed;
  if (dt.ntask) {
    dt.tasks = (PermTask*)al.alloc(tasks.size() * sizeof(PermTask));
    dt.chunks = (Chunk*)al.alloc(chunks.size() * sizeof(Chunk));
    ECK(cudaMemcpyAsync(dt.tasks, tasks.data(),
                        tasks.size() * sizeof(PermTask),
                        cudaMemcpyHostToDevice, st_));
    ECK(cudaMemcpyAsync(dt.chunks, chunks.data(),
                        chunks.size() * sizeof(Chunk), cudaMemcpyHostToDevice,
                        st_));
    ECK(cudaStreamSynchronize(st_));  // host vectors go out of scope
  }
  return task_cache_.emplace(key.str(), dt).first->second;
}

const DevTasks& Engine::update_tasks(const Layout& L) {
  int xq[MAXRANK] = {0, 1, 2, 3};
  return perm_tasks(L, L, xq, true);
}

void Engine::axpy_raw(double alpha, const Layout& XL, const double* X,
                      const std::string& ix, double beta, const Layout& YL,
                      double* Y, const std::string& iy,
                      const double* d_scale) {
  if ((int)ix.size() != XL.rank || (int)iy.size() != YL.rank ||
      XL.rank != YL.rank)
    throw EngineError("axpy: rank / index string mismatch " + ix + "->" + iy);
  if (XL.gtot != YL.gtot) throw EngineError("axpy: symmetry mismatch");
  int xq[MAXRANK] = {0, 0, 0, 0};
  for (int q = 0; q < YL.rank; ++q) {
    const size_t p = ix.find(iy[q]);
    if (p == std::string::npos)
      throw EngineError("axpy: index sets differ " + ix + "->" + iy);
    xq[q] = (int)p;
  }
  const DevTasks& dt = perm_tasks(YL, XL, xq, false);
  if (dt.embed && beta != 1.0)
    throw EngineError("axpy: embedding requires beta = 1");
  int64_t nel = 0;
  if (prof_on_) {
    // bytes: read X, write Y (+ read Y when accumulating)
    nel = (beta == 0.0 ? 16 : 24) * (dt.embed ? XL.size : YL.size);
  }
  timed(K_PERM, (double)nel, [&] {
    return perm_axpy(dt.tasks, dt.chunks, dt.nchunk, alpha, X, beta, Y, st_,
                     d_scale);
  });
}

void Engine::axpy(double alpha, Tensor* X, const char* ix, double beta,
                  Tensor* Y, const char* iy) {
  if (recording_) tape_.push_back({1, alpha, beta, X, nullptr, Y, ix, "", iy});
  if (record_only_) return;
  ++Y->ver;
  SigScope sig(this, std::string("axpy ") + ix + "->" + iy);
  axpy_raw(alpha, X->lay, X->d, ix, beta, Y->lay, Y->d, iy);
}

void Engine::contract(double alpha, Tensor* A, const char* ia_, Tensor* B,
                      const char* ib_, double beta, Tensor* C,
                      const char* ic_) {
  const std::string ia(ia_), ib(ib_), ic(ic_);
  if ((int)ia.size() != A->lay.rank || (int)ib.size() != B->lay.rank ||
      (int)ic.size() != C->lay.rank)
    throw EngineError("contract: index strings " + ia + "," + ib + "->" + ic +
                      " do not match ranks");
  if (recording_) tape_.push_back({0, alpha, beta, A, B, C, ia, ib, ic});
  if (record_only_) return;
  ++C->ver;
  SigScope sig(this, ia + ',' + ib + "->" + ic);
  cudaEvent_t tr_a = nullptr;
  if (prof_on_) {
    tr_a = get_event();
    cudaEventRecord(tr_a, st_);
  }
  // one operand a scalar (no summed index, e.g. the adjoint of an energy
  // contraction): C = beta*C + alpha*s*perm(other), a scaled permutation
  // read from the device scalar s instead of a GEMM with K = 1
  if ((A->lay.rank == 0 || B->lay.rank == 0) && A->lay.rank + B->lay.rank ==
                                                     C->lay.rank) {
    Tensor* S = A->lay.rank == 0 ? A : B;
    Tensor* X = A->lay.rank == 0 ? B : A;
    const std::string& ix = A->lay.rank == 0 ? ib : ia;
    if (S->lay.gtot == 0 && S->lay.size == 1 && X->lay.gtot == C->lay.gtot) {
      axpy_raw(alpha, X->lay, X->d, ix, beta, C->lay, C->d, ic, S->d);
      if (tr_a) {
        cudaEvent_t tr_b = get_event();
        cudaEventRecord(tr_b, st_);
        trace_pending_.push_back(
            {ia + ',' + ib + "->" + ic + " [scaled axpy]", tr_a, tr_b, 0.0});
      }
      return;
    }
  }

  std::string KA, KB, fA_A, fB_B, fA_C, fB_C;
  for (char x : ia) {
    if (ic.find(x) != std::string::npos) {
      if (ib.find(x) != std::string::npos)
        throw EngineError("contract: batch index unsupported");
      fA_A += x;
    } else if (ib.find(x) != std::string::npos) {
      KA += x;
    } else {
      throw EngineError("contract: index summed in one operand only");
    }
  }
  for (char x : ib) {
    if (ic.find(x) != std::string::npos)
      fB_B += x;
    else if (ia.find(x) != std::string::npos)
      KB += x;
    else
      throw EngineError("contract: index summed in one operand only");
  }
  for (char x : ic) {
    const bool a = ia.find(x) != std::string::npos;
    const bool b = ib.find(x) != std::string::npos;
    if (a == b) throw EngineError("contract: output index " +
                                  std::string(1, x) + " ambiguous");
    (a ? fA_C : fB_C) += x;
  }
  // letter -> space
  auto space_of = [&](char x) -> int {
    size_t p = ia.find(x);
    if (p != std::string::npos) return A->lay.sp[p];
    p = ib.find(x);
    return B->lay.sp[p];
  };
  for (char x : ia) {
    size_t p = ib.find(x);
    if (p != std::string::npos && B->lay.sp[p] != A->lay.sp[ia.find(x)])
      throw EngineError("contract: index space mismatch");
  }

  // a constant operand whose permuted copy is (or can be) kept costs
  // nothing per call
  // ... and so does a changing one whose copy of this version exists
  auto perm_cost = [&](Tensor* T, const std::string& tl, const std::string& r,
                       const std::string& c) -> int64_t {
    if (T->constant && permuted_constant(T, tl, r, c, false)) return 0;
    if (T->cacheable && permuted_current(T, tl, r, c)) return 0;
    return T->lay.size;
  };
  auto matches = [](const Tensor* T, const std::string& tl,
                    const std::string& r, const std::string& c, bool& tr) {
    if (tl == r + c && T->lay.split == (int)r.size()) {
      tr = false;
      return true;
    }
    if (tl == c + r && T->lay.split == (int)c.size()) {
      tr = true;
      return true;
    }
    return false;
  };

  // enumerate plans
  struct Plan {
    int form;
    std::string K, X, Y;
    int64_t cost;
  } best{0, "", "", "", -1};
  const std::string Ks[2] = {KA, KB};
  const std::string FAs[2] = {fA_C, fA_A};
  const std::string FBs[2] = {fB_C, fB_B};
  for (int kk = 0; kk < 2; ++kk)
    for (int fa = 0; fa < 2; ++fa)
      for (int fb = 0; fb < 2; ++fb)
        for (int form = 0; form < 2; ++form) {
          const std::string& K = Ks[kk];
          const std::string X = form ? FBs[fb] : FAs[fa];
          const std::string Y = form ? FAs[fa] : FBs[fb];
          Tensor* P = form ? B : A;
          Tensor* Q = form ? A : B;
          const std::string& pl = form ? ib : ia;
          const std::string& ql = form ? ia : ib;
          bool tr;
          int64_t cost = 0;
          if (!matches(P, pl, X, K, tr)) cost += perm_cost(P, pl, X, K);
          if (!matches(Q, ql, K, Y, tr)) cost += perm_cost(Q, ql, K, Y);
          if (!(ic == X + Y && C->lay.split == (int)X.size()))
            cost += 2 * C->lay.size;
          if (best.cost < 0 || cost < best.cost) best = {form, K, X, Y, cost};
        }

  Tensor* P = best.form ? B : A;
  Tensor* Q = best.form ? A : B;
  const std::string& pl = best.form ? ib : ia;
  const std::string& ql = best.form ? ia : ib;

  auto get = [&](Tensor* T, const std::string& tl, const std::string& r,
                 const std::string& c) -> Mat {
    bool tr;
    if (matches(T, tl, r, c, tr)) return {T->d, &T->lay, tr, T};
    if (T->constant || T->cacheable) {
      Tensor* Pc = permuted_constant(T, tl, r, c, true);
      if (Pc) return {Pc->d, &Pc->lay, false, Pc};
    }
    std::vector<int> sp;
    for (char x : r + c) sp.push_back(space_of(x));
    tmp_layouts_.push_back(std::make_unique<Layout>(
        make_layout(sp, (int)r.size(), T->lay.gtot)));
    const Layout* L = tmp_layouts_.back().get();
    double* buf = scratch(L->size);
    axpy_raw(1.0, T->lay, T->d, tl, 0.0, *L, buf, r + c);
    return {buf, L, false, nullptr};
  };
  Mat mp = get(P, pl, best.X, best.K);
  Mat mq = get(Q, ql, best.K, best.Y);
  const int gP = P->lay.gtot, gQ = Q->lay.gtot;
  const bool direct =
      (ic == best.X + best.Y && C->lay.split == (int)best.X.size());
  const Layout* DL;
  double* Dd;
  if (direct) {
    DL = &C->lay;
    Dd = C->d;
  } else {
    std::vector<int> sp;
    for (char x : best.X + best.Y) sp.push_back(space_of(x));
    tmp_layouts_.push_back(std::make_unique<Layout>(
        make_layout(sp, (int)best.X.size(), gP ^ gQ)));
    DL = tmp_layouts_.back().get();
    Dd = scratch(DL->size);
  }
  if ((gP ^ gQ) != C->lay.gtot)
    throw EngineError("contract: output symmetry mismatch");

  GemmProb probs[GEMM_MAXPROB];
  int np = 0;
  const int h = dims_.h;
  for (int GX = 0; GX < h; ++GX) {
    const int GK = GX ^ gP;
    GemmProb g;
    std::memset(&g, 0, sizeof(g));
    int64_t M, K, K2, N;
    if (!mp.trans) {
      M = mp.lay->nrow[GX];
      K = mp.lay->ncol[GX];
      g.A = mp.d + mp.lay->blk_off[GX];
      g.lda = (int)K;
    } else {
      M = mp.lay->ncol[GK];
      K = mp.lay->nrow[GK];
      g.A = mp.d + mp.lay->blk_off[GK];
      g.lda = (int)M;
      g.ta = 1;
    }
    if (!mq.trans) {
      K2 = mq.lay->nrow[GK];
      N = mq.lay->ncol[GK];
      g.B = mq.d + mq.lay->blk_off[GK];
      g.ldb = (int)N;
    } else {
      const int GY = GK ^ gQ;
      N = mq.lay->nrow[GY];
      K2 = mq.lay->ncol[GY];
      g.B = mq.d + mq.lay->blk_off[GY];
      g.ldb = (int)K2;
      g.tb = 1;
    }
    const int64_t Md = DL->nrow[GX], Nd = DL->ncol[GX];
    if (Md == 0 || Nd == 0) continue;
    if (M != Md || N != Nd || K != K2) {
      std::ostringstream os;
      os << "contract: block shape mismatch " << ia << "," << ib << "->"
         << ic << " G=" << GX << " M" << M << "/" << Md << " N" << N << "/"
         << Nd << " K" << K << "/" << K2;
      throw EngineError(os.str());
    }
    if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX)
      throw EngineError("contract: block too large");
    g.C = Dd + DL->blk_off[GX];
    g.ldc = (int)Nd;
    // operand extents inside their buffers (blocks are dense row-major)
    {
      const int64_t aoff = g.A - mp.d, boff = g.B - mq.d;
      if (aoff + M * K > mp.lay->size || boff + K * N > mq.lay->size ||
          DL->blk_off[GX] + M * N > DL->size)
        throw EngineError("internal: GEMM block out of bounds");
    }
    g.M = (int)M;
    g.N = (int)N;
    g.K = (int)K;
    probs[np++] = g;
  }
  double fl = 0;
  for (int i = 0; i < np; ++i)
    fl += 2.0 * probs[i].M * (double)probs[i].N * probs[i].K;
  const char* path = run_gemms(probs, np, mp, mq, alpha, direct ? beta : 0.0);
  if (!direct)
    axpy_raw(1.0, *DL, Dd, best.X + best.Y, beta, C->lay, C->d, ic);
  if (tr_a) {
    cudaEvent_t tr_b = get_event();
    cudaEventRecord(tr_b, st_);
    std::ostringstream key;
    if (A->ladder || B->ladder || C->ladder) key << "ladder ";
    key << ia << ',' << ib << "->" << ic << " [" << path << ']';
    trace_pending_.push_back({key.str(), tr_a, tr_b, fl});
  }
  release_scratch();
  tmp_layouts_.clear();
}

// Route the blocks of one product (they write disjoint parts of C) to the
// tensor cores or the FP64 kernel and launch them.  Tensor cores take every
// matrix-shaped block (both output sides >= 32; a short K is padded to the
// 64-wide stage, which costs MMAs the tensor pipe has to spare where the
// FP64 pipe has none): thin products (dots, outer products, o x o results,
// one output side of at most 16) stay on the FP64 path.  Returns the path
// taken.
const char* Engine::run_gemms(const GemmProb* probs, int np, const Mat& mp,
                              const Mat& mq, double alpha, double beta) {
  double fl = 0;
  for (int i = 0; i < np; ++i) {
    fl += 2.0 * probs[i].M * (double)probs[i].N * probs[i].K;
    flops += 2 * (int64_t)probs[i].M * probs[i].N * probs[i].K;
  }
  GemmProb ptc[GEMM_MAXPROB], p64[GEMM_MAXPROB];
  int ntc = 0, n64 = 0;
  double fl_tc = 0;
  const int prec = active_precision();
  for (int i = 0; i < np; ++i) {
    const GemmProb& g = probs[i];
    if (prec > 0 && std::min(g.M, g.N) >= 32 &&
        std::max(g.M, g.N) >= 64 && g.K >= 1) {
      fl_tc += 2.0 * g.M * (double)g.N * g.K;
      ptc[ntc++] = g;
    } else {
      p64[n64++] = g;
    }
  }
  if (!(fl_tc >= (double)tc_min_flops && d_err)) {
    for (int i = 0; i < ntc; ++i) p64[n64++] = ptc[i];
    ntc = 0;
    fl_tc = 0;
  }
  const char* path = ntc == 0 ? "fp64" : n64 == 0
                         ? (prec >= 12 ? "exact" : "split")
                         : (prec >= 12 ? "exact+fp64" : "split+fp64");
  if (ntc > 0) tc_contract(ptc, ntc, mp, mq, alpha, beta, fl_tc);
  if (n64 > 0) {
    const double f64 = fl - fl_tc;
    const int64_t sk = gemm_scratch_doubles(p64, n64);
    double* skb = sk > 0 ? scratch(sk) : nullptr;
    timed(K_GEMM64, f64, [&] {
      return gemm64_grouped(p64, n64, alpha, beta, skb, st_);
    });
  }
  return path;
}

void Engine::ladder_stats(double* sec, double* fl, int64_t* calls) {
  prof_collect();
  *sec = *fl = 0;
  *calls = 0;
  for (auto& kv : trace_)
    if (kv.first.rfind("ladder", 0) == 0) {
      *sec += kv.second.sec;
      *fl += kv.second.flops;
      *calls += kv.second.calls;
    }
}

void Engine::write_trace(const char* file) {
  prof_collect();
  FILE* f = std::fopen(file, "a");
  if (!f) return;
  std::vector<std::pair<double, std::string>> v;
  double tot = 0;
  for (auto& kv : trace_) {
    v.push_back({kv.second.sec, kv.first});
    tot += kv.second.sec;
  }
  std::sort(v.rbegin(), v.rend());
  std::fprintf(f, "# contraction trace: %.6f s in %zu signatures\n", tot,
               v.size());
  for (auto& p : v) {
    const TraceAgg& a = trace_[p.second];
    std::fprintf(f, "%10.6f s %7lld calls %9.3f TFLOP/s  %s\n", a.sec,
                 (long long)a.calls, a.sec > 0 ? a.flops / a.sec / 1e12 : 0.0,
                 p.second.c_str());
  }
  // device time of the launches issued for each signature, by class
  static const char* kn[K_NKIND] = {"gemm64", "permute", "update", "dot",
                                    "slice/other", "tc_float", "tc_exact"};
  std::vector<std::pair<double, int>> w;
  for (int i = 0; i < (int)sig_sec_.size(); ++i) {
    double t = 0;
    for (int k = 0; k < K_NKIND; ++k) t += sig_sec_[i][k];
    w.push_back({t, i});
  }
  std::sort(w.rbegin(), w.rend());
  std::fprintf(f, "# kernel classes per signature (device seconds)\n");
  for (auto& p : w) {
    if (p.first < 1e-4) break;
    std::fprintf(f, "%10.6f s ", p.first);
    for (int k = 0; k < K_NKIND; ++k)
      if (sig_sec_[p.second][k] > 0)
        std::fprintf(f, " %s %.4f", kn[k], sig_sec_[p.second][k]);
    std::fprintf(f, "  | %s\n", sig_name_[p.second].c_str());
  }
  std::fclose(f);
}

SlicedOp Engine::slice_side(Tensor* src, const double* ptr, int rows, int K,
                            int64_t ld, int trans, int nslice, bool exact,
                            uint8_t** cursor) {
  const int Kp = slice_kp(K);
  const size_t bytes = (size_t)nslice * rows * Kp * 2;
  const size_t ebytes = exact ? (size_t)rows * 4 : 0;
  auto split = [&](void* d, int* e) {
    timed(K_OTHER, 8.0 * rows * K + 2.0 * nslice * rows * Kp, [&] {
      return exact ? split_exact(ptr, rows, K, ld, trans, nslice, d, e, st_)
                   : split_float(ptr, rows, K, ld, trans, nslice, d, st_);
    });
  };
  bool cache = src && src->constant;
  if (cache && src->frozen) {
    // frozen tensors: cached within their budget (entries are replaced
    // in place when the key exists)
    std::ostringstream k0;
    k0 << (const void*)ptr << ':' << rows << ':' << K << ':' << ld << ':'
       << trans << ':' << nslice << ':' << (exact ? 'x' : 'f');
    if (!slice_cache_.count(k0.str()) &&
        (frozen_slice_bytes_ + (int64_t)(bytes + ebytes) > frozen_slice_cap_ ||
         !device_free_above(bytes + ebytes, (size_t)8 << 30)))
      cache = false;
  }
  if (cache) {
    std::ostringstream key;
    key << (const void*)ptr << ':' << rows << ':' << K << ':' << ld << ':'
        << trans << ':' << nslice << ':' << (exact ? 'x' : 'f');
    auto it = slice_cache_.find(key.str());
    if (it != slice_cache_.end() && it->second.ver == src->ver)
      return {it->second.data, it->second.exps, rows, Kp};
    if (it != slice_cache_.end()) {
      al.release(it->second.data, it->second.bytes);
      if (it->second.exps) al.release(it->second.exps, it->second.ebytes);
      if (it->second.owner && it->second.owner->frozen)
        frozen_slice_bytes_ -= (int64_t)(it->second.bytes + it->second.ebytes);
      slice_cache_.erase(it);
    }
    SliceEntry en;
    en.bytes = bytes;
    en.ebytes = ebytes;
    en.ver = src->ver;
    en.owner = src;
    if (src->frozen) frozen_slice_bytes_ += (int64_t)(bytes + ebytes);
    en.data = al.alloc(bytes);
    en.exps = exact ? (int*)al.alloc(ebytes) : nullptr;
    split(en.data, en.exps);
    slice_cache_[key.str()] = en;
    return {en.data, en.exps, rows, Kp};
  }
  uint8_t* d = *cursor;
  *cursor += (bytes + 1023) / 1024 * 1024;
  int* e = nullptr;
  if (exact) {
    e = (int*)*cursor;
    *cursor += (ebytes + 1023) / 1024 * 1024;
  }
  split(d, e);
  return {d, e, rows, Kp};
}

// Tensor-core contraction: each side is sliced once (constant tensors from
// the cache), symmetric blocks are read untransposed, then one grouped
// launch of the split-precision (1-3 slices) or exact-slice (12-14) kernel.
void Engine::tc_contract(const GemmProb* probs, int np, const Mat& mp,
                         const Mat& mq, double alpha, double beta, double fl) {
  const int prec = active_precision();
  const bool exact = prec >= 12;
  const int ns = exact ? prec - 10 : prec;
  int64_t wsb = 1024;
  for (int i = 0; i < np; ++i) {
    const int64_t Kp = slice_kp(probs[i].K);
    wsb += (int64_t)ns * (probs[i].M + probs[i].N) * Kp * 2 +
           (int64_t)(probs[i].M + probs[i].N) * 4 + 4 * 1024;
  }
  uint8_t* cur = (uint8_t*)scratch((wsb + 7) / 8);
  TcProb tp[GEMM_MAXPROB];
  for (int i = 0; i < np; ++i) {
    const GemmProb& g = probs[i];
    // op(A) rows: A[m][k] unless ta; symmetric square blocks: A^T == A
    int ta = g.ta;
    if (ta && mp.src && mp.src->symmetric && g.M == g.K) ta = 0;
    // op(B)^T rows: B[n][k] when tb, else B[k][n]
    int btr = g.tb ? 0 : 1;
    if (btr && mq.src && mq.src->symmetric && g.N == g.K) btr = 0;
    tp[i].a = slice_side(mp.src, g.A, g.M, g.K, g.lda, ta, ns, exact, &cur);
    tp[i].b = slice_side(mq.src, g.B, g.N, g.K, g.ldb, btr, ns, exact, &cur);
    tp[i].C = g.C;
    tp[i].M = g.M;
    tp[i].N = g.N;
    tp[i].K = g.K;
    tp[i].ldc = g.ldc;
  }
  tc_flops += (int64_t)fl;
  if (exact) {
    const int64_t sk = oz_sliced_scratch_doubles(tp, np);
    double* skb = sk > 0 ? scratch(sk) : nullptr;
    timed(K_OZ, fl, [&] {
      return oz_gemm_sliced(tp, np, alpha, beta, ns, skb, d_err, st_);
    });
  } else {
    const int64_t sk = tc_sliced_scratch_doubles(tp, np, ns);
    double* skb = sk > 0 ? scratch(sk) : nullptr;
    timed(K_TC, fl, [&] {
      return tc_gemm_sliced(tp, np, alpha, beta, ns, skb, d_err, st_);
    });
  }
}

void Engine::backward(const std::vector<std::pair<Tensor*, Tensor*>>& seeds,
                      int active) {
  const bool rec = recording_;
  recording_ = false;
  for (auto& kv : tensors_) kv.second->req = false;
  for (auto& kv : tensors_) {
    Tensor* t = kv.second.get();
    if (t->tag & active) t->req = true;
  }
  for (const Op& op : tape_) {
    if (op.A->req || (op.kind != 1 && op.B->req)) op.C->req = true;
  }
  // zero adjoints of everything that carries one
  std::vector<Tensor*> req;
  for (auto& kv : tensors_)
    if (kv.second->req) req.push_back(kv.second.get());
  for (Tensor* t : req) zero(adjoint(t));
  for (auto& s : seeds) {
    if (!s.first->req) continue;
    Tensor* a = adjoint(s.first);
    if (s.second) {
      ECK(cudaMemcpyAsync(a->d, s.second->d, (size_t)a->lay.size * 8,
                          cudaMemcpyDeviceToDevice, st_));
    } else {
      const double one = 1.0;
      ECK(cudaMemcpyAsync(a->d, &one, 8, cudaMemcpyHostToDevice, st_));
      ECK(cudaStreamSynchronize(st_));
    }
  }
  for (auto it = tape_.rbegin(); it != tape_.rend(); ++it) {
    const Op& op = *it;
    if (!op.C->req) continue;
    Tensor* Cb = op.C->adj;
    if (op.kind == 0) {
      if (op.A->req)
        contract(op.alpha, Cb, op.ic.c_str(), op.B, op.ib.c_str(), 1.0,
                 adjoint(op.A), op.ia.c_str());
      if (op.B->req)
        contract(op.alpha, op.A, op.ia.c_str(), Cb, op.ic.c_str(), 1.0,
                 adjoint(op.B), op.ib.c_str());
    } else if (op.kind == 2) {
      if (op.A->req && !op.B->req)   // amplitude adjoint only: the same map
        ladder_lin_apply(1, op.alpha, Cb, op.B, false, adjoint(op.A));
      else
        ladder_adjoint(op.alpha, Cb, op.A, op.B,
                       op.A->req ? adjoint(op.A) : nullptr,
                       op.B->req ? adjoint(op.B) : nullptr);
    } else if (op.kind == 3) {
      // R[ij,ab] += alpha T[ij,cd] W[ab,cd]; W symmetric per block
      if (op.A->req)
        ladder_lin_apply(1, op.alpha, Cb, op.B, true, adjoint(op.A));
      if (op.B->req)
        contract(op.alpha, op.A, "ijcd", Cb, "ijab", 1.0, adjoint(op.B),
                 "abcd");
    } else {
      if (op.A->req)
        axpy(op.alpha, Cb, op.ic.c_str(), 1.0, adjoint(op.A), op.ia.c_str());
    }
    if (op.beta == 0.0)
      zero(Cb);
    else if (op.beta != 1.0)
      launches += axpby(0.0, Cb->d, op.beta, Cb->d, Cb->lay.size, st_);
  }
  recording_ = rec;
}

}  // namespace cdcc
