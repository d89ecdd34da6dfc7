// engine.h -- symmetry-blocked tensor engine with a reverse-mode tape.
//
// Tensors are persistent, named DPD arrays (dpd.h) in device memory.  Two
// primitive operations are provided:
//   contract:  C = beta*C + alpha * sum_K A * B   (binary contraction; the
//              planner permutes operands into matrix form when needed and
//              issues ONE grouped GEMM over all irrep blocks)
//   axpy:      Y = beta*Y + alpha * perm(X)       (index permutation, also
//              extraction of / embedding into the "all orbitals" space)
// When recording, each call is appended to a tape; backward() replays the
// tape in reverse with the adjoint rules of the two primitives.  The Lambda
// equations (Sec. 2.3) are the adjoint of the amplitude residual with
// respect to the amplitudes, and the Cholesky-basis density Gamma^P
// (Sec. 2.4, 2.6) is its adjoint with respect to the Cholesky vectors.
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <map>
#include <memory>
#include <set>
#include <string>
#include <vector>

#include "dpd.h"
#include "kernels.h"

namespace cdcc {

struct DevAlloc {
  void* (*fa)(size_t, void*, void*) = nullptr;
  void (*ff)(void*, size_t, void*, void*) = nullptr;
  void* user = nullptr;
  cudaStream_t st = 0;
  void* alloc(size_t bytes);
  void release(void* p, size_t bytes);
};

// more than need + reserve bytes of device memory free right now
bool device_free_above(size_t need, size_t reserve);

enum LeafTag : int { TAG_NONE = 0, TAG_AMP = 1, TAG_L = 2, TAG_H = 4 };

struct Tensor {
  std::string name;
  Layout lay;
  double* d = nullptr;
  bool owns = true;
  Tensor* parent = nullptr;  // view into parent's buffer
  int64_t offset = 0;
  int tag = TAG_NONE;        // leaf tag (0 = not a leaf)
  Tensor* adj = nullptr;
  bool req = false;
  // every block is a square symmetric matrix (rows and columns are the same
  // index group), so it can be read as its own transpose
  bool symmetric = false;
  // amplitude independent: its tensor-core slices are cached per version
  bool constant = false;
  // operand of the particle-particle ladder ((ac|bd) integrals and their
  // adjoint): contractions touching it are timed as ladder work
  bool ladder = false;
  // constant only while the adjoint sweeps run (Engine::freeze_tape_operands)
  bool frozen = false;
  // written only through engine operations (each bumps ver), so a permuted
  // copy may be kept and reused while ver is unchanged
  bool cacheable = false;
  uint64_t ver = 0;   // bumped on every write
};

struct DevTasks {
  PermTask* tasks = nullptr;
  Chunk* chunks = nullptr;
  int ntask = 0, nchunk = 0;
  bool embed = false;
};

class EngineError : public std::exception {
 public:
  explicit EngineError(std::string m) : msg(std::move(m)) {}
  const char* what() const noexcept override { return msg.c_str(); }
  std::string msg;
};

// On-the-fly ladder row batch: the (ab|cd) rows (a,b) with a in [a0,a1) of
// irrep ga and b of irrep ga^G, for the pair irrep G.
struct LadBatch {
  int G, ga, a0, a1;   // pair irrep, irrep of a, a range (local indices)
  int64_t rows;        // (a,b) rows = (a1 - a0) * n_v(ga ^ G)
};
// row batches of a doubles layout {SO,SO,SV,SV}/2, at most batch_bytes of
// FP64 rows each (host only)
std::vector<LadBatch> ladder_batch_list(const Layout& TL, const Dims& d,
                                        int64_t batch_bytes);

// Index tables of the +/- packed ladder (ladder_pm.cu) for one doubles
// layout: per pair irrep G the canonical occupied pairs (rows of (i,j) and
// (j,i), [2][uo] at orow[G]) and virtual pairs (columns of (c,d) and (d,c),
// [2][uv] at vcol[G]); per row batch with ga >= gb its canonical (a,b) rows
// ([3][nv] at vrow: row in the batch, Y columns of (a,b) and (b,a) or -1).
// Offsets are 32-bit, inside the DPD block of G.
struct PmBatch {
  LadBatch b;
  int nv;          // canonical (a,b) rows of the batch
  int64_t vrow;    // offset of its [3][nv] table
};
struct PmPlan {
  std::string key;
  int uo[MAXIRR] = {}, uv[MAXIRR] = {};
  int64_t orow[MAXIRR] = {}, vcol[MAXIRR] = {};   // offsets in the table
  std::vector<PmBatch> batches;
  int* d_tab = nullptr;   // the table on the device (Engine::pm_plan)
  size_t bytes = 0;
  int64_t max_a = 0, max_w = 0;   // doubles of A+- and of a batch's W+-
};
// fill P (without d_tab) and the host table (host only; throws EngineError
// when an offset does not fit in 32 bits)
void pm_host_tables(const Layout& TL, const Dims& d, int64_t batch_bytes,
                    PmPlan& P, std::vector<int>& tab);

class Engine {
 public:
  Engine(const Dims& d, cudaStream_t st, DevAlloc al);
  ~Engine();

  const Dims& dims() const { return dims_; }
  cudaStream_t stream() const { return st_; }

  // get-or-create a persistent tensor
  Tensor* tensor(const std::string& name, std::vector<int> spaces, int split,
                 int gtot = 0);
  // a view of `n` doubles into `parent` at `offset` with its own layout
  Tensor* view(const std::string& name, Tensor* parent, int64_t offset,
               std::vector<int> spaces, int split, int gtot = 0);
  Tensor* flat(const std::string& name, int64_t n);  // 1-D helper buffer
  Tensor* find(const std::string& name);
  Layout layout(const std::vector<int>& spaces, int split, int gtot = 0) {
    return make_layout(spaces, split, gtot);
  }

  void zero(Tensor* t);
  void contract(double alpha, Tensor* A, const char* ia, Tensor* B,
                const char* ib, double beta, Tensor* C, const char* ic);
  void axpy(double alpha, Tensor* X, const char* ix, double beta, Tensor* Y,
            const char* iy);

  // Particle-particle ladder with the integrals assembled on the fly from
  // the Cholesky vectors (Sec. 2.3):
  //   R[ij,ab] += alpha * sum_cd T[ij,cd] (ac|bd),  (ac|bd) = sum_P L_ac L_bd
  // T, R: {SO,SO,SV,SV} split 2; L: {SQ,SV,SV} split 1, every L^P symmetric.
  // The (ab|cd) matrix is never stored whole: row batches (a in a range of
  // one irrep, all b) are built by one grouped GEMM over P, permuted into
  // (ab|cd) order and applied at once.  Recorded as one tape operation whose
  // adjoint rebuilds the batches (T and L adjoints).
  void ladder(double alpha, Tensor* T, Tensor* L, Tensor* R);
  // The same ladder with the (ac|bd) integrals stored as W[(ab),(cd)]
  // (symmetric per block):  R[ij,ab] += alpha * sum_cd T[ij,cd] W[ab,cd].
  // Recorded as one tape operation (adjoints for T and W).
  void ladder_stored(double alpha, Tensor* T, Tensor* W, Tensor* R);
  // device bytes of one row batch of the (ab|cd) matrix (two such buffers)
  int64_t ladder_batch_bytes = (int64_t)2 << 30;

  // Linearised ladder for the accurate phase of the mixed schedules.  The
  // ladder is linear in its input X (the amplitudes in the forward
  // residual, the adjoint dR in the Lambda sweep; W symmetric makes both the
  // same map Lad).  With an anchor X0 evaluated in the accurate arithmetic,
  //     Lad(X) = Lad_acc(X0) + Lad_delta(X - X0),
  // where Lad_delta runs in the cheaper arithmetic `prec`; its rounding
  // error scales with |X - X0|, which is small once the iterations are near
  // convergence.  which = 0: forward ladder, 1: amplitude adjoint of the
  // ladder (used when the Cholesky vectors need no adjoint).  mode 0: off
  // (every call accurate), 1: the next call evaluates a new anchor
  // accurately (then mode 2), 2: apply around the anchor.
  void ladder_lin(int which, int mode, int prec = 2);
  // true when the last linearised call of `which` evaluated an anchor (its
  // result was then the accurate ladder)
  bool ladder_lin_anchored(int which) const { return lin_[which].anchored; }

  // tape
  void record(bool on) { recording_ = on; }
  // append to the tape without executing (results already in place)
  void record_only(bool on) { record_only_ = on; }
  void clear_tape() { tape_.clear(); }
  size_t tape_size() const { return tape_.size(); }
  // Run the tape backwards.  `seeds`: (tensor, seed values tensor or null =
  // all ones for rank-0 tensors).  Leaves whose tag is in `active` receive
  // adjoints (tensor->adj).
  void backward(const std::vector<std::pair<Tensor*, Tensor*>>& seeds,
                int active);
  Tensor* adjoint(Tensor* t);

  // elementwise helpers on DPD tensors
  const DevTasks& update_tasks(const Layout& L);  // with orbital energies
  double* scratch(int64_t n);                     // per-call temporary
  void release_scratch();

  int64_t launches = 0;
  int64_t flops = 0;  // FP64 GEMM flops issued

  // Arithmetic of the contractions: 0 = FP64 DFMA; 1..3 = tensor-core GEMM
  // with that many BF16 slices (FP32 accumulation); 12..14 = exact-slice
  // tensor-core GEMM with 2..4 integer slices (FP64-class accuracy); applied
  // to every contraction of at least `tc_min_flops` flops (smaller ones stay
  // FP64).
  // (a change drops the cached slices of the previous arithmetic)
  void set_precision(int slices);
  int precision() const { return tc_slices_; }
  // arithmetic in effect for the next contraction (a temporary override of
  // the linearised ladder, else the precision set above)
  int active_precision() const {
    return tc_override_ >= 0 ? tc_override_ : tc_slices_;
  }
  int64_t tc_min_flops = (int64_t)1 << 26;
  unsigned int* d_err = nullptr;   // device error flag of bounded waits
  int64_t tc_flops = 0;            // algorithmic flops run on tensor cores

  // Optional per-kernel-class timing with CUDA events on the engine stream.
  enum ProfKind : int { K_GEMM64 = 0, K_PERM = 1, K_UPDATE = 2, K_DOT = 3,
                        K_OTHER = 4, K_TC = 5, K_OZ = 6, K_NKIND = 7 };
  void profile(bool on) { prof_on_ = on; }
  // device bytes for permuted copies of constant tensors (0: none); the
  // same budget again for the slices of frozen tensors
  void set_perm_cache_bytes(int64_t b) {
    perm_const_cap_ = b;
    frozen_slice_cap_ = b;
  }
  // The operands of the recorded forward operations keep their values
  // while adjoint sweeps of the tape run (the Lambda iterations and the
  // density sweep write adjoints only): treat them as constant, so that
  // their permuted copies and tensor-core slices are made once and reused
  // by every sweep (within the cache budgets).  thaw() ends this and frees
  // what was kept for them.
  void freeze_tape_operands();
  void thaw();
  // keep up to `bytes` of on-the-fly ladder batch slices across ladder
  // applications (0 frees them and stops keeping)
  void ladder_keep_slices(int64_t bytes);
  // on-the-fly ladder with symmetric/antisymmetric (+/-) packing of the
  // three index pairs (Sec. 2.3): a quarter of the product flops, for
  // pair-symmetric amplitudes (it returns the ladder of the pair-symmetrised
  // input)
  void set_ladder_pm(bool on) { ladder_pm_ = on; }
  bool ladder_pm() const { return ladder_pm_; }
  // a rejected launch (bad configuration, resources) is an error, never a
  // silently missing result
  static void check_launch() {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
      throw EngineError(std::string("kernel launch: ") +
                        cudaGetErrorString(e));
  }
  template <class F>
  void timed(int kind, double work, F launch) {
    if (!prof_on_) {
      launches += launch();
      check_launch();
      return;
    }
    cudaEvent_t a = get_event(), b = get_event();
    cudaEventRecord(a, st_);
    const int n = launch();
    check_launch();
    cudaEventRecord(b, st_);
    launches += n;
    pending_.push_back({kind, a, b, work, n, cur_sig_});
    if (pending_.size() > 8192) prof_collect();
  }
  void prof_collect();
  // append the per-contraction trace (profiling on) to `file`
  void write_trace(const char* file);
  // device seconds, algorithmic flops and calls of the ladder contractions
  // (profiling on): forward, adjoint, integral build and its adjoint
  void ladder_stats(double* sec, double* flops, int64_t* calls);
  double prof_sec[K_NKIND] = {}, prof_work[K_NKIND] = {};
  int64_t prof_n[K_NKIND] = {};

  DevAlloc al;

 private:
  struct Op {
    int kind;  // 0 contract, 1 axpy, 2 ladder (A = T, B = L, C = R),
               // 3 stored ladder (A = T, B = W, C = R)
    double alpha, beta;
    Tensor *A, *B, *C;
    std::string ia, ib, ic;
  };
  struct Mat {
    double* d;
    const Layout* lay;
    bool trans;
    Tensor* src;   // the tensor itself when used in place, else null
  };
  struct SliceEntry {
    void* data;
    int* exps;
    size_t bytes, ebytes;
    uint64_t ver;
    const Tensor* owner;
  };
  int64_t frozen_slice_bytes_ = 0;
  int64_t frozen_slice_cap_ = int64_t(32) << 30;
  std::vector<Tensor*> frozen_;
  std::map<std::string, SliceEntry> slice_cache_;
  // contraction trace (profiling on): signature -> events
  struct TraceRec {
    std::string key;
    cudaEvent_t a, b;
    double flops;
  };
  std::vector<TraceRec> trace_pending_;
  struct TraceAgg {
    double sec = 0, flops = 0;
    int64_t calls = 0;
  };
  std::map<std::string, TraceAgg> trace_;
  // K-major slices of one GEMM side (see kernels.h); cached for constant
  // tensors, else split into the workspace at *cursor
  SlicedOp slice_side(Tensor* src, const double* ptr, int rows, int K,
                      int64_t ld, int trans, int nslice, bool exact,
                      uint8_t** cursor);
  void tc_contract(const GemmProb* probs, int np, const Mat& mp,
                   const Mat& mq, double alpha, double beta, double fl);
  const char* run_gemms(const GemmProb* probs, int np, const Mat& mp,
                        const Mat& mq, double alpha, double beta);

  // on-the-fly ladder
  std::vector<LadBatch> ladder_batches(const Layout& TL);
  double ladder_build(const LadBatch& b, Tensor* L);   // -> lad_w_
  // float-slice arithmetic: the build GEMM writes the BF16 slices of the
  // batch rows directly (lad_ws_) and the apply reads them; false when a
  // block is too small for the tensor-core route
  bool ladder_fusable(const LadBatch& b, const Layout& TL, const Layout& LL);
  // into dst (ns * rows * Kp BF16; null: the batch buffer lad_ws_)
  double ladder_build_sliced(const LadBatch& b, Tensor* L, int ns,
                             void* dst = nullptr);
  void ladder_apply_sliced(const LadBatch& b, double alpha, Tensor* X,
                           Tensor* Y, int ns, const void* W = nullptr);
  void* lad_ws_ = nullptr;
  size_t lad_ws_bytes_ = 0;
  // BF16 slices of the on-the-fly batch rows kept across ladder
  // applications (float-slice arithmetic; they depend on L only): key
  // "G,ga,a0,a1,ns" -> buffer, valid for one version of L
  struct LadSlices {
    void* data;
    size_t bytes;
    uint64_t lver;
    const Tensor* L;
  };
  std::map<std::string, LadSlices> lad_cache_;
  int64_t lad_cache_bytes_ = 0, lad_cache_cap_ = 0;
  void ladder_perm(const LadBatch& b, bool inverse, const double* src,
                   double* dst);
  void ladder_apply_batch(const LadBatch& b, double alpha, Tensor* X,
                          Tensor* Y);
  void ladder_adjoint(double alpha, Tensor* dR, Tensor* T, Tensor* L,
                      Tensor* dT, Tensor* dL);
  void ladder_reserve(int64_t n);
  // plain ladder map Y += alpha * Lad(X) (on the fly from L, or stored W)
  void ladder_map(double alpha, Tensor* X, Tensor* LW, bool stored,
                  Tensor* Y);
  struct LadderLin {
    int mode = 0, prec = 2;
    bool anchored = false;
    Tensor *in = nullptr, *out = nullptr, *d = nullptr;
  };
  LadderLin lin_[2];
  void ladder_lin_apply(int which, double alpha, Tensor* X, Tensor* LW,
                        bool stored, Tensor* Y);
  // +/- packed ladder: index tables per layout (device, one allocation)
  PmPlan pm_;
  bool ladder_pm_ = false;
  double* pm_a_ = nullptr;   // A+ | A- of one pair irrep (FP64)
  double* pm_w_ = nullptr;   // W+ | W- of one batch (FP64)
  int64_t pm_a_n_ = 0, pm_w_n_ = 0;
  void* pm_as_ = nullptr;    // BF16 slices of A+ | A-
  size_t pm_as_bytes_ = 0;
  const PmPlan& pm_plan(const Layout& TL);
  void ladder_map_pm(double alpha, Tensor* X, Tensor* L, Tensor* Y);
  int tc_override_ = -1;
  double* lad_x_ = nullptr;
  double* lad_w_ = nullptr;
  int64_t lad_n_ = 0;

  Tensor* new_tensor(const std::string& name, std::vector<int> spaces,
                     int split, int gtot);
  const DevTasks& perm_tasks(const Layout& Y, const Layout& X,
                             const int* xq, bool eps);
  void axpy_raw(double alpha, const Layout& XL, const double* X,
                const std::string& ix, double beta, const Layout& YL,
                double* Y, const std::string& iy,
                const double* d_scale = nullptr);
  Layout make_layout(const std::vector<int>& spaces, int split, int gtot);

  Dims dims_;
  cudaStream_t st_;
  bool recording_ = false;
  bool record_only_ = false;
  std::vector<Op> tape_;
  std::map<std::string, std::unique_ptr<Tensor>> tensors_;
  std::map<std::string, DevTasks> task_cache_;
  // scratch pool
  struct Buf {
    double* d;
    int64_t n;
    bool busy;
  };
  std::vector<Buf> pool_;
  std::vector<std::unique_ptr<Layout>> tmp_layouts_;
  struct ProfRec {
    int kind;
    cudaEvent_t a, b;
    double work;
    int n;
    int sig;   // contraction / permutation signature (-1: none)
  };
  // per-signature device time of each kernel class (profiling on): the
  // signature of the contraction or permutation being issued
  int cur_sig_ = -1;
  std::map<std::string, int> sig_id_;
  std::vector<std::string> sig_name_;
  std::vector<std::array<double, 8>> sig_sec_;
  int sig_of(const std::string& s);
  // Permuted copies of amplitude-independent (constant) tensors, made once
  // per version of the source and kept (their tensor-core slices are then
  // cached with them): key = source name + position map + split.
  struct PermConst {
    Tensor* t;
    uint64_t src_ver;
    const Tensor* src;
  };
  std::map<std::string, PermConst> perm_const_;
  int64_t perm_const_bytes_ = 0;
  int64_t perm_const_cap_ = int64_t(32) << 30;
  Tensor* permuted_constant(Tensor* T, const std::string& tl,
                            const std::string& r, const std::string& c,
                            bool create);
  bool permuted_current(Tensor* T, const std::string& tl,
                        const std::string& r, const std::string& c);
  // sets the signature for the launches issued in its scope (profiling on)
  struct SigScope {
    Engine* e;
    int prev;
    SigScope(Engine* eng, const std::string& s)
        : e(eng), prev(eng->cur_sig_) {
      if (eng->prof_on_) eng->cur_sig_ = eng->sig_of(s);
    }
    ~SigScope() { e->cur_sig_ = prev; }
  };
  cudaEvent_t get_event();
  bool prof_on_ = false;
  int tc_slices_ = 0;
  std::vector<ProfRec> pending_;
  std::vector<cudaEvent_t> ev_pool_;
};

}  // namespace cdcc
