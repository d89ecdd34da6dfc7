// dpd.h -- direct-product-decomposition (DPD) layouts of symmetry-blocked
// tensors (Sec. 3.1).
//
// Every tensor index lives in a space (occupied, virtual, Cholesky or all
// orbitals); each space is split into irreps 0..h-1.  A tensor with indices
// (x_0..x_{k-1}) and total irrep G_tot stores only the irrep tuples with
// g_0 ^ ... ^ g_{k-1} == G_tot.  Its layout is a block-diagonal matrix: the
// first `split` indices form the row group, the rest the column group; one
// dense row-major block per row irrep G (rows: row tuples of irrep G, cols:
// column tuples of irrep G ^ G_tot).  Inside a group, tuples are ordered by
// their irrep labels (lexicographic, g_0 slowest) and then by the local
// indices, row-major.  Any fully specified irrep tuple therefore addresses a
// dense k-dimensional box with affine strides ("sub-block").
#pragma once
#include <cstdint>
#include <vector>
#include <string>
#include <functional>

namespace cdcc {

constexpr int MAXIRR = 8;
constexpr int MAXRANK = 4;

enum Space : int { SO = 0, SV = 1, SQ = 2, SA = 3, NSPACE = 4 };

struct Dims {
  int h = 1;
  int n[NSPACE][MAXIRR] = {};
  // offset of the occupied / virtual orbitals of irrep g inside the block of
  // all orbitals of irrep g (SO: 0, SV: n[SO][g], SA: 0)
  int off_all[NSPACE][MAXIRR] = {};
  // first global index of irrep g inside its space (orbitals: occupied
  // range starts at 0, virtual range at nocc)
  int gstart[NSPACE][MAXIRR] = {};
  int total(int s) const {
    int t = 0;
    for (int g = 0; g < h; ++g) t += n[s][g];
    return t;
  }
};

struct Layout {
  int rank = 0;
  int sp[MAXRANK] = {0, 0, 0, 0};
  int gtot = 0;
  int split = 0;
  int h = 1;
  int64_t blk_off[MAXIRR] = {};
  int64_t nrow[MAXIRR] = {};
  int64_t ncol[MAXIRR] = {};
  std::vector<int64_t> rsub;  // [G * ncode_r + code] row offset in block G
  std::vector<int64_t> csub;  // [Gc * ncode_c + code] col offset
  int ncode_r = 1, ncode_c = 1;
  int64_t size = 0;

  void build(const Dims& d);
  bool same(const Layout& o) const {
    if (rank != o.rank || gtot != o.gtot || split != o.split) return false;
    for (int q = 0; q < rank; ++q)
      if (sp[q] != o.sp[q]) return false;
    return true;
  }
  std::string key() const;
};

struct SubBlock {
  int64_t base;
  int64_t stride[MAXRANK];
  int dim[MAXRANK];
  bool empty;
};

SubBlock sub_block(const Layout& L, const Dims& d, const int* g);

// Enumerate all irrep tuples of `rank` indices with xor == gtot.
void for_each_tuple(int h, int rank, int gtot,
                    const std::function<void(const int*)>& f);

// A dense strided box copy/axpy task (device side descriptor).
struct PermTask {
  int64_t ybase, xbase;
  int64_t ys[MAXRANK], xs[MAXRANK];
  int dim[MAXRANK];
  int rank;
  int64_t n;       // elements in the box
  // global index bases for elementwise kernels that need orbital energies
  int gidx[MAXRANK];
  int sgn[MAXRANK];  // +1 occupied, -1 virtual, 0 unused
};

struct Chunk {
  int task;
  int len;          // elements of the task this chunk covers (from start)
  int64_t start;
};

}  // namespace cdcc
