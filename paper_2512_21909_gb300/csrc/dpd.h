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
  // division by dim[q] as a multiply and shift, exact for numerators below
  // 2^31: floor(r / dim[q]) = (r * mag[q]) >> shr[q] (set_division_magic)
  uint64_t mag[MAXRANK];
  int shr[MAXRANK];
  // 1: n < 2^31 and every offset within the box (from ybase / xbase) is
  // below 2^31, so the kernels index with 32-bit arithmetic
  int off32;
  // global index bases for elementwise kernels that need orbital energies
  int gidx[MAXRANK];
  int sgn[MAXRANK];  // +1 occupied, -1 virtual, 0 unused
};

// Fill mag/shr/off32 of a task whose dim/ys/xs/rank/n are set.  With
// l = ceil(log2 d), s = 31 + l and m = ceil(2^s / d), m d - 2^s < 2^l, so
// floor(r m / 2^s) = floor(r / d) for every 0 <= r < 2^31 (Granlund and
// Montgomery, "Division by invariant integers using multiplication",
// PLDI 1994, Theorem 4.2); r m stays below 2^64.
inline void set_division_magic(PermTask& t) {
  int64_t yspan = 0, xspan = 0;
  for (int q = 0; q < MAXRANK; ++q) {
    const int64_t d = q < t.rank && t.dim[q] > 0 ? t.dim[q] : 1;
    int l = 0;
    while ((int64_t(1) << l) < d) ++l;
    t.shr[q] = 31 + l;
    t.mag[q] = ((uint64_t(1) << t.shr[q]) + (uint64_t)d - 1) / (uint64_t)d;
    if (q < t.rank) {
      yspan += (d - 1) * (t.ys[q] < 0 ? -t.ys[q] : t.ys[q]);
      xspan += (d - 1) * (t.xs[q] < 0 ? -t.xs[q] : t.xs[q]);
    }
  }
  t.off32 = (t.n < (int64_t(1) << 31) && yspan < (int64_t(1) << 31) &&
             xspan < (int64_t(1) << 31))
                ? 1
                : 0;
}

// Merge neighbouring box dimensions q, q+1 that are contiguous in both
// tensors (ys[q] = dim[q+1] ys[q+1], same for xs) and drop extents of 1;
// the element order (row-major over the dims) is unchanged.  Only for tasks
// that do not need the per-dimension indices (no orbital energies).
inline void merge_box_dims(PermTask& t) {
  int64_t dim[MAXRANK], ys[MAXRANK], xs[MAXRANK];
  int r = 0;
  for (int q = 0; q < t.rank; ++q) {
    if (t.dim[q] == 1) continue;
    if (r > 0 && ys[r - 1] == (int64_t)t.dim[q] * t.ys[q] &&
        xs[r - 1] == (int64_t)t.dim[q] * t.xs[q] &&
        dim[r - 1] * t.dim[q] <= INT32_MAX) {
      dim[r - 1] *= t.dim[q];
      ys[r - 1] = t.ys[q];
      xs[r - 1] = t.xs[q];
      continue;
    }
    dim[r] = t.dim[q];
    ys[r] = t.ys[q];
    xs[r] = t.xs[q];
    ++r;
  }
  if (r == 0) {   // a single element
    dim[0] = 1;
    ys[0] = xs[0] = 0;
    r = 1;
  }
  for (int q = 0; q < MAXRANK; ++q) {
    t.dim[q] = q < r ? (int)dim[q] : 0;
    t.ys[q] = q < r ? ys[q] : 0;
    t.xs[q] = q < r ? xs[q] : 0;
  }
  t.rank = r;
}

struct Chunk {
  int task;
  int len;          // elements of the task this chunk covers (from start)
  int64_t start;
};

}  // namespace cdcc
