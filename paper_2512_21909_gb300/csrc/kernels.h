// kernels.h -- launchers of the CUDA kernels of the CD-CCSD library.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "dpd.h"

namespace cdcc {

constexpr int GEMM_MAXPROB = 16;

// One matrix product C = beta*C + alpha*op(A)*op(B), all row-major.
// op(A) is M x K (ta: A stored K x M), op(B) is K x N (tb: B stored N x K).
struct GemmProb {
  const double* A;
  const double* B;
  double* C;
  int M, N, K;
  int lda, ldb, ldc;
  int ta, tb;
};

// Grouped launch of up to GEMM_MAXPROB independent products sharing
// alpha/beta.  Returns the number of kernel launches issued.  `scratch` is
// used for split-K partial sums of thin products; it must hold
// gemm_scratch_doubles(...) doubles (may be null if that is 0).
int64_t gemm_scratch_doubles(const GemmProb* p, int np);
int gemm64_grouped(const GemmProb* p, int np, double alpha, double beta,
                   double* scratch, cudaStream_t st);

// K-major BF16 slices of one GEMM side: [nslice][rows][Kp] (slices.cu).
struct SlicedOp {
  const void* data;
  const int* exps;   // row exponents (exact slices only)
  int rows, Kp;
};
// one product for the pre-sliced tensor-core GEMMs: a = op(A) (rows M),
// b = op(B)^T (rows N); C row-major M x N
struct TcProb {
  SlicedOp a, b;
  double* C;
  int M, N, K, ldc;
};
int slice_kp(int K);
// src(row,k) = trans ? src[k*ld+row] : src[row*ld+k]; dst holds
// nslice*rows*slice_kp(K) BF16 (16-byte aligned); exps holds rows ints
int split_float(const double* src, int rows, int K, int64_t ld, int trans,
                int nslice, void* dst, cudaStream_t st);
int split_exact(const double* src, int rows, int K, int64_t ld, int trans,
                int nslice, void* dst, int* exps, cudaStream_t st);
int64_t sliced_workspace_bytes(const GemmProb* p, int np, int nslice,
                               bool exact);
int tc_gemm_sliced(const TcProb* p, int np, double alpha, double beta,
                   int nslice, double* scratch, unsigned int* d_err,
                   cudaStream_t st);
int64_t tc_sliced_scratch_doubles(const TcProb* p, int np, int nslice);
// Exact-slice GEMM on pre-sliced operands; `scratch` holds
// oz_sliced_scratch_doubles() doubles for the split-K partials (may be null
// when that is 0).
int64_t oz_sliced_scratch_doubles(const TcProb* p, int np);
int oz_gemm_sliced(const TcProb* p, int np, double alpha, double beta,
                   int nslice, double* scratch, unsigned int* d_err,
                   cudaStream_t st);

// Fused build of on-the-fly ladder rows (tc_gemm.cu): the product of
// problem i is X_gc[(a,c),(b,d)] (a of the batch, M = na*nc, N = nb*nd) and
// its element goes, cut into `ns` BF16 slices, to row a*nb + b, column
// coff + c*nd + d of the K-major slices W[ns][rows][Kp] of the batch's
// (ab|cd) rows (the B operand of the ladder product).
struct TcLadEpi {
  void* W;            // __nv_bfloat16 [ns][rows][Kp]
  int64_t rows, Kp, coff;
  int nc, nd, nb, ns;
};
int tc_gemm_ladder(const TcProb* p, int np, int nslice, const TcLadEpi* epi,
                   unsigned int* d_err, cudaStream_t st);

// Split-precision tensor-core GEMM (tc_gemm.cu): same semantics as
// gemm64_grouped, at most 8 products, nslice BF16 slices per operand (1-3).
// `workspace` holds tc_workspace_bytes() bytes of BF16 slices, `scratch`
// tc_scratch_doubles() doubles of split-K partials; *d_err becomes nonzero
// if a bounded device wait gave up.
int64_t tc_workspace_bytes(const GemmProb* p, int np, int nslice);
int64_t tc_scratch_doubles(const GemmProb* p, int np, int nslice);
int tc_gemm_grouped(const GemmProb* p, int np, double alpha, double beta,
                    int nslice, void* workspace, double* scratch,
                    unsigned int* d_err, cudaStream_t st);

// FP64-accurate tensor-core GEMM with exact integer slices (tc_ozaki.cu):
// nslice in 2..4 (4: 29 bits of every element relative to its row /
// column maximum).  `workspace` holds oz_workspace_bytes() bytes (slices,
// exponents and the split-K partials).
int64_t oz_workspace_bytes(const GemmProb* p, int np, int nslice);
int oz_gemm_grouped(const GemmProb* p, int np, double alpha, double beta,
                    int nslice, void* workspace, unsigned int* d_err,
                    cudaStream_t st);

// Y = beta*Y + alpha*s*X over the boxes described by tasks/chunks, with s
// the device scalar *d_scale (1 when d_scale is null).
int perm_axpy(const PermTask* d_tasks, const Chunk* d_chunks, int nchunks,
              double alpha, const double* X, double beta, double* Y,
              cudaStream_t st, const double* d_scale = nullptr);

// Jacobi step over DPD boxes: s = R / D (D from orbital energies),
// t += s, err = s, and atomically max |s| into *d_maxbits.
int jacobi_update(const PermTask* d_tasks, const Chunk* d_chunks, int nchunks,
                  const double* R, double* t, double* err, const double* eps,
                  unsigned long long* d_maxbits, cudaStream_t st);

// Jacobi step on a block-diagonal amplitude layout with the denominator
// separable per block, D[r,c] = rv[rv0 + r] + cv[cv0 + c] (row part: sum of
// the occupied orbital energies of the row indices, column part: minus the
// virtual ones): s = R / D, t += s (t may be null), err = s (may be null),
// atomically max |s| into *d_maxbits.  Rows are swept contiguously; each
// chunk is a run of rows of one block.
struct Block2D {
  int64_t off, ncol, rv0, cv0;
};
struct Chunk2D {
  int blk, row0, nrows;
};
int jacobi2d(const Block2D* d_blocks, const Chunk2D* d_chunks, int nchunks,
             const double* rv, const double* cv, const double* R, double* t,
             double* err, unsigned long long* d_maxbits, cudaStream_t st);

// out[k] = dot(xs[k], y) for k < m (m <= 16), deterministic two-pass.
int multi_dot(const double* const* xs, int m, const double* y, int64_t n,
              double* d_partial, double* d_out, cudaStream_t st);
int64_t multi_dot_partial_doubles(int64_t n, int m);

// out = sum_k c[k] * xs[k]  (m <= 16)
int lincomb(double* out, const double* const* xs, const double* c, int m,
            int64_t n, cudaStream_t st);

// y = a*x + b*y elementwise over n doubles
int axpby(double a, const double* x, double b, double* y, int64_t n,
          cudaStream_t st);

// g[x] = sum_e G[e] * dL[x*nnz + e] for x < nx; deterministic, uses
// `partial` (batched_dot_partial_doubles(nnz, nx) doubles).
int64_t batched_dot_partial_doubles(int64_t nnz, int nx);
int batched_dot(const double* G, const double* dL, int nx, int64_t nnz,
                double* partial, double* d_g, cudaStream_t st);

int chunk_elems();

// Metric blocks of the density-fitting form (df.cu): block b is the
// n[b] x n[b] row-major matrix at offset off[b].  metric_factor replaces M
// by its lower Cholesky factor K (upper triangle zeroed; *d_err = 1 if a
// block is not positive definite) and writes KinvT = (K^{-1})^T.
struct MetricBlocks {
  int64_t off[MAXIRR];
  int n[MAXIRR];
  int nblk;
};
int metric_factor(double* M, double* KinvT, const MetricBlocks& B,
                  unsigned int* d_err, cudaStream_t st);

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount,
// looked up once per device); grids are sized in multiples of it.
int sm_count();

// Row-batch permutation of the on-the-fly ladder (ladder.cu):
// X_gc[a][c][b][d] (blocks back to back at xoff[gc]) <-> W[(a,b)][coff[gc] +
// c*nd + d] with row length ncol.  `rows` = sum over gc of na*nc.
struct LadPerm {
  int na, nb, h;
  int nc[MAXIRR], nd[MAXIRR];
  int row0[MAXIRR + 1];
  int64_t xoff[MAXIRR], coff[MAXIRR];
  int64_t ncol;
};
int ladder_permute(const LadPerm& P, bool inverse, const double* src,
                   double* dst, int rows, cudaStream_t st);

// +/- packed ladder (ladder_pm.cu; Sec. 2.3).  Inside one DPD block of
// pair irrep G (row length ncol): orow[2][uo] the row offsets of (i,j) and
// (j,i) per canonical occupied pair, vcol[2][uv] the column offsets of
// (c,d) and (d,c) per canonical virtual pair, vrow[3][nv] per canonical
// (a,b) of a row batch its row in the batch's (ab|cd) rows W and the
// columns of (a,b) and (b,a) in Y (-1: a == b).
//   pm_pack_x: Ap/Am[r][u] = (X11 + X22 +- (X12 + X21)) / 4 of rows r1, r2
//              and columns c1, c2 (uo x uv, row-major)
//   pm_pack_w: Wp/Wm[v][u] = W[row][c1] +- W[row][c2] (c1 == c2: W, 0)
//   pm_unpack: Y[(ij),(ab)] += alpha (Sp + Sm) and the swapped elements
//              with the signs of the pair swaps (Sp, Sm: uo x nv)
int pm_pack_x(const double* X, int64_t ncol, const int* orow, int uo,
              const int* vcol, int uv, double* Ap, double* Am,
              cudaStream_t st);
int pm_pack_w(const double* W, int64_t ncol, const int* vrow, int nv,
              const int* vcol, int uv, double* Wp, double* Wm,
              cudaStream_t st);
int pm_unpack(const double* Sp, const double* Sm, int uo, int nv,
              const int* orow, const int* vrow, double alpha, double* Y,
              int64_t ncol, cudaStream_t st);

}  // namespace cdcc
