// dpd.cpp -- host-side DPD layout arithmetic (see dpd.h).
#include "dpd.h"

#include <sstream>
#include <stdexcept>

namespace cdcc {

static int ipow(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

void Layout::build(const Dims& d) {
  h = d.h;
  const int r = split, c = rank - split;
  ncode_r = r >= 2 ? ipow(h, r - 1) : 1;
  ncode_c = c >= 2 ? ipow(h, c - 1) : 1;
  rsub.assign(MAXIRR * ncode_r, 0);
  csub.assign(MAXIRR * ncode_c, 0);
  auto group = [&](int q0, int m, int G, int64_t* sub, int64_t& total) {
    total = 0;
    if (m == 0) {
      total = (G == 0) ? 1 : 0;
      return;
    }
    const int ncode = m >= 2 ? ipow(h, m - 1) : 1;
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
      for (int q = 0; q < m; ++q) cnt *= d.n[sp[q0 + q]][g[q]];
      sub[code] = total;
      total += cnt;
    }
  };
  size = 0;
  for (int G = 0; G < MAXIRR; ++G) {
    nrow[G] = ncol[G] = 0;
    blk_off[G] = size;
  }
  for (int G = 0; G < h; ++G) {
    const int Gc = G ^ gtot;
    group(0, r, G, &rsub[G * ncode_r], nrow[G]);
    group(r, c, Gc, &csub[Gc * ncode_c], ncol[G]);
    blk_off[G] = size;
    size += nrow[G] * ncol[G];
  }
}

std::string Layout::key() const {
  std::ostringstream os;
  os << rank << ':' << gtot << ':' << split << ':';
  for (int q = 0; q < rank; ++q) os << sp[q];
  return os.str();
}

SubBlock sub_block(const Layout& L, const Dims& d, const int* g) {
  SubBlock s{};
  int G = 0;
  for (int q = 0; q < L.split; ++q) G ^= g[q];
  const int Gc = G ^ L.gtot;
  int code_r = 0, code_c = 0;
  for (int q = 0; q < L.split - 1; ++q) code_r = code_r * L.h + g[q];
  for (int q = L.split; q < L.rank - 1; ++q) code_c = code_c * L.h + g[q];
  const int64_t rowoff = L.split > 0 ? L.rsub[G * L.ncode_r + code_r] : 0;
  const int64_t coloff =
      L.rank - L.split > 0 ? L.csub[Gc * L.ncode_c + code_c] : 0;
  s.base = L.blk_off[G] + rowoff * L.ncol[G] + coloff;
  s.empty = false;
  int64_t st = 1;
  for (int q = L.rank - 1; q >= L.split; --q) {
    s.stride[q] = st;
    s.dim[q] = d.n[L.sp[q]][g[q]];
    st *= s.dim[q];
  }
  st = L.ncol[G];
  for (int q = L.split - 1; q >= 0; --q) {
    s.stride[q] = st;
    s.dim[q] = d.n[L.sp[q]][g[q]];
    st *= s.dim[q];
  }
  for (int q = 0; q < L.rank; ++q)
    if (s.dim[q] == 0) s.empty = true;
  return s;
}

void for_each_tuple(int h, int rank, int gtot,
                    const std::function<void(const int*)>& f) {
  int g[MAXRANK] = {0, 0, 0, 0};
  if (rank == 0) {
    if (gtot == 0) f(g);
    return;
  }
  const int ncode = ipow(h, rank - 1);
  for (int code = 0; code < ncode; ++code) {
    int x = gtot, cc = code;
    for (int q = rank - 2; q >= 0; --q) {
      g[q] = cc % h;
      cc /= h;
      x ^= g[q];
    }
    g[rank - 1] = x;
    f(g);
  }
}

}  // namespace cdcc
