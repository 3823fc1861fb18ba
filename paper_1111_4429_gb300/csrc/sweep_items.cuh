// Work items of the tensor-core sweep's update launches, shared by the
// kernel (sweep_tc.cu) and host code: the tiles a launch covers at one sweep
// step, how they are grouped into items and which tiles an item skips.
//
// A matrix is cut into row tiles of BM rows and column tiles of BN columns;
// the Hermitian sweep updates the tiles (I, J) with J < 4 I + 4 (the lower
// triangle at tile granularity), the general Gauss-Jordan sweep every tile.
// At step k0 the tiles inside the pivot block's rows or columns are left to
// the step itself.
#pragma once

namespace bgw {
namespace oz {

constexpr int BM = 128;   // tile rows (i)
constexpr int BN = 32;    // tile cols (j)
constexpr int kJPI = 4;   // most column tiles per work item (see pipe_jpi)

__host__ __device__ inline int imin(int a, int b) { return a < b ? a : b; }

__host__ __device__ inline int row_width(int mode, int I, int nJ) { return mode == 3 ? nJ : imin(4 * I + 4, nJ); }

// Number of work items of a mode, and the decode of one.  Mode 1 starts with
// the tile holding the next diagonal block alone (its CTA sweeps that block:
// the critical path of the next step), then the rest of row tile In in
// chunks (tile Jn skipped there), then the tiles (I > In, Jn).
// Column tiles per work item: 2 in the look-ahead launch (its CTAs are on the
// critical path); else the launch's width (oz_update picks it: 4 with seven
// slices, 3 with five, 2 where those would number no more than the SMs or
// where the plan fixes it).
__host__ __device__ inline int pipe_jpi(int mode, int wide) { return mode == 1 ? 2 : wide; }
__host__ __device__ inline int pipe_items(int mode, int wide, int nI, int nJ, int In, bool has_next) {
  int n = 0;
  const int jpi = pipe_jpi(mode, wide);
  if (mode == 1) {
    const int w = (4 * In + 4 < nJ) ? 4 * In + 4 : nJ;
    return 1 + (w + jpi - 1) / jpi + (nI - In - 1 > 0 ? nI - In - 1 : 0);
  }
  for (int I = 0; I < nI; ++I) {
    if (mode == 2 && has_next && I == In) continue;
    const int w = mode == 3 ? nJ : ((4 * I + 4 < nJ) ? 4 * I + 4 : nJ);
    n += (w + jpi - 1) / jpi;
  }
  return n;
}
__host__ __device__ inline void pipe_decode(int mode, int wide, int item, int nI, int nJ, int In, int Jn, bool has_next, int& I, int& J0,
                                   int& J1) {
  const int jpi = pipe_jpi(mode, wide);
  if (mode == 1) {
    const int w = row_width(1, In, nJ);
    const int nrow = (w + jpi - 1) / jpi;
    if (item == 0) {
      I = In;
      J0 = Jn;
      J1 = Jn + 1;
    } else if (item <= nrow) {
      I = In;
      J0 = (item - 1) * jpi;
      J1 = imin(J0 + jpi, w);
    } else {
      I = In + 1 + (item - 1 - nrow);
      J0 = Jn;
      J1 = Jn + 1;
    }
    return;
  }
  for (I = 0; I < nI; ++I) {
    if (mode == 2 && has_next && I == In) continue;
    const int w = row_width(mode, I, nJ);
    const int n = (w + jpi - 1) / jpi;
    if (item < n) {
      J0 = item * jpi;
      J1 = imin(J0 + jpi, w);
      return;
    }
    item -= n;
  }
  J0 = J1 = 0;
}
// The same decode for a CTA that takes its items in increasing order: the
// cursor keeps the row tile reached and its first item, so a persistent CTA
// walks the rows once in all instead of once per item.
struct PipeCursor {
  int I = 0, base = 0;
};
__host__ __device__ inline void pipe_decode_next(PipeCursor& cur, int mode, int wide, int item, int nI, int nJ, int In, int Jn,
                                        bool has_next, int& I, int& J0, int& J1) {
  if (mode == 1) {
    pipe_decode(mode, wide, item, nI, nJ, In, Jn, has_next, I, J0, J1);
    return;
  }
  const int jpi = pipe_jpi(mode, wide);
  for (; cur.I < nI; ++cur.I) {
    const int w = row_width(mode, cur.I, nJ);
    const int n = (mode == 2 && has_next && cur.I == In) ? 0 : (w + jpi - 1) / jpi;
    if (item < cur.base + n) {
      I = cur.I;
      J0 = (item - cur.base) * jpi;
      J1 = imin(J0 + jpi, w);
      return;
    }
    cur.base += n;
  }
  I = nI;
  J0 = J1 = 0;
}
__host__ __device__ inline bool pipe_skip(int mode, int item, int I, int J, int ng, int k0, int kb, int In, int Jn,
                                 bool has_next) {
  const int i0 = I * BM, j0 = J * BN;
  if (j0 >= ng) return true;
  if (mode == 2 && has_next && J == Jn) return true;
  if (mode == 1 && item > 0 && I == In && J == Jn) return true;   // done by item 0
  if (i0 >= k0 && imin(i0 + BM, ng) <= k0 + kb) return true;
  if (mode != 3 && j0 >= k0 && imin(j0 + BN, ng) <= k0 + kb) return true;
  return false;
}

}  // namespace oz
}  // namespace bgw
