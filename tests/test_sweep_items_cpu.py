"""The tensor-core sweep's work decomposition, checked on the host.

`csrc/sweep_items.cuh` holds the functions the update kernel uses to count
its work items, decode them (directly, or with the cursor of a persistent
CTA that takes items in increasing order) and skip tiles.  This test
compiles them into a small host program with nvcc and checks, for every
sweep step of a range of sizes, item widths and grids, that the look-ahead
and bulk launches (Hermitian sweep) or the single launch (general sweep)
cover each tile the step must update exactly once, no other tile, and never
more than kJPI tiles per item (the kernel's per-item tile array).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1111_4429_gb300", "csrc")

CHECK = r'''
#include <cstdio>
#include <vector>
#include "sweep_items.cuh"
using namespace bgw::oz;

static const int NB = 32;   // sweep block width
static long long g_errors = 0, g_tiles = 0;

static void fail(const char* what, int ng, int k0, int wide, int grid, int I, int J) {
  if (g_errors++ < 20) std::printf("%s: ng %d k0 %d wide %d grid %d tile (%d, %d)\n", what, ng, k0, wide, grid, I, J);
}

// one launch of `mode` on `grid` CTAs (a CTA takes items b, b + grid, ...)
static void launch(int mode, int wide, int grid, int ng, int k0, std::vector<int>& count) {
  const int kb = imin(NB, ng - k0);
  const int nI = (ng + BM - 1) / BM, nJ = (ng + BN - 1) / BN;
  const int k1 = k0 + NB;
  const bool has_next = k1 < ng;
  const int In = k1 / BM, Jn = k1 / BN;
  const int n = pipe_items(mode, wide, nI, nJ, In, has_next);
  for (int b = 0; b < grid; ++b) {
    PipeCursor cur;
    for (int item = b; item < n; item += grid) {
      int I, J0, J1, I2, J02, J12;
      pipe_decode(mode, wide, item, nI, nJ, In, Jn, has_next, I, J0, J1);
      pipe_decode_next(cur, mode, wide, item, nI, nJ, In, Jn, has_next, I2, J02, J12);
      if (I != I2 || J0 != J02 || J1 != J12) fail("cursor decode differs", ng, k0, wide, grid, I, J0);
      if (I < 0 || I >= nI || J0 < 0 || J1 <= J0 || J1 > nJ) { fail("item out of range", ng, k0, wide, grid, I, J0); continue; }
      if (J1 - J0 > kJPI || J1 - J0 > pipe_jpi(mode, wide)) fail("item too wide", ng, k0, wide, grid, I, J0);
      for (int J = J0; J < J1; ++J)
        if (!pipe_skip(mode, item, I, J, ng, k0, kb, In, Jn, has_next)) ++count[I * nJ + J];
    }
  }
}

static void step(bool general, int ng, int k0, int wide, int grid) {
  const int kb = imin(NB, ng - k0);
  const int nI = (ng + BM - 1) / BM, nJ = (ng + BN - 1) / BN;
  const int k1 = k0 + NB;
  const bool has_next = k1 < ng;
  const int In = k1 / BM;
  std::vector<int> count(nI * nJ, 0);
  if (general) {
    launch(3, wide, grid, ng, k0, count);
  } else {
    if (has_next) launch(1, wide, pipe_items(1, wide, nI, nJ, In, true), ng, k0, count);
    launch(2, wide, grid, ng, k0, count);
  }
  for (int I = 0; I < nI; ++I)
    for (int J = 0; J < nJ; ++J) {
      const int i0 = I * BM, j0 = J * BN;
      const bool in_pivot_rows = i0 >= k0 && imin(i0 + BM, ng) <= k0 + kb;
      const bool in_pivot_cols = j0 >= k0 && imin(j0 + BN, ng) <= k0 + kb;
      const bool want = (general ? true : J < 4 * I + 4) && j0 < ng && !in_pivot_rows &&
                        (general || !in_pivot_cols);
      const int c = count[I * nJ + J];
      if (c != (want ? 1 : 0)) fail(c > 1 ? "tile updated twice" : (want ? "tile missed" : "tile not owned"),
                                    ng, k0, wide, grid, I, J);
      g_tiles += c;
    }
}

int main() {
  const int sizes[] = {1, 2, 31, 32, 33, 63, 64, 85, 127, 128, 129, 151, 160, 255, 256, 257, 300, 743, 1185,
                       2104, 2120, 2545, 3911};
  const int widths[] = {2, 3, 4};
  for (int ng : sizes)
    for (int wide : widths)
      for (int general = 0; general < 2; ++general) {
        for (int k0 = 0; k0 < ng; k0 += NB) {
          const int nI = (ng + BM - 1) / BM, nJ = (ng + BN - 1) / BN;
          const int k1 = k0 + NB;
          const int n = pipe_items(general ? 3 : 2, wide, nI, nJ, k1 / BM, k1 < ng);
          const int grids[] = {n > 0 ? n : 1, 1, 7, 152, n + 5};
          for (int grid : grids) step(general != 0, ng, k0, wide, grid);
        }
      }
  std::printf("tiles %lld errors %lld\n", g_tiles, g_errors);
  return g_errors ? 1 : 0;
}
'''


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_update_items_cover_each_tile_once(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "items_check.cu"
    exe = tmp_path / "items_check"
    src.write_text(CHECK)
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                        f"-I{CSRC}", str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "errors 0" in r.stdout
