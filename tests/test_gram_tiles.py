"""Host check of the tensor-core Gram's tile order (csrc/gram_tc.cu,
gram_tile): for every tile count and band height the launch's CTA indices
map one to one onto the upper-triangle tiles (bi <= bj), and a band of one
row is the plain row-major order.  The Gram of Algorithm 1 (T <- X^T X) is
symmetric, so each upper-triangle tile must be computed exactly once for
S to be complete.  The function is host-and-device code; this test builds
a small host program around it with nvcc (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2106_09382_gb300", "csrc")

PROGRAM = r"""
#include "gram_tc.cu"
#include <cstdio>
#include <vector>
namespace concord { void note_launches(unsigned) {} }
int main() {
  for (int nbt = 1; nbt <= 170; ++nbt)
    for (int g = 1; g <= 24; ++g) {
      const int tiles = nbt * (nbt + 1) / 2;
      std::vector<int> seen((size_t)nbt * nbt, 0);
      int pi = -1, pj = -1;
      for (int t = 0; t < tiles; ++t) {
        int bi = -1, bj = -1;
        concord::gram_tile(t, nbt, g, bi, bj);
        if (bi < 0 || bj < bi || bj >= nbt) { printf("out of range %d %d %d\n", nbt, g, t); return 1; }
        seen[(size_t)bi * nbt + bj]++;
        if (g == 1 && !(bi > pi || (bi == pi && bj == pj + 1))) { printf("order %d\n", t); return 1; }
        pi = bi; pj = bj;
      }
      for (int i = 0; i < nbt; ++i)
        for (int j = i; j < nbt; ++j)
          if (seen[(size_t)i * nbt + j] != 1) { printf("tile %d %d of %d %d\n", i, j, nbt, g); return 1; }
    }
  printf("ok\n");
  return 0;
}
"""


def test_gram_tile_order_covers_the_upper_triangle_once(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "tiles.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "tiles"
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1",
                        "-I" + CSRC, "-I" + os.path.join(ROOT, "include"),
                        "-o", str(exe), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
