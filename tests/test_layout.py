"""The tiled rotated window's row map (h_row in csrc/common.cuh), checked on
the host: a small program built from the library's own header with nvcc and
run on the CPU (no GPU).  In pq order the row of (p, q) is p*p + p + q.  The
FP32 window of L_h > 16 is stored order-major: for every band limit the map
must be a permutation of the L_h^2 rows in which each order's degrees
p = |q| .. L_h - 1 form one contiguous, increasing run, the runs following
each other in order q = -(L_h - 1) .. L_h - 1; the wide engine's first pass
reads a run chunk by chunk with one bulk copy, so a gap or an overlap would
read another order's rows."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1207_5558_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "common.cuh"
int main() {
  for (int Lh = 1; Lh <= SLSHT_MAX_LH; ++Lh) {
    const int n2 = Lh * Lh;
    std::vector<int> seen(n2, 0);
    int next = 0;                                   // where the next order's run must start
    for (int q = -(Lh - 1); q <= Lh - 1; ++q) {
      const int a = q < 0 ? -q : q;
      for (int p = a; p < Lh; ++p) {
        const int r = h_row(p, q, Lh, true);
        if (r != next + (p - a)) { std::printf("run Lh=%d p=%d q=%d row=%d\n", Lh, p, q, r); return 1; }
        if (r < 0 || r >= n2 || seen[r]++) { std::printf("perm Lh=%d p=%d q=%d row=%d\n", Lh, p, q, r); return 1; }
        if (h_row(p, q, Lh, false) != p * p + p + q) { std::printf("pq Lh=%d p=%d q=%d\n", Lh, p, q); return 1; }
      }
      next += Lh - a;
    }
    if (next != n2) { std::printf("count Lh=%d\n", Lh); return 1; }
    if (h_order_major(Lh) != (Lh > 16)) { std::printf("rule Lh=%d\n", Lh); return 1; }
  }
  std::printf("ok\n");
  return 0;
}
"""


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_order_major_rows_are_contiguous_runs_of_a_permutation(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "rows.cu"
    exe = tmp_path / "rows"
    src.write_text(PROGRAM)
    build = subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)],
                           capture_output=True, text=True)
    assert build.returncode == 0, build.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0 and run.stdout.strip() == "ok", run.stdout + run.stderr
