"""Host logic of the dynamically scheduled launches: the row-chunk height
rule (`dyn_chunk_rows` in csrc/lbm_internal.cuh), compiled as host code and
checked for its invariants over a grid of box shapes, and for the heights
the step and two-component launchers take on the measured boxes. No GPU is
needed (nvcc compiles the host program; the test is skipped without it)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1708_01613_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "lbm_internal.cuh"
using lbm::dyn_chunk_rows;
static long long items(long long gx, long long ny, int rows) { return gx * ((ny + rows - 1) / rows); }
int main() {
  long long bad = 0, cases = 0;
  const int res_list[] = {152, 456, 608};
  for (int gx = 1; gx <= 40; ++gx)
    for (int ny = 4; ny <= 20000; ny += (ny < 200 ? 1 : 97))
      for (int res : res_list)
        for (int keep : {4, 8})
          for (int minw : {1, 4}) {
            ++cases;
            const int r = dyn_chunk_rows(gx, ny, res, 48, keep, minw);
            const long long i48 = items(gx, ny, 48);
            bool ok = r >= 1 && r <= 48;
            if (i48 >= (long long)keep * res) {
              ok = ok && r == 48;
            } else {
              long long waves = (i48 + res - 1) / res;
              if (i48 > res && waves < minw) waves = minw;
              // the chunks fill at most the chosen whole number of waves
              ok = ok && items(gx, ny, r) <= waves * res;
              // and the height is the smallest that does (one row less overflows)
              ok = ok && (r == 1 || items(gx, ny, r - 1) > waves * res ||
                          (ny + r - 2) / (r - 1) == (ny + r - 1) / r);
            }
            if (!ok && bad++ < 5)
              printf("violation gx=%d ny=%d res=%d keep=%d minw=%d rows=%d\n", gx, ny, res, keep, minw, r);
          }
  // heights the launchers take on the measured boxes (one component: 512-column
  // strips, 4 waves kept, fewest waves for 16-bit storage at 608 CTAs, at
  // least four for FP32 at 456; two components: 256-column strips, 8 waves
  // kept, at least four, 456 CTAs)
  printf("f16 4096 %d\n", dyn_chunk_rows(8, 4096, 608, 48, 4, 1));
  printf("f16 5120 %d\n", dyn_chunk_rows(10, 5120, 608, 48, 4, 1));
  printf("f16 6144 %d\n", dyn_chunk_rows(12, 6144, 608, 48, 4, 1));
  printf("f16 6144x3072 %d\n", dyn_chunk_rows(12, 3072, 608, 48, 4, 1));
  printf("f16 8192 %d\n", dyn_chunk_rows(16, 8192, 608, 48, 4, 1));
  printf("f32 4096 %d\n", dyn_chunk_rows(8, 4096, 456, 48, 4, 4));
  printf("f32 5120 %d\n", dyn_chunk_rows(10, 5120, 456, 48, 4, 4));
  printf("f32 6144 %d\n", dyn_chunk_rows(12, 6144, 456, 48, 4, 4));
  printf("f32 8192 %d\n", dyn_chunk_rows(16, 8192, 456, 48, 4, 4));
  printf("2c 3072 %d\n", dyn_chunk_rows(12, 3072, 456, 48, 8, 4));
  printf("2c 4096 %d\n", dyn_chunk_rows(16, 4096, 456, 48, 8, 4));
  printf("2c 6144 %d\n", dyn_chunk_rows(24, 6144, 456, 48, 8, 4));
  printf("2c 8192 %d\n", dyn_chunk_rows(32, 8192, 456, 48, 8, 4));
  printf("cases %lld violations %lld\n", cases, bad);
  return bad != 0;
}
"""

EXPECTED = {
    "f16 4096": 27, "f16 5120": 43, "f16 6144": 41, "f16 6144x3072": 31, "f16 8192": 48,
    "f32 4096": 18, "f32 5120": 29, "f32 6144": 41, "f32 8192": 48,
    "2c 3072": 21, "2c 4096": 36, "2c 6144": 47, "2c 8192": 48,
}


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_chunk_height_rule(tmp_path):
    cc = nvcc()
    if not cc:
        pytest.skip("nvcc not available")
    src = tmp_path / "chunk_rule.cu"
    exe = tmp_path / "chunk_rule"
    src.write_text(PROGRAM)
    r = subprocess.run([cc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    lines = dict(l.rsplit(" ", 1) for l in out.stdout.splitlines() if not l.startswith(("violation", "cases")))
    assert out.returncode == 0, out.stdout
    got = {k: int(v) for k, v in lines.items()}
    assert got == EXPECTED, got
