"""The multiply-high division of the general sweep kernels (FastDiv in
csrc/internal.h, Granlund & Montgomery 1994, Fig. 4.1) against the hardware
division, on the host: a small program compiled by nvcc (no GPU needed)
divides by every d < 70000 and by random d up to 2^32 - 1, for small,
random, multiple-boundary and maximal 32-bit dividends."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include "internal.h"
using namespace pf;
static uint64_t state = 88172645463325252ull;
static uint32_t next32() { state ^= state << 13; state ^= state >> 7; state ^= state << 17; return (uint32_t)(state >> 16); }
static long bad = 0, checks = 0;
static void check(uint32_t n, const FastDiv& f) {
  checks++;
  if (fdiv(n, f) != n / f.d) { if (bad < 5) std::printf("d=%u n=%u got %u\n", f.d, n, fdiv(n, f)); bad++; }
}
int main() {
  for (uint32_t d = 1; d < 70000; d++) {
    const FastDiv f = make_fastdiv(d);
    for (uint32_t n = 0; n < 2048; n++) check(n, f);
    for (int k = 0; k < 64; k++) check(next32(), f);
    for (uint64_t q = 1; q < 40; q++) {
      const uint64_t n = q * d;
      if (n < (1ull << 32)) { check((uint32_t)n, f); check((uint32_t)(n - 1), f); }
    }
    check(0xffffffffu, f);
  }
  for (int k = 0; k < 200000; k++) {
    uint32_t d = next32() >> (next32() % 32);
    if (d == 0) d = 1;
    const FastDiv f = make_fastdiv(d);
    check(next32(), f);
    check(0xffffffffu, f);
    check(d, f);
    check(d - 1, f);
  }
  std::printf("checks %ld bad %ld\n", checks, bad);
  return bad != 0;
}
"""


def _nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return exe if os.path.exists(exe) else None


def test_fastdiv_matches_hardware_division(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "fastdiv_check.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "fastdiv_check"
    inc = os.path.join(ROOT, "paper_1409_8116_gb300", "csrc")
    build = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", inc, str(src), "-o", str(exe)],
                           capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-2000:]
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stdout[-2000:]
    assert "bad 0" in run.stdout
