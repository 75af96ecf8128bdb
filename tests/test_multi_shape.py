"""Host-side choice of the slice ranges per system of the multi-system walk launch
(csrc/multi_shape.h), compiled on its own with the host C++ compiler: no GPU.

Each case is worked by hand from the launch's cost, ceil(nsys G / R) rounds of
2 ceil(Ntau / G) + 1 sweeps for G ranges per system and R resident CTAs."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2508_16298_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "multi_shape.h"
using namespace hqmc;
int main() {
  int bad = 0;
  auto expect = [&](int got, int want, const char* what) {
    if (got != want) { std::printf("%s: got %d want %d\n", what, got, want); ++bad; }
  };
  // L = 66: one CTA per SM on 152 SMs.  40 systems: 19 ranges of 34-35 slices, five
  // rounds of 71 sweeps (355); 20 ranges need six rounds of 67 (402), 38 ranges ten of
  // 37 (370), 15 ranges four of 89 (356).
  expect(multi_ranges_model(660, 40, 152), 19, "L=66, 40 systems");
  // one system: a single round whatever G <= 152; 132..152 ranges all give 11 sweeps,
  // the largest is kept (the split of the one-system launch)
  expect(multi_ranges_model(660, 1, 152), 152, "L=66, one system");
  // small lattices with many resident CTAs: one slice per CTA in one round (3 sweeps)
  expect(multi_ranges_model(40, 5, 4864), 40, "L=8, 5 systems");
  expect(multi_ranges_model(70, 5, 4864), 70, "L=10, 5 systems");
  // one resident CTA: all work serial, nsys G (2 ceil(N/G) + 1) is least at G = 1
  expect(multi_ranges_model(12, 3, 1), 1, "one resident CTA");
  // degenerate inputs stay in range
  expect(multi_ranges_model(1, 7, 152), 1, "one slice");
  // nsys and resident clamped to 1: G = 1 is one round of 13 sweeps, G = 6 six rounds of 3 (18)
  expect(multi_ranges_model(6, 0, 0), 1, "clamped inputs");
  return bad;
}
"""


def test_multi_ranges_model(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "multi_shape.cpp"
    exe = tmp_path / "multi_shape"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True, capture_output=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout
