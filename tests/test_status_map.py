"""Host-side mapping of the device CG loop's outcome to the C ABI's status codes
(csrc/status.h), compiled on its own with the host C++ compiler: no GPU, and no
run that makes a device-side wait time out.  A timed-out wait poisons its
kernel's outputs with NaN, so the loop ends as non-finite; the solve must report
the cause, HQMC_ETIMEOUT, not the symptom."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2508_16298_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

PROGRAM = r"""
#include <cstdio>
#include "status.h"
using namespace hqmc;
int main() {
  int bad = 0;
  auto expect = [&](int got, int want, const char* what) {
    if (got != want) { std::printf("%s: got %d want %d\n", what, got, want); ++bad; }
  };
  expect(solve_status(CG_CONVERGED, false), HQMC_OK, "converged");
  expect(solve_status(CG_MAXIT, false), HQMC_ENOTCONV, "maxit");
  expect(solve_status(CG_STAGNATED, false), HQMC_ENOTCONV, "stagnated");
  expect(solve_status(CG_BREAKDOWN, false), HQMC_EBREAKDOWN, "breakdown");
  expect(solve_status(CG_NONFINITE, false), HQMC_ENONFINITE, "nonfinite");
  const int states[] = {CG_RUNNING, CG_CONVERGED, CG_MAXIT, CG_BREAKDOWN, CG_NONFINITE, CG_REC_CONVERGED, CG_STAGNATED};
  for (int d : states) expect(solve_status(d, true), HQMC_ETIMEOUT, "timed out");
  return bad;
}
"""


def test_solve_status_mapping(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "status_map.cpp"
    exe = tmp_path / "status_map"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-std=c++17", "-I", CSRC, "-I", INCLUDE, str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout
