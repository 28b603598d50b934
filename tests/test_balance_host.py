"""Host logic of the persistent kernels' CTA division (paper_1301_1247_gb300/csrc/balance.hpp).

The batch of a persistent launch lasts as long as its slowest matrix, so the division of G
CTAs among nj matrices should minimise the largest modelled time max_j cost(j, nb_j) with
every nb_j >= 1 and sum nb_j = G.  A small C++ harness (compiled with the host compiler, no
GPU) checks the header against brute force over every division on small cases, for
modelled times that are non-increasing in the CTA count and for ones that are not.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1301_1247_gb300", "csrc")

HARNESS = r"""
#include "balance.hpp"
#include <cstdio>
#include <cstdint>
#include <random>
#include <vector>
using namespace hbs;

// best achievable max_j min_{b' <= b_j} cost(j, b') over all divisions (b_j >= 1, sum = G)
static double brute(int G, int nj, const std::vector<std::vector<double>>& t, std::vector<int>& b, int j, int left) {
  if (j == nj - 1) {
    b[j] = left;
    double mx = 0;
    for (int q = 0; q < nj; ++q) {
      double best = t[q][0];
      for (int c = 1; c <= b[q]; ++c) best = std::min(best, t[q][c - 1]);
      mx = std::max(mx, best);
    }
    return mx;
  }
  double res = 1e300;
  for (int c = 1; c <= left - (nj - 1 - j); ++c) {
    b[j] = c;
    res = std::min(res, brute(G, nj, t, b, j + 1, left - c));
  }
  return res;
}

int main() {
  std::mt19937 rng(7);
  int fails = 0, cases = 0;
  for (int rep = 0; rep < 400; ++rep) {
    const int nj = 1 + (int)(rng() % 4);
    const int G = nj + (int)(rng() % 9);
    const bool monotone = rep % 2 == 0;
    std::vector<std::vector<double>> t(nj, std::vector<double>(G));
    for (int j = 0; j < nj; ++j) {
      // integer-valued times: steps x ceil(work / b) + overhead, or arbitrary values
      const int steps = 1 + (int)(rng() % 50), work = 1 + (int)(rng() % 200), over = (int)(rng() % 20);
      for (int b = 1; b <= G; ++b)
        t[j][b - 1] = monotone ? (double)steps * ((work + b - 1) / b + over) : (double)(1 + rng() % 1000);
    }
    auto cost = [&](int j, int b) { return t[j][b - 1]; };
    const std::vector<int> nb = balance_ctas(G, nj, cost);
    int sum = 0;
    bool ok = (int)nb.size() == nj;
    for (int v : nb) { sum += v; ok = ok && v >= 1; }
    ok = ok && sum == G;
    double got = 0;
    for (int j = 0; j < nj && ok; ++j) {
      double best = t[j][0];
      for (int c = 1; c <= nb[j]; ++c) best = std::min(best, t[j][c - 1]);
      got = std::max(got, best);
    }
    std::vector<int> b(nj);
    const double opt = brute(G, nj, t, b, 0, G);
    ++cases;
    if (!ok || got != opt) {
      ++fails;
      std::printf("FAIL nj=%d G=%d monotone=%d got=%g opt=%g\n", nj, G, (int)monotone, got, opt);
    }
  }
  // G == nj: one CTA each
  {
    auto nb = balance_ctas(5, 5, [](int, int b) { return 100.0 / b; });
    for (int v : nb) if (v != 1) { ++fails; std::printf("FAIL G == nj\n"); break; }
  }
  std::printf("%s %d cases\n", fails ? "FAILED" : "OK", cases);
  return fails ? 1 : 0;
}
"""


def test_balance_ctas_matches_brute_force(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "balance_harness.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "balance_harness"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().startswith("OK")
