// Division of a persistent launch's CTAs among the matrices of a batch.
//
// Every matrix of a batch runs its steps behind its own barrier, so the launch lasts as
// long as its slowest matrix.  cost(j, nb) is a model of matrix j's time on nb CTAs (its
// step count times the work of the busiest warp in a step, plus a fixed per-step
// overhead).  The division minimises the largest modelled time: a binary search on the
// time bound W, each matrix taking the fewest CTAs that meet W; CTAs left over go to the
// matrices with the largest modelled time.
#pragma once

#include <algorithm>
#include <functional>
#include <vector>

namespace hbs {

inline std::vector<int> balance_ctas(int G, int nj, const std::function<double(int, int)>& cost) {
  std::vector<int> nb(nj, 1);
  if (nj <= 0 || G <= nj) return nb;
  const int cap = G - nj + 1;  // most CTAs one matrix can take
  // t[j][b - 1]: modelled time on b CTAs, made non-increasing in b (more CTAs never hurt)
  std::vector<std::vector<double>> t(nj, std::vector<double>(cap));
  double hi = 0.0, lo = 0.0;
  for (int j = 0; j < nj; ++j) {
    double run = cost(j, 1);
    for (int b = 1; b <= cap; ++b) {
      run = std::min(run, cost(j, b));
      t[j][b - 1] = run;
    }
    hi = std::max(hi, t[j][0]);
    lo = std::max(lo, t[j][cap - 1]);
  }
  auto need = [&](int j, double W) {  // fewest CTAs with time <= W (cap if none)
    const auto& v = t[j];
    const auto it = std::lower_bound(v.begin(), v.end(), W, [](double a, double w) { return a > w; });
    return it == v.end() ? cap : (int)(it - v.begin()) + 1;
  };
  for (int iter = 0; iter < 60 && hi - lo > 1e-9 * hi; ++iter) {
    const double W = 0.5 * (lo + hi);
    long long tot = 0;
    for (int j = 0; j < nj; ++j) tot += need(j, W);
    (tot <= G ? hi : lo) = W;
  }
  int used = 0;
  for (int j = 0; j < nj; ++j) used += (nb[j] = need(j, hi));
  while (used > G) {  // guard against rounding in the search
    int jm = -1;
    for (int j = 0; j < nj; ++j)
      if (nb[j] > 1 && (jm < 0 || t[j][nb[j] - 2] < t[jm][nb[jm] - 2])) jm = j;
    if (jm < 0) break;
    --nb[jm];
    --used;
  }
  while (used < G) {
    int jm = 0;
    for (int j = 1; j < nj; ++j)
      if (t[j][nb[j] - 1] > t[jm][nb[jm] - 1]) jm = j;
    ++nb[jm];
    ++used;
  }
  return nb;
}

}  // namespace hbs
