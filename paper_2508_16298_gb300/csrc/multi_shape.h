// Slice ranges per system of the multi-system tau-walking M^dagger M launch
// (plain C++: the host-only test compiles this header alone).
#pragma once

namespace hqmc {

// nsys systems of Ntau slices each share one launch; `resident` CTAs of the walk
// kernel fit on the device at once.  A CTA walking a range of n slices runs
// 2n + 1 sweeps (one halo sweep), so with G ranges per system the launch takes
// about ceil(nsys G / resident) rounds of the longest range, 2 ceil(Ntau / G) + 1
// sweeps each.  Returns the G in [1, Ntau] with the fewest sweeps over all rounds,
// the largest G among equals (more, shorter ranges leave less idle at the end).
inline int multi_ranges_model(int Ntau, int nsys, long long resident) {
  if (Ntau < 1) return 1;
  if (nsys < 1) nsys = 1;
  if (resident < 1) resident = 1;
  long long best = -1;
  int bestG = 1;
  for (int G = 1; G <= Ntau; ++G) {
    const long long rounds = ((long long)nsys * G + resident - 1) / resident;
    const long long cost = rounds * (2LL * ((Ntau + G - 1) / G) + 1);
    if (best < 0 || cost <= best) {
      best = cost;
      bestG = G;
    }
  }
  return bestG;
}

}  // namespace hqmc
