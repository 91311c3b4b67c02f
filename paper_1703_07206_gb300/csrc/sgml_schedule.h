// sgml_schedule.h -- host-side phase table of one cycle (Algorithm 3's saw-like schedule) and the
// choice of the CTA that runs the coarse tail; used by sgml_api.cu, checked on the CPU by
// tests/native/schedule_check.cpp.
#pragma once
#include <algorithm>
#include <vector>

#include "sgml_internal.cuh"

namespace sgml {

// Phase table of one cycle (Algorithm 3) for the deepest problem of the batch; shallower problems
// follow its suffix.  On levels below pair_levels the sweeps of a visit run two at a time (kPair; a
// visit with an odd number of sweeps ends with a single one).
inline std::vector<Phase> build_phases(int n_max, int n_r, int pair_levels, bool any_eq10, bool tail = false) {
  std::vector<Phase> ph;
  for (int l = 1; l <= n_max - 1; ++l) ph.push_back(Phase{OP_RESTRICT, l, l - 1, 0, 0, 0});
  struct Visit {
    int level, tooth, first, final_visit;
  };
  std::vector<Visit> vs;
  for (int nu1 = n_max - 1; nu1 >= 1; --nu1) {
    vs.push_back({nu1, nu1, 1, 0});
    vs.push_back({nu1 - 1, nu1, 0, 0});
    vs.push_back({nu1, nu1, 0, 0});
  }
  vs.push_back({0, 0, 1, 1});  // tooth 0 (two level-0 visits) merged with the final level-0 visit
  for (size_t q = 0; q < vs.size(); ++q) {
    const Visit& v = vs[q];
    if (q > 0) {
      const Visit& u = vs[q - 1];
      if (v.level == u.level - 1) {
        const bool init = v.tooth == u.tooth;
        ph.push_back(Phase{OP_PROLONG, v.level, u.tooth, 0, init ? kInit : 0, v.level + 1});
      } else if (v.level == u.level + 1) {
        ph.push_back(Phase{OP_INJECT, v.level, u.tooth, 0, 0, 0});
      }
    }
    const int e = n_max - v.tooth;
    const int k = std::min<long long>(n_r, 1LL << std::min(e, 30));
    const int kk = v.final_visit ? 3 * k : k;
    const int flags = (v.final_visit ? kFinalVisit : 0) | (v.first ? kFirstOfTooth : 0);
    const int step = v.level < pair_levels ? 2 : 1;
    for (int s = 0; s < kk; s += step)
      ph.push_back(Phase{OP_SWEEP, v.level, v.tooth, s, flags | (step == 2 && s + 1 < kk ? kPair : 0), 0});
  }
  if (any_eq10) {  // Eq. 10: project the constant mode out of u after the cycle
    ph.push_back(Phase{OP_MEAN_ROWS, 0, 0, 0, 0, 0});
    ph.push_back(Phase{OP_MEAN_REDUCE, 0, 0, 0, 0, 0});
    ph.push_back(Phase{OP_MEAN_APPLY, 0, 0, 0, 0, 0});
  }
  if (tail) {  // coarse tail: from the restriction into level n - 3 up to the first phase below it
    const int lt = n_max - 3;
    auto lowest = [](const Phase& f) {  // lowest level a phase reads or writes
      if (f.op == OP_RESTRICT || f.op == OP_INJECT) return f.level - 1;
      if (f.op == OP_SWEEP || f.op == OP_PROLONG) return f.level;
      return 0;
    };
    for (size_t q0 = 0; q0 < ph.size(); ++q0)
      if (ph[q0].op == OP_RESTRICT && ph[q0].level == lt) {
        size_t q1 = q0 + 1;
        while (q1 < ph.size() && lowest(ph[q1]) >= lt) ++q1;
        ph[q0].flags |= kTailStart;
        ph[q0].prev_tooth = (int)q1;
        break;
      }
  }
  return ph;
}

// The CTA that runs the coarse tail: the last one without tiles on the levels around it (n - 5 ..
// n - 1), so that its SM's instruction cache, which the tail's code displaces, is not needed by the
// grid phases right after the tail; CTA 0 if every CTA has some.  toff: the partition's task offsets,
// kMaxLevels x (G + 1).
inline int pick_tail_cta(const std::vector<int>& toff, int G, int n_max) {
  for (int c = G - 1; c >= 0 && n_max >= 4; --c) {
    bool idle = true;
    for (int l = std::max(0, n_max - 5); l <= n_max - 1; ++l)
      idle = idle && toff[(size_t)l * (G + 1) + c + 1] == toff[(size_t)l * (G + 1) + c];
    if (idle) return c;
  }
  return 0;
}

}  // namespace sgml
