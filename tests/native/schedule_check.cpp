// Host-side check of the cycle's phase table (sgml_schedule.h).  Prints one line per case:
//   phases n n_r pair eq10 same_with_tail starts q0_op q0_level tail_len inner_ok boundary_ok
// where same_with_tail: the table with the coarse tail marked equals the plain one except for the
// start phase's flag and end index; starts: phases carrying kTailStart; inner_ok: every phase inside
// the tail touches only levels >= n - 3; boundary_ok: the phase after the tail touches a lower level.
// Then the sweep sequence of the 33^2 (n = 5, n_r = 2) cycle as "visits level:sweeps ...", and
//   tailcta dim n G tile_x cta idle_ok last_ok
// for the CTA picked to run the coarse tail on real partitions.
#include <cstdio>
#include <vector>

#include "sgml_schedule.h"
#include "sgml_tasks.h"

using namespace sgml;

static int lowest(const Phase& f) {
  if (f.op == OP_RESTRICT || f.op == OP_INJECT) return f.level - 1;
  if (f.op == OP_SWEEP || f.op == OP_PROLONG) return f.level;
  return 0;
}

int main() {
  for (int n = 2; n <= 12; ++n)
    for (int n_r = 1; n_r <= 3; ++n_r)
      for (int pair = 0; pair <= 1; ++pair)
        for (int eq10 = 0; eq10 <= 1; ++eq10) {
          const std::vector<Phase> a = build_phases(n, n_r, pair, eq10 != 0, false);
          const std::vector<Phase> b = build_phases(n, n_r, pair, eq10 != 0, n >= 4);
          bool same = a.size() == b.size();
          int starts = 0, q0 = -1, q1 = -1;
          for (size_t q = 0; same && q < a.size(); ++q) {
            const Phase &x = a[q], &y = b[q];
            same = x.op == y.op && x.level == y.level && x.tooth == y.tooth && x.sweep == y.sweep &&
                   (x.flags & ~kTailStart) == (y.flags & ~kTailStart);
            if (y.flags & kTailStart) {
              ++starts;
              q0 = (int)q;
              q1 = y.prev_tooth;
            } else {
              same = same && x.prev_tooth == y.prev_tooth;
            }
          }
          bool inner = true, boundary = true;
          if (q0 >= 0) {
            const int lt = n - 3;
            for (int q = q0 + 1; q < q1; ++q) inner = inner && lowest(b[q]) >= lt;
            boundary = q1 == (int)b.size() || lowest(b[q1]) < lt;
          }
          std::printf("phases %d %d %d %d %d %d %d %d %d %d %d\n", n, n_r, pair, eq10, same ? 1 : 0, starts,
                      q0 >= 0 ? b[q0].op : -1, q0 >= 0 ? b[q0].level : -1, q0 >= 0 ? q1 - q0 : 0, inner ? 1 : 0,
                      boundary ? 1 : 0);
        }
  // visit sequence of one 33^2 cycle: runs of sweeps at one level
  const std::vector<Phase> v = build_phases(5, 2, 0, false, false);
  std::printf("visits");
  int cur = -1, cnt = 0;
  for (const Phase& f : v) {
    if (f.op != OP_SWEEP) {
      if (cnt) std::printf(" %d:%d", cur, cnt);
      cur = -1;
      cnt = 0;
      continue;
    }
    if (f.level != cur && cnt) {
      std::printf(" %d:%d", cur, cnt);
      cnt = 0;
    }
    cur = f.level;
    ++cnt;
  }
  if (cnt) std::printf(" %d:%d", cur, cnt);
  std::printf("\n");
  // the tail CTA on real partitions (3-D one problem, both tile shapes, contiguous and slab cuts)
  for (int n = 4; n <= 9; ++n)
    for (int tx : {32, 64})
      for (int G : {8, 152, 304}) {
        const int ty = 2 * 256 / tx;
        int nb[1] = {n}, dir_hi[1] = {3};
        std::vector<TileTask> t((size_t)partition_bound(3, nb, 1, G, tx, ty, 32) + 1);
        std::vector<int> off((size_t)kMaxLevels * (G + 1));
        build_partition(3, nb, dir_hi, 1, G, tx, ty, t.data(), off.data(), 32);
        const int c = pick_tail_cta(off, G, n);
        auto idle = [&](int cta) {
          bool ok = true;
          for (int l = std::max(0, n - 5); l <= n - 1; ++l)
            ok = ok && off[(size_t)l * (G + 1) + cta + 1] == off[(size_t)l * (G + 1) + cta];
          return ok;
        };
        bool last = true;
        for (int d = c + 1; d < G; ++d) last = last && !idle(d);
        const bool any = [&] { for (int d = 0; d < G; ++d) if (idle(d)) return true; return false; }();
        std::printf("tailcta 3 %d %d %d %d %d %d\n", n, G, tx, c, (idle(c) || (!any && c == 0)) ? 1 : 0,
                    last ? 1 : 0);
      }
  return 0;
}
