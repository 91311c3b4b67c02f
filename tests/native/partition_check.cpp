// Host-side check of the tiled phases' work partition (sgml_tasks.h): for every level, the tasks of
// all CTAs cover every (problem, tile, plane) that holds an unknown exactly once, stay within the
// bound the allocation uses, and give the CTAs equal shares.  Prints one line per case:
//   dim n_list G tile_x slab ok max_share_over_mean_level0 longest_level0_piece
#include <cstdio>
#include <cstdlib>
#include <map>
#include <tuple>
#include <vector>

#include "sgml_tasks.h"

using namespace sgml;

static void run(int dim, std::vector<int> nb, int G, int tx, int slab) {
  const int ty = 2 * 256 / tx;
  const int batch = (int)nb.size();
  std::vector<int> dir_hi(batch);
  for (int b = 0; b < batch; ++b) dir_hi[b] = (b % 2) ? 1 : 3;  // odd problems: +y face not Dirichlet
  const long long bound = partition_bound(dim, nb.data(), batch, G, tx, ty, slab);
  std::vector<TileTask> t((size_t)bound + 1);
  std::vector<int> off((size_t)kMaxLevels * (G + 1));
  const int nt = build_partition(dim, nb.data(), dir_hi.data(), batch, G, tx, ty, t.data(), off.data(), slab);
  bool ok = nt <= bound;
  double share0 = 0.0;
  int maxnz0 = 0;
  for (int k = off[0]; k < off[G]; ++k) maxnz0 = std::max<int>(maxnz0, t[k].nz);
  for (int l = 0; l < kMaxLevels; ++l) {
    const int* o = off.data() + (size_t)l * (G + 1);
    std::map<std::tuple<int, int, int, int>, int> cover;
    long long maxw = 0, sumw = 0;
    for (int c = 0; c < G; ++c) {
      ok &= o[c] <= o[c + 1] && o[c + 1] <= nt;
      long long w = 0;
      for (int k = o[c]; k < o[c + 1]; ++k) {
        const TileTask& tk = t[k];
        ok &= tk.b >= 0 && tk.b < batch && tk.nz >= 1;
        w += tk.nz;
        for (int z = tk.z0; z < tk.z0 + tk.nz; ++z) cover[{tk.b, tk.x0, tk.y0, z}]++;
      }
      maxw = std::max(maxw, w);
      sumw += w;
    }
    long long expect = 0;
    for (int b = 0; b < batch; ++b) {
      if (l > nb[b] - 1) continue;
      const int N = (1 << (nb[b] - l)) + 1;
      for (int y0 = 0; y0 < N; y0 += ty)
        for (int x0 = 0; x0 < N; x0 += tx)
          if (!tile_all_fixed(N, x0, y0, dir_hi[b])) {
            expect += dim == 3 ? N : 1;
            for (int z = 0; z < (dim == 3 ? N : 1); ++z) ok &= cover.count({b, x0, y0, z}) == 1;
          }
    }
    ok &= (long long)cover.size() == expect;
    for (auto& kv : cover) ok &= kv.second == 1;
    if (l == 0 && sumw > 0) share0 = (double)maxw / ((double)sumw / G);
  }
  std::printf("%d ", dim);
  for (int b = 0; b < batch; ++b) std::printf("%s%d", b ? "," : "", nb[b]);
  std::printf(" %d %d %d %d %.4f %d\n", G, tx, slab, ok ? 1 : 0, share0, maxnz0);
}

int main() {
  const int tiles[] = {32, 64};
  const int slabs[] = {0, 4, 16};
  for (int tx : tiles)
    for (int slab : slabs) {
      run(3, {8}, 304, tx, slab);
      run(3, {7}, 304, tx, slab);
      run(3, {5}, 304, tx, slab);
      run(3, {1}, 304, tx, slab);
      run(3, {4}, 7, tx, slab);
      run(3, {7, 7, 7, 7, 7, 7, 7, 7, 7, 7, 7, 7, 7, 7, 7, 7}, 304, tx, slab);
      run(3, {6, 4, 5}, 152, tx, slab);
      run(2, {10}, 304, tx, slab);
      run(2, {7, 3, 5}, 304, tx, slab);
    }
  return 0;
}
