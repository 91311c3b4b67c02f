// sgml_tasks.h -- host-side work partition of the tiled phases (tiles of kTX x kTY columns) (used by sgml_api.cu and
// sgml_noalloc.cu).  For every level, the column tiles of all problems are cut along z into
// contiguous pieces so that each of the G CTAs of the persistent kernel receives the same number of
// tile-planes; CTA c owns tasks[off[l * (G + 1) + c] .. off[l * (G + 1) + c + 1]).  A tile costs the
// same whatever number of its columns lie inside the level (the halo and the arithmetic run at full
// width), so every tile weighs one; tiles whose inside columns all lie on a Dirichlet face (the
// last column / row of an N = 2^n + 1 level) hold no unknowns and are left out.  A static, balanced
// partition keeps both CTAs of an SM equally loaded, which matters for the FP64-pipe-bound residual
// and the issue-bound sweeps alike.
#pragma once
#include <algorithm>
#include <cmath>

#include "sgml_internal.cuh"

namespace sgml {

// Number of tasks the partition produces is at most count_bound(...); `tasks` must hold that many
// and `off` kMaxLevels * (G + 1) ints.  Returns the number of tasks written.
// Tile (x0, y0) of a level with N nodes per side holds no unknown: its inside columns all lie on
// the +x face (x0 = N - 1) or the +y face (y0 = N - 1) and that face is Dirichlet.  dir_hi bit 0:
// +x Dirichlet, bit 1: +y Dirichlet.
inline bool tile_all_fixed(int N, int x0, int y0, int dir_hi) {
  return (x0 == N - 1 && (dir_hi & 1)) || (y0 == N - 1 && (dir_hi & 2));
}

inline long long partition_bound(int dim, const int* n_of_b, int batch, int G, int kTX, int kTY) {
  long long tiles = 0;
  for (int b = 0; b < batch; ++b)
    for (int l = 0; l <= n_of_b[b] - 1; ++l) {
      const long long N = (1LL << (n_of_b[b] - l)) + 1;
      tiles += ((N + kTX - 1) / kTX) * ((N + kTY - 1) / kTY);
    }
  // every tile yields at most one piece per CTA boundary it crosses, plus itself
  return tiles + (long long)kMaxLevels * G + (dim == 3 ? 0 : 0);
}

inline int build_partition(int dim, const int* n_of_b, const int* dir_hi, int batch, int G, int kTX, int kTY,
                           TileTask* tasks, int* off) {
  int nt = 0;
  for (int k = 0; k < kMaxLevels * (G + 1); ++k) off[k] = 0;
  for (int l = 0; l < kMaxLevels; ++l) {
    int* o = off + (size_t)l * (G + 1);
    // total weighted work of the level
    double total = 0.0;
    for (int b = 0; b < batch; ++b) {
      if (l > n_of_b[b] - 1) continue;
      const int N = (1 << (n_of_b[b] - l)) + 1;
      const int planes = dim == 3 ? N : 1;
      for (int y0 = 0; y0 < N; y0 += kTY)
        for (int x0 = 0; x0 < N; x0 += kTX)
          if (!tile_all_fixed(N, x0, y0, dir_hi[b])) total += planes;
    }
    const double target = total / G;
    int c = 0;
    double acc = 0.0;
    o[0] = nt;
    auto advance = [&]() {
      while (c < G - 1 && acc >= (c + 1) * target - 1e-9) {
        ++c;
        o[c] = nt;
      }
    };
    for (int b = 0; b < batch; ++b) {
      if (l > n_of_b[b] - 1) continue;
      const int N = (1 << (n_of_b[b] - l)) + 1;
      for (int y0 = 0; y0 < N; y0 += kTY)
        for (int x0 = 0; x0 < N; x0 += kTX) {
          if (tile_all_fixed(N, x0, y0, dir_hi[b])) continue;
          const double w = 1.0;
          if (dim == 2) {
            tasks[nt++] = TileTask{b, (short)x0, (short)y0, 0, 1};
            acc += w;
            advance();
            continue;
          }
          int z = 0;
          while (z < N) {
            int take = N - z;
            if (c < G - 1) {
              const double need = (c + 1) * target - acc;
              take = std::min(take, std::max(1, (int)std::ceil(need / w - 1e-9)));
            }
            tasks[nt++] = TileTask{b, (short)x0, (short)y0, (short)z, (short)take};
            acc += take * w;
            z += take;
            advance();
          }
        }
    }
    for (int k = c + 1; k <= G; ++k) o[k] = nt;
  }
  return nt;
}

}  // namespace sgml
