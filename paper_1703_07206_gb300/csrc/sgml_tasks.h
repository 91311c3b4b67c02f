// sgml_tasks.h -- host-side work partition of the tiled phases (tiles of kTX x kTY columns), used by
// sgml_api.cu and sgml_noalloc.cu.  For every level, the column tiles of all problems are cut along
// z into pieces so that each of the G CTAs of the persistent kernel receives the same number of
// tile-planes -- contiguous runs, or slabs dealt in turn (see build_partition); CTA c owns
// tasks[off[l * (G + 1) + c] .. off[l * (G + 1) + c + 1]).  A tile costs the
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

inline long long partition_bound(int dim, const int* n_of_b, int batch, int G, int kTX, int kTY, int slab = 0) {
  long long tiles = 0, slab_pieces = 0;
  const int hmin = std::max(1, (2 * slab) / 3);  // smallest slab height the slab cut picks
  for (int b = 0; b < batch; ++b)
    for (int l = 0; l <= n_of_b[b] - 1; ++l) {
      const long long N = (1LL << (n_of_b[b] - l)) + 1;
      const long long t = ((N + kTX - 1) / kTX) * ((N + kTY - 1) / kTY);
      tiles += t;
      if (dim == 3 && slab > 0) slab_pieces += t * ((N + hmin - 1) / hmin);
    }
  // contiguous cut: every tile yields at most one piece per CTA boundary it crosses, plus itself;
  // slab cut: one piece per tile and slab
  return tiles + (long long)kMaxLevels * G + slab_pieces;
}

// Level l, contiguous cut: the level's tile-planes in (problem, tile, z) order are cut into G runs of
// equal length (pieces end at tile boundaries and at run boundaries).
inline int partition_level_runs(int dim, int l, const int* n_of_b, const int* dir_hi, int batch, int G, int kTX,
                                int kTY, TileTask* tasks, int nt, int* o) {
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
        if (dim == 2) {
          tasks[nt++] = TileTask{b, (short)x0, (short)y0, 0, 1};
          acc += 1.0;
          advance();
          continue;
        }
        int z = 0;
        while (z < N) {
          int take = N - z;
          if (c < G - 1) {
            const double need = (c + 1) * target - acc;
            take = std::min(take, std::max(1, (int)std::ceil(need - 1e-9)));
          }
          tasks[nt++] = TileTask{b, (short)x0, (short)y0, (short)z, (short)take};
          acc += take;
          z += take;
          advance();
        }
      }
  }
  for (int k = c + 1; k <= G; ++k) o[k] = nt;
  return nt;
}

// Level l, slab cut (3-D): each problem's z range is cut into ceil(N / h) slabs of near-equal
// height, each (slab, tile) is one piece, and the pieces, in (problem, slab, tile) order, are dealt
// to the CTAs in turn.  All CTAs then march through the same few slabs at a time, so that the halo
// rows and columns a tile reads from its neighbours are read by their own CTAs at about the same
// time and come from L2 once.  The slab height h is picked within [2/3, 3/2] of the requested one
// so that the piece count is as close as possible to (just below) a multiple of G.
inline int partition_level_slabs(int l, const int* n_of_b, const int* dir_hi, int batch, int G, int kTX, int kTY,
                                 int slab, TileTask* tasks, int nt, int* o) {
  auto tiles_of = [&](int b, int N) {
    long long t = 0;
    for (int y0 = 0; y0 < N; y0 += kTY)
      for (int x0 = 0; x0 < N; x0 += kTX) t += tile_all_fixed(N, x0, y0, dir_hi[b]) ? 0 : 1;
    return t;
  };
  auto pieces_for = [&](int h) {
    long long count = 0;
    for (int b = 0; b < batch; ++b) {
      if (l > n_of_b[b] - 1) continue;
      const int N = (1 << (n_of_b[b] - l)) + 1;
      count += tiles_of(b, N) * ((N + h - 1) / h);
    }
    return count;
  };
  int h = slab;
  double best = 1e30;
  for (int cand = std::max(1, (2 * slab) / 3); cand <= (3 * slab + 1) / 2; ++cand) {
    const long long P = pieces_for(cand);
    if (P == 0) continue;
    const double r = (double)((P + G - 1) / G) * G / (double)P;  // busiest CTA's pieces over the mean
    if (r < best - 1e-9 || (r < best + 1e-9 && std::abs(cand - slab) < std::abs(h - slab))) {
      best = r;
      h = cand;
    }
  }
  const long long count = pieces_for(h);
  // CTA c receives pieces c, c + G, c + 2G, ...
  for (int c = 0; c <= G; ++c) o[c] = nt + (int)(c * (count / G) + std::min<long long>(c, count % G));
  long long j = 0;  // piece index in (problem, slab, tile) order
  for (int b = 0; b < batch; ++b) {
    if (l > n_of_b[b] - 1) continue;
    const int N = (1 << (n_of_b[b] - l)) + 1;
    const int ns = (N + h - 1) / h;
    for (int s = 0; s < ns; ++s) {
      const int z0 = (int)((long long)s * N / ns), z1 = (int)((long long)(s + 1) * N / ns);
      for (int y0 = 0; y0 < N; y0 += kTY)
        for (int x0 = 0; x0 < N; x0 += kTX) {
          if (tile_all_fixed(N, x0, y0, dir_hi[b])) continue;
          tasks[o[j % G] + j / G] = TileTask{b, (short)x0, (short)y0, (short)z0, (short)(z1 - z0)};
          ++j;
        }
    }
  }
  return nt + (int)count;
}

// All levels.  slab > 0 (3-D): levels whose tile-planes give every CTA at least two slabs of work
// use the slab cut, the others (small levels, where the per-piece pipeline start-up would dominate)
// the contiguous cut.
inline int build_partition(int dim, const int* n_of_b, const int* dir_hi, int batch, int G, int kTX, int kTY,
                           TileTask* tasks, int* off, int slab = 0) {
  int nt = 0;
  for (int k = 0; k < kMaxLevels * (G + 1); ++k) off[k] = 0;
  for (int l = 0; l < kMaxLevels; ++l) {
    int* o = off + (size_t)l * (G + 1);
    bool slabs = false;
    if (dim == 3 && slab > 0) {
      long long total = 0;
      for (int b = 0; b < batch; ++b) {
        if (l > n_of_b[b] - 1) continue;
        const int N = (1 << (n_of_b[b] - l)) + 1;
        for (int y0 = 0; y0 < N; y0 += kTY)
          for (int x0 = 0; x0 < N; x0 += kTX) total += tile_all_fixed(N, x0, y0, dir_hi[b]) ? 0 : N;
      }
      slabs = total >= 2LL * slab * G;
    }
    nt = slabs ? partition_level_slabs(l, n_of_b, dir_hi, batch, G, kTX, kTY, slab, tasks, nt, o)
               : partition_level_runs(dim, l, n_of_b, dir_hi, batch, G, kTX, kTY, tasks, nt, o);
  }
  return nt;
}

}  // namespace sgml
