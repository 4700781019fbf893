// Host-side tables of the PCG's halo layout (SR_HALO, pcg_sr.cu): for each CTA
// of a launch, the rows of other CTAs that columns of its rows refer to, and
// every block's column in the CTA's local numbering.  Pure host code, so that
// the tables can be built and checked without a GPU.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

#include "kernels.h"

namespace ppn {

// BSR pattern of one scene of the launch (slot order); its rows are split
// into PCG_TILE-row tiles, all of them in the launch's tile table.
struct HaloPattern {
  int nv;
  const int64_t* row_ptr;  // nv + 1
  const int* col;          // row_ptr[nv], ascending per row
};

// Tables for `grid` CTAs over the launch's tile table (every tile of slot 0,
// then of slot 1, ...; CTA b owns tiles [b n / grid, (b + 1) n / grid)), laid
// out as PcgLaunch::halo_off, halo_col, halo_ref one after the other in `tab`:
//   [2 (grid + 1)]   first block and first halo row of each CTA, then the totals
//   [blocks]         local column of each block: own row item (tile index in the
//                    CTA x PCG_TILE + row within the tile), or n_items + the
//                    column's index in the CTA's halo list
//   [halo rows]      slot << HALO_ROW_BITS | row, ascending within each CTA
// Blocks are in the kernel's order: the CTA's tiles, their rows, each row's
// blocks.  Returns the most halo rows of one CTA; -1 when a scene has
// 2^HALO_ROW_BITS rows or more, there are more than HALO_MAX_SCENES scenes, or
// grid is outside [1, tiles].
inline int build_halo_tables(const std::vector<HaloPattern>& pats, int grid, std::vector<int>& tab) {
  const size_t ns = pats.size();
  if (ns == 0 || ns > (size_t)HALO_MAX_SCENES) return -1;
  std::vector<int> toff(ns + 1, 0);
  for (size_t k = 0; k < ns; ++k) {
    if (pats[k].nv <= 0 || pats[k].nv >= (1 << HALO_ROW_BITS)) return -1;
    toff[k + 1] = toff[k] + (pats[k].nv + PCG_TILE - 1) / PCG_TILE;
  }
  const int n_tiles = toff[ns];
  if (grid < 1 || grid > n_tiles) return -1;
  std::vector<int> tslot(n_tiles);
  for (size_t k = 0; k < ns; ++k)
    for (int t = toff[k]; t < toff[k + 1]; ++t) tslot[t] = (int)k;
  std::vector<std::vector<int>> mark(ns), hidx(ns);
  for (size_t k = 0; k < ns; ++k) {
    mark[k].assign(pats[k].nv, -1);
    hidx[k].assign(pats[k].nv, 0);
  }
  std::vector<int> off(2 * (grid + 1), 0), col, ref;
  std::vector<long long> hs;
  int maxh = 0;
  // every block of launch tiles [t0, t1), in the kernel's order: f(slot, column, column's launch tile)
  auto blocks = [&](int t0, int t1, auto&& f) {
    for (int t = t0; t < t1; ++t) {
      const int k = tslot[t];
      const HaloPattern& p = pats[k];
      const int r0 = (t - toff[k]) * PCG_TILE, r1 = std::min(p.nv, r0 + PCG_TILE);
      for (int r = r0; r < r1; ++r)
        for (int64_t q = p.row_ptr[r]; q < p.row_ptr[r + 1]; ++q) {
          const int j = p.col[q];
          f(k, j, toff[k] + j / PCG_TILE);
        }
    }
  };
  for (int b = 0; b < grid; ++b) {
    const int t0 = (int)(((long long)b * n_tiles) / grid), t1 = (int)(((long long)(b + 1) * n_tiles) / grid);
    const int n_items = (t1 - t0) * PCG_TILE;
    off[2 * b] = (int)col.size();
    off[2 * b + 1] = (int)ref.size();
    hs.clear();
    blocks(t0, t1, [&](int k, int j, int gt) {
      if ((gt < t0 || gt >= t1) && mark[k][j] != b) {
        mark[k][j] = b;
        hs.push_back(((long long)k << 32) | j);
      }
    });
    std::sort(hs.begin(), hs.end());
    for (size_t h = 0; h < hs.size(); ++h) {
      const int k = (int)(hs[h] >> 32), j = (int)(hs[h] & 0xffffffffll);
      hidx[k][j] = (int)h;
      ref.push_back((k << HALO_ROW_BITS) | j);
    }
    blocks(t0, t1, [&](int k, int j, int gt) {
      col.push_back(gt >= t0 && gt < t1 ? (gt - t0) * PCG_TILE + j % PCG_TILE : n_items + hidx[k][j]);
    });
    maxh = std::max(maxh, (int)hs.size());
  }
  off[2 * grid] = (int)col.size();
  off[2 * grid + 1] = (int)ref.size();
  tab = off;
  tab.insert(tab.end(), col.begin(), col.end());
  tab.insert(tab.end(), ref.begin(), ref.end());
  return maxh;
}

}  // namespace ppn
