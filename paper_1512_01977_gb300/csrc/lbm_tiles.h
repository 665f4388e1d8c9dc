// Internal: tiles of the batched step kernel and their planner (lbm_tiles.cu).
#pragma once

#include <vector>

namespace lbm {

// Rows [j0, jend) of z-strip `strip` of solve `solve`.
struct Tile {
    int solve, strip, j0, jend;
};

// Pipeline rows a tile costs beyond its own: 6 halo rows above it and the 12-row
// lag between the first and the last marching stage.
constexpr int kTileFillRows = 18;

// Plan for n solves (nz[i] x nr[i]), z-strips of `strip` columns, `slots` CTAs:
// tiles in CTA order, first[c] .. first[c + 1] those of CTA c (first has one entry
// per CTA with work, plus one).  Returns LBM_OK, LBM_ERR_INVALID_ARG or LBM_ERR_OOM.
int plan_tiles(const int* nz, const int* nr, int n, int strip, int slots, std::vector<Tile>& tiles,
               std::vector<int>& first, long long* makespan);

}  // namespace lbm
