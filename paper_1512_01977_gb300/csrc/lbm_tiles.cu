// Work plan of the batched step kernel: the (z-strip, row) space of every solve
// is cut into tiles (rows [j0, jend) of one strip of one solve) and the tiles
// are dealt to the CTAs of one launch, largest first, each to the CTA with the
// smallest load so far (longest-processing-time scheduling).  A tile costs its
// rows plus kTileFillRows rows of pipeline fill: the kernel marches 6 halo rows
// above the tile and its last stage trails the first by 12 rows.  Host code.
#include <algorithm>
#include <new>
#include <queue>
#include <vector>

#include "lbm_axi_batch.h"
#include "lbm_tiles.h"

namespace lbm {

namespace {

struct Cand {
    std::vector<Tile> tiles;
    std::vector<int> first;
    long long makespan = -1;
    int ncta = 0;
};

// Tiles of chunk height at most h (h <= 0: one tile per strip), rows split evenly.
void cut(const int* nz, const int* nr, int n, int strip, int h, std::vector<Tile>& out) {
    out.clear();
    for (int s = 0; s < n; s++) {
        const int strips = (nz[s] + strip - 1) / strip;
        const int c = h > 0 ? std::max(1, (nr[s] + h - 1) / h) : 1;
        const int q = nr[s] / c, r = nr[s] % c;
        for (int t = 0; t < strips; t++) {
            int j = 0;
            for (int k = 0; k < c; k++) {
                const int rows = q + (k < r ? 1 : 0);
                out.push_back(Tile{s, t, j, j + rows});
                j += rows;
            }
        }
    }
}

long long count_tiles(const int* nz, const int* nr, int n, int strip, int h) {
    long long t = 0;
    for (int s = 0; s < n; s++)
        t += (long long)((nz[s] + strip - 1) / strip) * std::max(1, (nr[s] + h - 1) / h);
    return t;
}

void deal(std::vector<Tile>& tiles, int slots, Cand& c) {
    std::vector<int> order(tiles.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return tiles[a].jend - tiles[a].j0 > tiles[b].jend - tiles[b].j0;
    });
    // min-heap of (load, cta)
    typedef std::pair<long long, int> L;
    std::priority_queue<L, std::vector<L>, std::greater<L>> heap;
    const int used = (int)std::min<size_t>((size_t)slots, tiles.size());
    for (int k = 0; k < used; k++) heap.push(L(0, k));
    std::vector<int> owner(tiles.size());
    std::vector<long long> load(used, 0);
    for (int i : order) {
        L top = heap.top();
        heap.pop();
        owner[i] = top.second;
        top.first += tiles[i].jend - tiles[i].j0 + kTileFillRows;
        load[top.second] = top.first;
        heap.push(top);
    }
    // group by CTA; within a CTA keep the cut order (solve, strip, rows)
    std::vector<int> count(used + 1, 0);
    for (size_t i = 0; i < tiles.size(); i++) count[owner[i] + 1]++;
    for (int k = 0; k < used; k++) count[k + 1] += count[k];
    c.first = count;
    c.tiles.assign(tiles.size(), Tile{0, 0, 0, 0});
    std::vector<int> pos(count.begin(), count.end() - 1);
    for (size_t i = 0; i < tiles.size(); i++) c.tiles[pos[owner[i]]++] = tiles[i];
    c.makespan = 0;
    for (long long x : load) c.makespan = std::max(c.makespan, x);
    c.ncta = used;
}

}  // namespace

int plan_tiles(const int* nz, const int* nr, int n, int strip, int slots, std::vector<Tile>& tiles,
               std::vector<int>& first, long long* makespan) {
    if (!nz || !nr || n < 1 || strip < 1 || slots < 1) return LBM_ERR_INVALID_ARG;
    int max_nr = 0;
    for (int s = 0; s < n; s++) {
        if (nz[s] < 1 || nr[s] < 1) return LBM_ERR_INVALID_ARG;
        max_nr = std::max(max_nr, nr[s]);
    }
    try {
        // candidate chunk heights: whole strips, and the smallest height (>= 16 rows)
        // whose tiles fill k = 1..4 waves of CTAs
        std::vector<int> heights = {0};
        for (int k = 1; k <= 4; k++) {
            int lo = std::min(16, max_nr), hi = max_nr;
            if (count_tiles(nz, nr, n, strip, hi) > (long long)k * slots) continue;
            while (lo < hi) {
                const int mid = (lo + hi) / 2;
                if (count_tiles(nz, nr, n, strip, mid) <= (long long)k * slots) hi = mid;
                else lo = mid + 1;
            }
            heights.push_back(lo);
        }
        Cand best;
        std::vector<Tile> cutv;
        for (int h : heights) {
            cut(nz, nr, n, strip, h, cutv);
            Cand c;
            deal(cutv, slots, c);
            if (best.makespan < 0 || c.makespan < best.makespan ||
                (c.makespan == best.makespan && c.tiles.size() < best.tiles.size()))
                best = std::move(c);
        }
        tiles = std::move(best.tiles);
        first = std::move(best.first);
        if (makespan) *makespan = best.makespan;
    } catch (const std::bad_alloc&) {
        return LBM_ERR_OOM;
    }
    return LBM_OK;
}

}  // namespace lbm

extern "C" int lbm_axi_tile_plan(const int* nz, const int* nr, int n, int strip, int slots, int max_tiles,
                                 int* tiles_out, int* first_out, int* ntiles, int* ncta, long long* makespan) {
    if (!ntiles || !ncta || max_tiles < 0) return LBM_ERR_INVALID_ARG;
    std::vector<lbm::Tile> tiles;
    std::vector<int> first;
    long long ms = 0;
    const int rc = lbm::plan_tiles(nz, nr, n, strip, slots, tiles, first, &ms);
    if (rc != LBM_OK) return rc;
    *ntiles = (int)tiles.size();
    *ncta = (int)first.size() - 1;
    if (makespan) *makespan = ms;
    if ((int)tiles.size() > max_tiles || !tiles_out || !first_out) return LBM_ERR_INVALID_ARG;
    for (size_t i = 0; i < tiles.size(); i++) {
        tiles_out[4 * i] = tiles[i].solve;
        tiles_out[4 * i + 1] = tiles[i].strip;
        tiles_out[4 * i + 2] = tiles[i].j0;
        tiles_out[4 * i + 3] = tiles[i].jend;
    }
    for (size_t c = 0; c < first.size(); c++) first_out[c] = first[c];
    return LBM_OK;
}
