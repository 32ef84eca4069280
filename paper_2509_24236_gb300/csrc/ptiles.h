// Point tiles of a fitness launch: how many tiles the evaluated points of a
// launch are split into (grid = particle chunks x point tiles).  Host code
// only, shared by the launches and the workspace sizing, and compiled on
// its own by the host tests.
#pragma once

#include <algorithm>
#include <cmath>

namespace pf {

// Point tiles for a launch of `chunks` particle chunks over at most `ne_max`
// evaluated points, `cap` resident CTA slots on the device and `subtile`
// points per CTA pass.  The CTA count is chosen to fill whole waves of
// resident CTAs: among 3.5 to 8.5 waves, the count with the least time in
// waves x sub-tile passes per CTA (a partial last wave, and a CTA's partial
// last sub-tile, cost whole ones), then the fullest last wave, then the
// fewest waves -- on the 640x480 / 512^3 search, 4 exact waves run 9% faster
// than 2.7 waves, and with the paper's 1/32 decimation (10240 particles x
// 9600 points) 5 tiles of two full passes beat 7 tiles whose second pass is
// a third full.  Tiles never go below one sub-tile of points; a launch too
// small for 3.5 waves takes as many tiles as it has sub-tiles.
inline int choose_ptiles_for(long long cap, long long subtile, int chunks, long long ne_max)
{
    const long long max_tiles = std::max(1LL, (ne_max + subtile - 1) / subtile);
    long long best = 0, best_cost = 0;
    double best_eff = 0.0, best_waves = 0.0;
    for (long long t = 1; t <= max_tiles; ++t) {
        const double waves = (double)(chunks * t) / (double)cap;
        if (waves > 8.5) break;
        if (waves < 3.5) continue;
        const long long passes = (ne_max + t * subtile - 1) / (t * subtile);
        const long long cost = (long long)std::ceil(waves) * passes;
        const double eff = waves / std::ceil(waves);
        if (best == 0 || cost < best_cost ||
            (cost == best_cost && (eff > best_eff + 1e-9 || (eff > best_eff - 1e-9 && waves < best_waves)))) {
            best = t;
            best_cost = cost;
            best_eff = eff;
            best_waves = waves;
        }
    }
    if (best == 0) best = std::min(max_tiles, std::max(1LL, (long long)std::ceil(3.5 * cap / chunks)));
    return (int)best;
}

// The most tiles choose_ptiles_for takes for `chunks` chunks over at most
// `ne_max` points or any fewer (a decimated schedule): what the partial
// sums are sized for.
inline int ptiles_bound_for(long long cap, long long subtile, int chunks, long long ne_max)
{
    const long long max_tiles = std::max(1LL, (ne_max + subtile - 1) / subtile);
    const long long hi = std::max((long long)std::floor(8.5 * cap / chunks), (long long)std::ceil(3.5 * cap / chunks));
    return (int)std::min(max_tiles, std::max(1LL, hi));
}

}  // namespace pf
