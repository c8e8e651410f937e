// autotune.h -- coordinate search over the launch-shape / search parameters
// of an evaluation (host code).  time(u, cold, &ms) times evaluations with
// tuning u (cold: without radius hints).  Each coordinate is swept with the
// others fixed, in the order concurrent chunks, topology lanes per cell, bin
// load, topology warps per block, topology grid cap, quadrature block,
// first-pass target;
// knn_target only matters for
// evaluations without hints, so it is compared on cold evaluations.
#pragma once

#include <string.h>

#include "scvt_internal.cuh"

namespace scvt {

template <class TimeFn>
scvt_status autotune(Tune cur, TimeFn &&time, Tune *out) {
    static const int loads[] = {1, 2, 4, 8};
    static const int warps[] = {2, 4, 8};
    static const int bpsm[] = {8, 16, 32};
    static const int qblk[] = {128, 256, 512};
    static const int targets[] = {16, 24, 32, 48};
    static const int lanes[] = {32, 16};
    static const int chunks[] = {1, 2, 3, 4};
    float cur_ms;
    scvt_status s = time(cur, false, &cur_ms);
    if (s) return s;
    for (int coord = 0; coord < 7; ++coord) {
        const int *vals;
        int nv;
        switch (coord) {
        case 0: vals = chunks; nv = 4; break;
        case 1: vals = lanes; nv = 2; break;
        case 2: vals = loads; nv = 4; break;
        case 3: vals = warps; nv = 3; break;
        case 4: vals = bpsm; nv = 3; break;
        case 5: vals = qblk; nv = 3; break;
        default: vals = targets; nv = 4; break;
        }
        const bool cold = coord == 6;
        Tune best = cur;
        float best_ms = cur_ms;
        if (cold && (s = time(cur, true, &best_ms))) return s;
        for (int k = 0; k < nv; ++k) {
            Tune u = cur;
            switch (coord) {
            case 0: u.chunks = vals[k]; break;
            case 1: u.topo_lanes = vals[k]; break;
            case 2: u.bin_load = vals[k]; break;
            case 3: u.topo_warps = vals[k]; break;
            case 4: u.topo_bpsm = vals[k]; break;
            case 5: u.quad_block = vals[k]; break;
            default: u.knn_target = vals[k]; break;
            }
            if (memcmp(&u, &cur, sizeof(Tune)) == 0) continue;
            float ms;
            if ((s = time(u, cold, &ms))) return s;
            if (ms < best_ms) {
                best_ms = ms;
                best = u;
            }
        }
        cur = best;
        if (!cold) cur_ms = best_ms;
    }
    *out = cur;
    return SCVT_OK;
}

}  // namespace scvt
