// lockstep.cu -- many problems' LBFGS iterations in lockstep (see lockstep.cuh).
#include <math.h>
#include <string.h>

#include <algorithm>

#include "lockstep.cuh"

namespace scvt {

namespace {

cudaError_t sync_statuses(EvalSet &E) {
    cudaError_t e = cudaMemcpyAsync(E.h_ist, E.d_ist, sizeof(DevStatus) * E.B, cudaMemcpyDeviceToHost, E.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E.stream);
    return e;
}

// Descriptors of every problem of the layout for the segmented kernels:
// geometry, resident buffers and chunking; the round's flags are cleared.
// Problems without a lane this round keep all flags 0.
void seg_layout(EvalSet &E, const std::vector<Lane *> &lanes, int m) {
    int blk3 = 0, blk1 = 0;
    size_t pb = 0;
    for (int b = 0; b < E.B; ++b) {
        SegLane &d = E.h_seg[b];
        memset(&d, 0, sizeof(d));
        d.row = E.geom[b].p0;
        d.n = E.geom[b].n;
        d.m = m;
        d.nb3 = reduce_blocks(3 * (int64_t)d.n);
        d.nb1 = reduce_blocks(d.n);
        d.blk3 = blk3;
        d.blk1 = blk1;
        blk3 += d.nb3;
        blk1 += d.nb1;
        d.scal = E.seg_scal + (size_t)b * kTwoLoopScratch;
        d.partials = E.seg_partials + pb;
        pb += (size_t)std::max(kCmpQ * d.nb3, 4 * d.nb1);
        d.st = E.d_ist + b;
    }
    E.nblk3 = blk3;
    E.nblk1 = blk1;
    for (const Lane *L : lanes) {
        SegLane &d = E.h_seg[L->b];
        d.z = L->z;
        d.g = L->g;
        d.h = L->h;
        d.hist = L->hist;
        d.yhist = L->hist + L->y_off;
        d.slot_stride = (int64_t)L->slot_stride;
        d.rho = L->rho;
        d.method = L->opt.method;
    }
}

cudaError_t seg_upload(EvalSet &E) {
    return cudaMemcpyAsync(E.d_seg, E.h_seg, sizeof(SegLane) * E.B, cudaMemcpyHostToDevice, E.stream);
}

// the direction of every lane in dir (its history as the ring holds it; none for Lloyd)
cudaError_t seg_directions(EvalSet &E, const std::vector<Lane *> &dir, int64_t *launches) {
    for (int b = 0; b < E.B; ++b) E.h_seg[b].dir = 0;
    bool gathered = false;
    int max_step = -1;
    for (Lane *L : dir) {
        SegLane &d = E.h_seg[L->b];
        d.dir = 1;
        d.count = (L->opt.method == 2) ? 0 : L->count;
        for (int k = 0; k < d.count; ++k) d.slots[k] = L->slots[k];
        d.new_pair = L->new_pair ? 1 : 0;
        L->new_pair = false;
        if (d.count >= 1 && d.count <= kCmpMax) gathered = true;
        else max_step = std::max(max_step, d.count);
    }
    cudaError_t e = seg_upload(E);
    if (e != cudaSuccess) return e;
    seg_direction(E.d_seg, E.B, gathered, max_step, E.nblk3, E.q, E.stream, launches);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return sync_statuses(E);
}

}  // namespace

void lane_reset_history(Lane &L, int m) {
    L.count = 0;
    L.new_pair = false;
    for (int k = 0; k <= m; ++k) L.slots[k] = k;
    L.spare = m;
}

scvt_status lane_options(const scvt_solve_opts *in, scvt_solve_opts *o) {
    memset(o, 0, sizeof(*o));
    if (in) *o = *in;
    else {
        o->max_iter = 200;
        o->grad_tol = 1e-8;
    }
    if (o->ls_max_evals <= 0) o->ls_max_evals = 10;
    if (o->c1 <= 0.0) o->c1 = 1e-4;
    if (o->c2 <= 0.0) o->c2 = 0.9;
    if (o->max_iter < 0 || !(o->c1 < o->c2) || o->c2 >= 1.0 || o->method < 0 || o->method > 2)
        return SCVT_ERR_INVALID;
    return SCVT_OK;
}

cudaError_t lockstep_round(EvalSet &E, std::vector<Lane *> &lanes, int m, scvt_stats *stats) {
    cudaStream_t s = E.stream;
    int64_t *launches = &stats->kernel_launches;
    cudaError_t e;
    // ---- stopping tests of the running lanes
    std::vector<Lane *> act, init;
    for (Lane *L : lanes) {
        if (L->done) continue;
        if (L->need_init) {
            init.push_back(L);
            continue;
        }
        L->rep.energy = L->F;
        L->rep.grad_norm = L->gnorm;
        const scvt_solve_opts &o = L->opt;
        bool stop = false;
        if (L->gnorm <= o.grad_tol) { L->rep.converged = 1; stop = true; }
        else if (o.rel_grad_tol > 0 && L->gnorm / L->F <= o.rel_grad_tol) { L->rep.converged = 1; stop = true; }
        else if (L->rep.iters > 0 && o.rel_df_tol > 0 && fabs(L->F - L->Fprev) / L->Fprev < o.rel_df_tol) {
            L->rep.converged = 1;
            stop = true;
        } else if (L->rep.iters >= o.max_iter) {
            stop = true;
        }
        if (stop) L->done = true;
        else act.push_back(L);
    }
    seg_layout(E, lanes, m);
    // ---- directions, one launch per pass for every lane (again, from an empty
    // history, where one is not a descent direction)
    if (!act.empty()) {
        Phase ph("scvt batch directions");
        if ((e = seg_directions(E, act, launches)) != cudaSuccess) return e;
        std::vector<Lane *> redo;
        for (Lane *L : act) {
            L->d0 = E.h_ist[L->b].dots[3];
            if (!(L->d0 < 0.0)) redo.push_back(L);
        }
        if (!redo.empty()) {
            for (Lane *L : redo) {
                lane_reset_history(*L, m);
                L->rep.resets++;
            }
            if ((e = seg_directions(E, redo, launches)) != cudaSuccess) return e;
            for (Lane *L : redo) {
                L->d0 = E.h_ist[L->b].dots[3];
                if (!(L->d0 < 0.0)) {
                    L->rep.status = SCVT_ERR_DEGENERATE;
                    L->done = true;
                    L->state_valid = false;
                }
            }
        }
    }
    // ---- line searches in lockstep; the first round also evaluates the new lanes
    std::vector<Lane *> ls;
    for (Lane *L : act) {
        if (L->done) continue;
        L->ls.ftol = L->opt.c1;
        L->ls.gtol = L->opt.c2;
        L->ls.maxfev = L->opt.ls_max_evals;
        L->unit_step = L->opt.method == 2;
        L->ls_state = L->unit_step ? 0 : L->ls.begin(L->F, L->d0, 1.0);
        if (L->ls_state == 0) ls.push_back(L);
    }
    bool first = true;
    Phase pl("scvt batch line search");
    while (!ls.empty() || (first && !init.empty())) {
        for (int b = 0; b < E.B; ++b) {
            E.h_active[b] = 0;
            E.h_seg[b].trial = 0;
        }
        for (Lane *L : ls) {
            E.h_seg[L->b].alpha = L->unit_step ? 1.0 : L->ls.trial();
            E.h_seg[L->b].trial = 1;
            E.h_active[L->b] = 1;
        }
        if (!ls.empty()) {
            if ((e = seg_upload(E)) != cudaSuccess) return e;
            seg_trial(E.d_seg, E.d_pinst, E.ntot, E.q, E.zt, E.nrm, s, launches);
        }
        if (first) {
            for (Lane *L : init) {
                e = cudaMemcpyAsync(E.zt + 3 * L->row, L->z, sizeof(double) * 3 * L->n, cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) return e;
                E.h_active[L->b] = 1;
            }
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = evalset_run(E, stats)) != cudaSuccess) return e;
        if (first) {
            for (Lane *L : init) {
                const DevStatus &ds = E.h_ist[L->b];
                L->need_init = false;
                L->rep.fevals += 1;
                const scvt_status sb = status_of_flags(ds.flags);
                if (sb) {
                    L->rep.status = sb;
                    L->done = true;
                    L->state_valid = false;
                    continue;
                }
                L->F = ds.red[0];
                L->Fprev = L->F;
                L->gnorm = sqrt(ds.red[1]);
                L->state_valid = true;
                lane_reset_history(*L, m);
                cudaMemcpyAsync(L->g, E.gt + 3 * L->row, sizeof(double) * 3 * L->n, cudaMemcpyDeviceToDevice, s);
                cudaMemcpyAsync(L->h, E.ht + L->row, sizeof(double) * L->n, cudaMemcpyDeviceToDevice, s);
            }
            first = false;
        }
        std::vector<Lane *> next;
        for (Lane *L : ls) {
            const DevStatus &ds = E.h_ist[L->b];
            const scvt_status sb = status_of_flags(ds.flags);
            L->g2_last = ds.red[1];
            if (L->unit_step) {
                // Lloyd: the unit step is taken as it is; a broken tessellation ends the lane
                L->ls.nfev = 1;
                L->ls.last_a = 1.0;
                L->ls.last_f = ds.red[0];
                L->ls.last_d = ds.red[2];
                if (sb) {
                    L->rep.fevals += 1;
                    L->rep.status = SCVT_ERR_DEGENERATE;
                    L->done = true;
                    L->state_valid = false;
                }
                L->ls_state = 1;
                continue;
            }
            // a step that breaks the tessellation is a failed trial, not an error
            L->ls_state = L->ls.feed(sb ? 1 : 0, sb ? 0.0 : ds.red[0], sb ? 0.0 : ds.red[2]);
            if (L->ls_state == 0) next.push_back(L);
        }
        ls.swap(next);
    }
    // ---- accept (or restart): one launch for every accepting lane
    std::vector<Lane *> acc;
    for (int b = 0; b < E.B; ++b) {
        E.h_seg[b].accept = 0;
        E.h_seg[b].trial = 0;
    }
    for (Lane *L : act) {
        if (L->done) continue;
        L->rep.fevals += L->ls.nfev;
        const int info = L->ls_state;
        const double fa = L->ls.last_f;
        if (info != 1) {
            if (!(fa < L->F)) {
                if (L->count == 0) {
                    L->rep.status = SCVT_ERR_LINESEARCH;
                    L->done = true;
                    continue;
                }
                lane_reset_history(*L, m);
                L->rep.resets++;
                continue;
            }
            lane_reset_history(*L, m);
            L->rep.resets++;
        }
        // (the status block's maxmove_bits was cleared by the last evaluation)
        E.h_seg[L->b].accept = 1;
        E.h_seg[L->b].spare = L->spare;
        acc.push_back(L);
    }
    if (!acc.empty()) {
        if ((e = seg_upload(E)) != cudaSuccess) return e;
        seg_accept(E.d_seg, E.B, E.nblk1, E.zt, E.gt, E.ht, s, launches);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = sync_statuses(E)) != cudaSuccess) return e;
    }
    for (Lane *L : acc) {
        const DevStatus &ds = E.h_ist[L->b];
        const double ys = ds.dots[0], yy = ds.dots[1], ss = ds.dots[2];
        double maxmove;
        unsigned long long mb = ds.maxmove_bits;
        memcpy(&maxmove, &mb, sizeof(double));
        const int slot = L->spare;
        // the same curvature test the accept kernel took (it has set 1/(y.s))
        if (L->opt.method != 2 && m > 0 && ys > 1e-12 * sqrt(yy) * sqrt(ss)) {
            if (L->count == m) {
                int old = L->slots[0];
                for (int k = 1; k < L->count; ++k) L->slots[k - 1] = L->slots[k];
                L->count--;
                L->spare = old;
            } else {
                bool used[kLaneMaxM + 1] = {false};
                for (int k = 0; k < L->count; ++k) used[L->slots[k]] = true;
                used[slot] = true;
                for (int k = 0; k <= m; ++k)
                    if (!used[k]) { L->spare = k; break; }
            }
            L->slots[L->count++] = slot;
            L->new_pair = true;
        } else if (L->opt.method != 2) {
            L->rep.skipped++;
        }
        // (z, g and h moved to the trial point in the accept kernel)
        L->Fprev = L->F;
        L->F = L->ls.last_f;
        L->gnorm = sqrt(L->g2_last);
        L->rep.iters++;
        L->rep.energy = L->F;
        L->rep.grad_norm = L->gnorm;
        if (L->opt.step_tol > 0 && maxmove <= L->opt.step_tol) {
            L->rep.converged = 1;
            L->done = true;
        }
    }
    return cudaGetLastError();
}

}  // namespace scvt
