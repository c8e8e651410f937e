// lockstep.cuh -- Lloyd-preconditioned LBFGS of many problems in lockstep
// (not installed).
//
// A Lane is one problem of an EvalSet layout: its resident iterate,
// gradient, preconditioner and history live wherever the owner keeps them
// (rows of concatenated arrays for a batch, the job's own buffers in the
// server); its trial point, trial gradient and direction are the problem's
// rows of the EvalSet.  lockstep_round() advances every lane by one LBFGS
// iteration (Sec. 3.1): stopping test, two-loop direction with diag(h) as
// H0, strong-Wolfe line search (one EvalSet evaluation per round of trial
// points of all searching lanes), curvature test and history update.  The
// per-lane logic is that of the single-problem solver, so a lane reproduces
// a single-problem solve bit for bit.
#pragma once

#include <vector>

#include "evalset.cuh"
#include "wolfe.h"

namespace scvt {


struct Lane {
    int b = 0;            // problem index in the EvalSet layout
    int n = 0;
    int64_t row = 0;      // first row in the EvalSet
    double *z = nullptr, *g = nullptr, *h = nullptr;  // resident state (n x 3, n x 3, n)
    double *hist = nullptr;                 // S of slot k at hist + k slot_stride, Y at S + y_off
    size_t slot_stride = 0, y_off = 0;
    double *rho = nullptr;                  // kLaneRho doubles: 1 / (y.s) of each slot, then gamma
    scvt_solve_opts opt;                    // this lane's options (defaults filled in)
    // solver state
    int slots[kLaneMaxM + 1];
    int count = 0, spare = 0;
    bool new_pair = false;                  // a pair was stored after the last direction
    double F = 0.0, gnorm = 0.0, Fprev = 0.0;
    bool done = false, need_init = false, state_valid = false;
    scvt_solve_report rep;
    WolfeSearch ls;
    int ls_state = 0;
    double d0 = 0.0, g2_last = 0.0;
    bool unit_step = false;  // Lloyd: one evaluation at alpha = 1, no line search
};

void lane_reset_history(Lane &L, int m);
// options with defaults filled in; INVALID on bad values
scvt_status lane_options(const scvt_solve_opts *in, scvt_solve_opts *out);
// one outer iteration of every lane that is not done, each with its own
// options; lanes with need_init get their first evaluation (at z) in the
// first evaluation round instead.  The LBFGS steps of all lanes run as
// segmented kernels (one launch per two-loop pass, one for the trial points
// of a line-search round, one for the accepted pairs), each lane with the
// single-problem kernels' chunking and arithmetic.  Returns a CUDA error only
// for failures of the device itself; a problem's own failure ends that lane
// with rep.status set.
cudaError_t lockstep_round(EvalSet &E, std::vector<Lane *> &lanes, int m, scvt_stats *stats);

}  // namespace scvt
