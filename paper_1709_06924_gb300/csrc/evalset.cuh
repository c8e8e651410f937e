// evalset.cuh -- the evaluation workspace shared by batches and the server
// (not installed).
//
// An EvalSet evaluates a set of independent problems laid out in rows: the
// problem b of the current layout owns rows [p0_b, p0_b + n_b) of the row
// arrays (zt, gt, ht, fc, q, nrm, radius) and its own block of cube-map
// bins.  One evaluation = binning, topology passes, corners, per-edge
// quadrature, per-cell sums over all problems' cells, then one reduction per
// problem (the chunking of a single problem of its size), for the problems
// marked active.  The sequence has fixed pointers and launch shapes for a
// given layout and tuning, so it is captured once as a CUDA graph and
// replayed; a new layout or tuning drops the graph.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "scvt_internal.cuh"

namespace scvt {

struct EvalSet {
    // capacity
    int64_t cap_n = 0;
    int cap_b = 0;
    int precision = 0;
    int fan = 0;
    cudaStream_t stream = nullptr;
    // current layout
    int B = 0;
    int64_t ntot = 0;
    std::vector<InstGeom> geom;
    std::vector<int> gsel;  // per problem: bins per face edge chosen by adapt_bins (0 = the tuning's)
    std::vector<int> pbase;
    int max_nb = 1;
    int nbins = 0;
    Tune tune;
    Pipes pipes;
    // device tables and their pinned mirrors
    InstGeom *d_inst = nullptr;
    int *d_pinst = nullptr, *d_pbase = nullptr, *d_active = nullptr;
    Density *d_rho = nullptr;
    DensityF *d_rhof = nullptr;
    DensDF *d_rhodf = nullptr;
    DevStatus *d_ist = nullptr, *d_st = nullptr;
    DevStatus *h_ist = nullptr, *h_st = nullptr;
    int *h_active = nullptr;
    // row arrays
    double *zt = nullptr, *gt = nullptr, *ht = nullptr, *fc = nullptr, *q = nullptr, *nrm = nullptr;
    float *radius = nullptr;
    double *partials = nullptr;
    size_t partials_len = 0;
    // workspace
    P4 *zs = nullptr, *cvx = nullptr;
    float4 *zf = nullptr, *zl = nullptr, *zll = nullptr, *vo = nullptr, *ctab = nullptr;
    int *cdeg = nullptr, *cnb = nullptr, *eoff = nullptr, *ecell = nullptr, *escan = nullptr;
    double *eacc = nullptr;
    // density tables of the problems (FP64 forms): a pool carved per layout
    void *tab_pool = nullptr;
    size_t tab_pool_bytes = 0;
    DensTab *d_tabs = nullptr;
    std::vector<DensTab> tabs;
    int *bin_of = nullptr, *count = nullptr, *start = nullptr, *cursor = nullptr, *scan_tmp = nullptr;
    int *sidx = nullptr, *list1 = nullptr, *list2 = nullptr;
    // segmented LBFGS of the problems (lockstep.cu): per-problem descriptors
    // (device and pinned host copies), chunk sums and scalars; nblk3 / nblk1 =
    // the blocks of the segmented grids of this layout
    SegLane *d_seg = nullptr, *h_seg = nullptr;
    double *seg_partials = nullptr, *seg_scal = nullptr;
    size_t seg_partials_len = 0;
    int nblk3 = 0, nblk1 = 0;
    // the captured evaluation
    cudaGraphExec_t graph = nullptr;
    int64_t graph_launches = 0, graph_cell_launches = 0;
    int64_t bytes = 0;
};

// device bytes an EvalSet of this capacity allocates
int64_t evalset_bytes(int64_t cap_n, int cap_b, int precision);
// allocate for up to cap_n rows and cap_b problems; work is ordered on s
cudaError_t evalset_alloc(EvalSet &E, int64_t cap_n, int cap_b, int precision, cudaStream_t s);
void evalset_free(EvalSet &E);
// lay out B problems (sizes ns, densities rhos) in rows 0.. in order; the
// row arrays (radius hints included) are left as they are
cudaError_t evalset_layout(EvalSet &E, int B, const int *ns, const scvt_density *rhos);
// new tuning: re-bins the problems, drops the graph
cudaError_t evalset_set_tune(EvalSet &E, const Tune &t);
// one evaluation of the problems marked in h_active at their zt rows;
// synchronises; per-problem results in h_ist, global counters in h_st
cudaError_t evalset_run(EvalSet &E, scvt_stats *stats);
// time evaluations (best of two, events on E.stream) with tuning u; cold
// clears the radius hints first
cudaError_t evalset_time(EvalSet &E, const Tune &u, bool cold, float *ms, scvt_stats *stats);
scvt_status status_of_flags(unsigned f);

}  // namespace scvt
