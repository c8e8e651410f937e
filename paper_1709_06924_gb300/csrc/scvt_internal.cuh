// scvt_internal.cuh -- shared definitions of the CUDA library (not installed).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "df.cuh"
#include "scvt.h"

namespace scvt {

// NVTX range over the host code that enqueues one phase of the method (bin,
// topology, corners, quadrature, cell sums, reductions, direction, line
// search, accept); profilers project it onto the GPU work it launches.
// Header-only NVTX: a no-op unless a tool is attached.
struct Phase {
    explicit Phase(const char *name) { nvtxRangePushA(name); }
    ~Phase() { nvtxRangePop(); }
    Phase(const Phase &) = delete;
    Phase &operator=(const Phase &) = delete;
};

// a generator in bin order: 32-byte aligned (x, y, z, unused)
struct alignas(32) P4 {
    double x, y, z, w;
};

// ---- status bits written by the kernels (DevStatus::flags) ----
enum : unsigned {
    FLAG_BAD_POINT = 1u,      // non-finite or |z|^2 off 1 by more than 2e-12
    FLAG_DUPLICATE = 2u,      // two identical generators
    FLAG_UNBOUNDED = 4u,      // a cell reached the bounding box with every point considered
    FLAG_EXHAUSTED = 8u,      // a cell failed certification in the last retry pass
    FLAG_VMAX = 16u,          // polygon vertex capacity exceeded in the last pass
    FLAG_NONPOSITIVE = 32u,   // c_i . z_i <= 0
    FLAG_NONCONVEX = 64u,     // clip pattern with more than one outside run
    FLAG_EMPTY = 128u,        // clip removed every vertex
    FLAG_ECAP = 256u,         // the cells' edges exceed the edge list (6 per generator): neighbouring
                              // cells disagree on a Voronoi vertex (four or more cocircular generators)
};

// Device-side status of one evaluation; reset before each evaluation and
// copied to the host with the reduction results in a single transfer.
struct DevStatus {
    unsigned flags;
    unsigned retry_count[3];        // cells queued for retry pass 1, 2, (3 = failed)
    unsigned long long ambiguous;   // clip decisions within rounding of zero
    double red[4];                  // sum F_i, sum |g_i|^2, phi'(alpha), spare
    unsigned long long maxmove_bits;// max_i |s_i| as the bits of a nonnegative double
    double dots[4];                 // y.s, y.y, s.s, g.q
    unsigned differs;               // set by vec_differs
    unsigned long long ser_edges;   // edges whose density came from the density table
    unsigned long long ser_terms;   // their series' terms, summed
    unsigned max_bin;               // generators in the fullest cube-map bin (per problem in a batch)
};

struct Density {
    int kind;
    double gamma, alpha, beta;
    double xc0, xc1, xc2;
    double inv_alpha;  // 1 / alpha, divided once on the host
};

// the density in FP32 for the mixed-precision quadrature (inv_alpha = 1/alpha)
// The density's direction as a double-float vector (x_c for the tanh cap,
// e_z for X3) and its constants 1 - gamma, gamma: the double-float
// quadrature's view of a density, converted once per problem.
struct DensDF {
    df3 ev;
    df g1, gam;
};
__host__ __device__ inline DensDF dens_df(const Density &r) {
    DensDF d;
    d.ev = (r.kind == 1) ? df3{df{0.0f, 0.0f}, df{0.0f, 0.0f}, df{1.0f, 0.0f}} : df3_from(r.xc0, r.xc1, r.xc2);
    d.g1 = df_from(1.0 - r.gamma);
    d.gam = df_from(r.gamma);
    return d;
}

struct DensityF {
    int kind;
    float gamma, beta, inv_alpha, xc0, xc1, xc2;
};

// The density at a unit vector p, directly from its definition: 1; X3
// (1 - gamma) z^4 + gamma; the tanh cap on the geodesic distance d to x_c in
// its logistic form (1 - gamma) / (1 + exp(-2 (beta - d) / alpha)) + gamma,
// to the 4th power for kind 3.
__device__ __forceinline__ double rho_value(const Density &r, double px, double py, double pz) {
    if (r.kind == 0) return 1.0;
    if (r.kind == 1) {
        const double z2 = pz * pz;
        return (1.0 - r.gamma) * z2 * z2 + r.gamma;
    }
    const double cx = py * r.xc2 - pz * r.xc1, cy = pz * r.xc0 - px * r.xc2, cz = px * r.xc1 - py * r.xc0;
    const double d = atan2(sqrt(cx * cx + cy * cy + cz * cz), px * r.xc0 + py * r.xc1 + pz * r.xc2);
    const double inv_alpha = 1.0 / r.alpha;
    double v = (1.0 - r.gamma) / (1.0 + exp(-2.0 * (r.beta - d) * inv_alpha)) + r.gamma;
    if (r.kind == 3) {
        v = v * v;
        v = v * v;
    }
    return v;
}

// Density table of the FP64 forms (tanh-cap kinds).  The density depends on a
// point p only through c = x_c.p; the table holds, at M centres c_j =
// cos(theta_j), theta_j = j pi / (M - 1), the Taylor series of rho in
// u = c - c_j to kTabK terms, each with the radius r_j over which it was
// validated against the direct formula (0: none, evaluate directly).  Built
// once per density and problem size; each quadrature edge takes the centre
// nearest to its generator and as many terms as its own range of u needs.
constexpr int kTabK = 24;
struct alignas(32) TabCentre {
    double c;      // c_j = cos(theta_j)
    double r;      // validated radius r_j (0: none)
    float scale;   // 2^-e_j, the scale of the double-float coefficients (2^e_j >= r_j)
    float rf;      // r_j in FP32
    float K;       // terms at r_j
    float pad;
};
struct DensTab {
    int M;              // centres; 0 = no table (direct evaluation)
    float dth;          // theta spacing pi / (M - 1)
    const TabCentre *meta;  // per centre
    const double *cf;   // M x kTabK coefficients of the series in u
    const float2 *cdf;  // M x kTabK the same as double-float pairs, coefficients of the series in u 2^-e_j
    const float *mag;   // M x kTabK |cf_k| r_j^k in FP32 (the term count for a range |u| <= U <= r_j)
};
// centres for a problem of n generators; device bytes of a table of M centres
int dens_table_centres(int64_t n);
size_t dens_table_bytes(int M);
// build the table of density r (kinds 2 and 3) in buf (dens_table_bytes(M)
// bytes, 256-byte aligned) on stream s; *out describes it
cudaError_t dens_table_build(const Density &r, int M, void *buf, DensTab *out, cudaStream_t s);

// One problem of a batch: its generators occupy positions (and original
// indices) [p0, p0 + n) of the concatenated arrays, its G x G x 6 bins start
// at bin0 of the concatenated bin array.
struct InstGeom {
    int p0, n, G, bin0;
};

// Geometry of one evaluation (device pointers).  A single problem uses n, G,
// bstart, rho0 and the caller's status block; a batch of problems sets inst
// (with pinst: the problem of each position), per-problem densities and
// per-problem status blocks, and may mark problems inactive (their cells are
// skipped and their results left untouched).
struct Grid {
    int n;                  // generators (all problems)
    int G;                  // bins per face edge (single problem)
    int nbins;              // bins (all problems)
    const P4 *zs;           // generators in bin order (w unused)
    const float4 *zf;       // the same, rounded to FP32 (hi part); w = search-radius hint (0 = none)
    const float4 *zl;       // FP32 remainder z - hi (lo part): hi + lo carries ~48 bits
    const float4 *zll;      // the third part z - hi - lo (hi + lo + ll == z exactly) and, in w,
                            // |z|^2 - 1 from exact products and sums, rounded to FP32
    const int *sidx;        // bin-order position -> original index
    const int *bstart;      // nbins + 1 offsets into zs
    Density rho0;           // density of a single problem
    DensityF rho0f;
    DensTab tab0;           // its density table (M = 0: none)
    int fan;                // 1: one triangle (z_i, v_a, v_b) per Voronoi edge
    // batch of problems (all null for a single problem)
    const InstGeom *inst;   // per problem
    const int *pinst;       // problem of each position / original index
    const Density *rho;     // per-problem densities
    const DensityF *rhof;
    const DensDF *rhodf;    // the same as double-float constants (FP64 form)
    const DensTab *tabs;    // per-problem density tables
    DevStatus *ist;         // per-problem status (flags, sums)
    const int *active;      // per-problem: evaluate (1) or skip (0); null = all
    int nprob;              // problems of a batch (inst, ist, active have nprob entries)
};

// Per-cell outputs, indexed by ORIGINAL generator index.  Any may be null.
struct CellOut {
    double *grad;    // 3n
    double *hdiag;   // n
    double *mass;    // n
    double *moment;  // 3n
    double *fcell;   // n
    int *deg;        // n
    int *nbr;        // n * max_deg (original ids)
    int max_deg;
    float *radius;   // n, kNN search radius hint of the next evaluation (in/out)
};

// Certified cells between the topology and quadrature kernels, in bin
// order: deg (0 = integrated elsewhere or failed), corners (offsets v - z_i
// from the cell's generator) and the bin-order index of the neighbour across
// edge k (corner k -> k+1).
constexpr int kCellSlots = 16;

struct CellBuf {
    int *deg;          // n
    P4 *vx;            // n * kCellSlots
    int *nb;           // n * kCellSlots
    int *eoff;         // n + 1: exclusive scan of deg (edge list offsets)
    int *ecell;        // 6n: cell of each edge
    int *scan_tmp;     // scratch of the scan over n (2 * (n / 2048 + 64) + 64 ints)
    double *eacc;      // 5 * 6n: per-edge sums (m, c or o, F), component-major; FP32 in the mixed form
    float4 *vo;        // n * kCellSlots corner offsets v - z_i in FP32 (mixed precision only)
    float4 *ctab;      // n (FP64 form): the cell's density-table centre j (int bits, -1: none), its
                       // scale 2^-e_j, and x_c.z_i - c_j as a double-float pair
};

// ---- binning (cells.cu) ----
// g supplies n, G / nbins and the batch fields (inst, pinst, ist); zs, zf,
// zl, sidx and bstart (= start) are written here.  hint (nullable): search
// radius per original index, carried into zf[].w
void bin_points(const double *z, const Grid &g, int *bin_of, int *count, int *start, int *cursor, int *scan_tmp,
                P4 *zs, float4 *zf, float4 *zl, float4 *zll, int *sidx, const float *hint, DevStatus *st, cudaStream_t s,
                int64_t *launches);

// Launch shape and search parameters of an evaluation.  None of them changes
// a result: the cell of a generator is unique, its corners are computed from
// its neighbour triples and its sums are taken in its own edge order.
struct Tune {
    int bin_load = 2;      // target generators per bin: G = ceil(sqrt(n / (6 bin_load)))
    int knn_target = 24;   // candidates aimed at by the first radius without a hint
    int topo_warps = 4;    // warps per block of the topology pass (2, 4, 8)
    int topo_bpsm = 16;    // grid cap of the topology pass, blocks per SM
    int topo_lanes = 32;   // lanes per cell in the topology pass (32, 16)
    int chunks = 3;        // cell pipelines run concurrently on forked streams (1..kMaxChunks)
    int quad_block = 256;  // threads per block of the quadrature (128, 256, 512)
};
int bins_per_edge(int64_t n, int bin_load);
// largest bins per face edge the workspace of a problem of n generators holds
// (twice the finest tuning's: four times its bins)
inline int max_bins_per_edge(int64_t n) { return 2 * bins_per_edge(n, 1); }
// Bins per face edge for the next evaluation.  G0 = bins_per_edge(n,
// bin_load) suits generators spread evenly; where the last evaluation's
// fullest bin (max_bin generators with Gcur bins per edge) shows them
// concentrated beyond a uniform spread's fluctuations -- a converged mesh of
// a graded density -- the bins are refined so the dense region's bins hold
// about bin_load again: G = G0 sqrt(M0 / (6 bin_load)), M0 = max_bin
// (Gcur / G0)^2, within [G0, Gmax], kept at Gcur unless it moves by more
// than 15 %.  The bins do not change any result, only the search's cost.
int adapt_bins(int G0, int Gcur, int Gmax, unsigned max_bin, int bin_load);
// public tuning record <-> Tune (SCVT_ERR_INVALID when out of range)
scvt_status tune_from(const scvt_tuning &t, Tune *out);
scvt_tuning tuning_of(const Tune &t);

// ---- cell passes (cells.cu) ----
// topology pass 0 over all cells, passes 1..2 over the retry lists, then the
// quadrature kernel over all cells (timed by ev0/ev1 when given).
// mixed: corners and quadrature in FP32 local coordinates, FP64 accumulation
// Concurrent cell pipelines: up to kMaxChunks chunks of cells, the first on
// the caller's stream, the others on n_aux auxiliary streams forked from it
// (fork / join events; rebased[c]: chunk c's first edge and edge count are
// known, which chunk c + 1 waits for); counts: 8 * kMaxChunks device words
// (per chunk: the retry counts of the three passes, the edge count, the
// first edge), cleared by every evaluation.  cb.scan_tmp holds kMaxChunks
// scan scratch areas.
constexpr int kMaxChunks = 4;
struct Pipes {
    int n_aux = 0;
    cudaStream_t aux[kMaxChunks - 1] = {};
    cudaEvent_t fork = nullptr, join[kMaxChunks - 1] = {}, rebased[kMaxChunks - 1] = {};
    unsigned *counts = nullptr;
};
cudaError_t pipes_create(Pipes &px, int n_aux);
void pipes_destroy(Pipes &px);
inline size_t scan_tmp_ints(int64_t n) { return (size_t)kMaxChunks * (2 * ((size_t)n / 2048 + 64) + 64); }

// topo_ev (nullable): two events recorded around the first topology pass,
// like ev0 / ev1 around the quadrature, when the cells run as one pipeline
// precision: 0 = FP64 form (corners and rule points in double-float relative to z_i), 1 = mixed (FP32
// corners and quadrature, FP64 sums), 2 = plain FP64 (corners and rule points in FP64 arithmetic)
void cell_passes(const Grid &g, const CellOut &out, const CellBuf &cb, int *list1, int *list2, DevStatus *st,
                 int precision, const Tune &t, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, int64_t *launches,
                 int64_t *cell_launches, const Pipes *px, const cudaEvent_t *topo_ev = nullptr);
Density to_device_density(const scvt_density &r);
// exclusive scan of len ints (tmp: 2 * (len / 2048 + 64) + 64 ints)
void exclusive_scan(const int *in, int *out, int len, int *tmp, cudaStream_t s, int64_t *launches);
DensityF to_density32(const Density &d);

// ---- bisection refinement and mesh quality (refine.cu) ----
// deg / nbr: neighbour cycles with original ids, at most maxd per cell;
// cnt, off: n ints of scratch; scan_tmp as for exclusive_scan.  *n_out /
// *n_tri receive the sizes; nothing is written when they exceed cap.
cudaError_t bisect_midpoints(int n, const double *z, const int *deg, const int *nbr, int maxd, int *cnt, int *off,
                             int *scan_tmp, double *out, int64_t cap, int64_t *n_out, cudaStream_t s);
cudaError_t mesh_quality(int n, const double *z, const int *deg, const int *nbr, int maxd, int *cnt, int *off,
                         int *scan_tmp, double *cellq, double *triq, int64_t cap, int64_t *n_tri, cudaStream_t s);

// ---- reductions and vector kernels (lbfgs.cu) ----
int reduce_blocks(int64_t n);
// red[0] = sum fcell, red[1] = sum |g|^2, red[2] = sum g_i.q_i nrm_i (if q), nrm_i = 1 / |z_i + alpha q_i|
void reduce_eval(int n, const double *fcell, const double *grad, const double *q, const double *nrm,
                 double *partials, DevStatus *st, cudaStream_t s, int64_t *launches);
// the same per problem of a batch: problem b sums its own range with the
// chunking a single problem of its size uses (reduce_blocks(n_b) chunks, the
// chunk sums stored from partials + 4 * pbase[b]) into ist[b].red; inactive
// problems are skipped.  max_nb = max_b reduce_blocks(n_b); inst, pbase and
// active are device arrays.
void reduce_eval_batch(int nprob, int max_nb, const InstGeom *inst, const int *pbase, const int *active,
                       const double *fcell, const double *grad, const double *q, const double *nrm, double *partials,
                       DevStatus *ist, cudaStream_t s, int64_t *launches);
// out[slot] = sum x.y (deterministic), optionally scaled: out[slot] = scale[si] * sum
void dot_to(int64_t len, const double *x, const double *y, double *partials, double *out, cudaStream_t s,
            int64_t *launches);
// zt = (z + alpha q) / |z + alpha q| per generator, nrm = 1 / |z + alpha q|
void trial_point(int n, const double *z, const double *q, double alpha, double *zt, double *nrm, cudaStream_t s,
                 int64_t *launches);
void lloyd_project(int n, const double *c, double *zout, cudaStream_t s, int64_t *launches);
void accept_pair(int n, const double *zt, const double *z, const double *gt, const double *g, double *S, double *Y,
                 double *partials, DevStatus *st, cudaStream_t s, int64_t *launches);
// Scratch of one direction (kTwoLoopScratch doubles): the scalars alpha_k,
// the coefficients alpha_k - beta_k, the products s_k.g, and the ticket
// counters of the passes whose last block finishes a reduction.
constexpr int kScalAlpha = 0, kScalCoef = 64, kScalU = 128, kScalTicket = 192, kScalAcceptTicket = 193;
constexpr int kTwoLoopScratch = 200;
// q = -H g by the two-loop recursion one step per pass; pairs are given
// oldest first as host arrays of device pointers, rho[k] -> 1/(y_k.s_k) on
// the device; count <= 64.  Leaves g.q in st->dots[3]; partials: 1024
// doubles.  H0 = diag(h) per generator, or (h null) hs[0] I, or (both null) I.
void two_loop(int n, const double *g, const double *h, const double *hs, int count, const double *const *S,
              const double *const *Y, const double *const *rho, double *q, double *partials, double *scal,
              DevStatus *st, cudaStream_t s, int64_t *launches);
// ---- segmented LBFGS kernels over the problems of a batch (lbfgs.cu) ----
// A problem's LBFGS memory holds up to kLaneMaxM pairs in kLaneMaxM + 1
// history slots.  Its kLaneRho scalars: 1/(y.s) per slot, then gamma (plain
// LBFGS), then s_k.g per slot as the last gathered direction formed it, then
// the products s_a.y_b of the stored pairs by slot (rho[kLaneGram + a
// kGramDim + b], a older than b).
constexpr int kLaneMaxM = 32;
constexpr int kGramDim = kLaneMaxM + 1;
constexpr int kLaneSg = kLaneMaxM + 2;
constexpr int kLaneGram = kLaneSg + kGramDim;
constexpr int kLaneRho = kLaneGram + kGramDim * kGramDim;
// Directions with 1 .. kCmpMax pairs take the three gathered passes; the
// others one pass per step of the recursion.  Chunk sums of the gathered
// passes: kCmpQ per chunk.
constexpr int kCmpMax = 8;
constexpr int kCmpQ = 16;
// One problem of a batch as the segmented kernels see it.  Each problem
// keeps the chunking of a single problem of its size (nb3 chunks of its 3n
// direction components, nb1 chunks of its n generators), so its results
// are bit for bit those of the single-problem kernels.
struct SegLane {
    int64_t row;                  // first row of the problem in the evaluation workspace
    int n;                        // generators
    int count;                    // pairs in this round's direction
    int method;                   // 0 Lloyd-preconditioned LBFGS, 1 plain LBFGS, 2 Lloyd
    int m;                        // LBFGS memory
    int dir, trial, accept;       // takes part in the direction, the line-search round, the accept
    int nb3, blk3, nb1, blk1;     // chunks, and the problem's first block in the segmented grids
    int spare;                    // history slot that receives the accepted pair
    int new_pair;                 // the newest pair was stored after the last direction
    int slots[kLaneMaxM];         // history slots of the direction's pairs, oldest first
    double alpha;                 // trial step of the line-search round
    double *z, *g, *h;            // resident iterate, gradient, preconditioner
    double *hist, *yhist;         // S of slot k at hist + k slot_stride, Y at yhist + k slot_stride
    int64_t slot_stride;
    double *rho;                  // kLaneRho scalars
    double *scal;                 // kTwoLoopScratch
    double *partials;             // max(kCmpQ nb3, 4 nb1) chunk sums
    DevStatus *st;                // the problem's status block
};
// q = -H g for one problem described by a lane (row 0 of q): the gathered
// passes for 1 .. kCmpMax pairs, else two_loop(); g.q in st->dots[3]
void lane_direction(const SegLane &L, double *q, cudaStream_t s, int64_t *launches);
// the products s_a.y_b (a < b) of pairs 0 .. count-1 of a lane whose history
// holds no products yet, as dot products (a solver's are formed by its
// directions); count <= kCmpMax
void lane_pair_products(const SegLane &L, cudaStream_t s, int64_t *launches);
// q of every problem taking part (rows of q_rows): the gathered passes for
// the problems with 1 .. kCmpMax pairs (three launches if any), then
// 2 max_step_count + 1 step passes for the others (none if max_step_count <
// 0); each launch over nblk3 = sum nb3 blocks; g.q in each problem's
// st->dots[3]
void seg_direction(const SegLane *lanes, int nl, bool any_gathered, int max_step_count, int nblk3, double *q_rows,
                   cudaStream_t s, int64_t *launches);
// zt = normalize(z + alpha q) for the rows of the problems of the round
// (pinst: problem of each row)
void seg_trial(const SegLane *lanes, const int *pinst, int64_t ntot, const double *q_rows, double *zt_rows,
               double *nrm_rows, cudaStream_t s, int64_t *launches);
// accepted pairs: s = zt - z, y = gt - g into the spare slot, y.s, y.y, s.s
// and max |s_i| into st->dots / maxmove_bits, 1/(y.s) (and gamma) when the
// curvature test passes, then z, g, h take the trial point's values; one
// launch over nblk1 = sum nb1 blocks
void seg_accept(const SegLane *lanes, int nl, int nblk1, const double *zt_rows, const double *gt_rows,
                const double *ht_rows, cudaStream_t s, int64_t *launches);

// gamma_dev[0] = y.s / y.y from st->dots (plain LBFGS scaling)
void set_gamma(double *gamma_dev, const DevStatus *st, cudaStream_t s, int64_t *launches);
void set_rho(double *rho_dev, int k, const DevStatus *st, cudaStream_t s, int64_t *launches);
// st->differs = 1 if a[i] != b[i] for some i < len (bitwise on the values)
void vec_differs(int64_t len, const double *a, const double *b, DevStatus *st, cudaStream_t s, int64_t *launches);

}  // namespace scvt
