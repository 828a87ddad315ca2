#pragma once
#include "far_internal.cuh"

namespace far {

struct Pose16 {
    double m[16];
};

struct GnArgs {
    MapView map;                 // registration map (points + covariances)
    const float4* src;           // source points (sensor frame), w = local rank
    const float4* src_cov;       // two float4 per source point, valid flag in [1].z
    const u32* n_src;            // device count of source points
    u32 n_max;                   // upper bound of n_src (grid sizing)
    RegState* st;
    double* partials;            // gn_partials_doubles(n_max)
    float tau2, kappa2;
    double conv_eps;
    int update;                  // 0: linearise only (stage entry point)
    int32_t* corr_out;           // optional per-source correspondence ids
    unsigned long long budget_ns;  // 0: no time cap
    int tpp;                     // lanes per source point in the search: 1, 4, 8 or 32 (other: default)
    // Linearisation anchor A (world): J = [[q - A]x, -I] and T <- exp(xi) T about A. Zero for plain
    // maps; for the precision variant the corner of the tile holding the initial position,
    // with ftile that tile (the search frame of the iteration).
    double anchor[3];
    int ftile[3];
    // initial sensor position relative to the anchor: the termination test measures the
    // increment there (see the solve)
    double conv_center[3];
    // precision variant source covariances (FP16 with the scan-local voxel's exponent)
    const uint2* src_h4;
    const u32* src_h2;
    const signed char* src_exp;
    u32 max_iters;               // updates at most (device-side loop of gn_graph)
};

// One problem of a batched registration: its arguments and its share of the shared grid.
struct BatchProblem {
    GnArgs args;
    u32 block_begin;   // first block of the batched linearisation grid owned by this problem
    u32 nblocks;       // number of blocks it owns (its partials hold nblocks entries per value)
};

// Batched Gauss-Newton: one linearisation launch and one solve launch per iteration for all
// problems; every problem stops on its own flag.
u32 gn_threads_per_block();
cudaError_t gn_batch_begin(const BatchProblem* probs, u32 nprob, const double* init, cudaStream_t s);
cudaError_t gn_batch_iteration(const BatchProblem* probs, const u32* block_prob, u32 total_blocks, u32 nprob,
                               int tpp, bool prec, cudaStream_t s);   // prec: every problem's map is precision mode
cudaError_t gn_batch_gather(const BatchProblem* probs, u32 nprob, RegState* out, cudaStream_t s);

// Supported lanes-per-point value for a request (unsupported values map to the default).
int gn_tpp(int requested);
u32 gn_grid(u32 n_upper, int tpp);
size_t gn_partials_doubles(u32 n_upper);
u32 gn_max_blocks(u32 n_upper);   // largest grid gn_grid returns for n_upper points, any lanes per point
// Reset the registration state to `init`; n_src (device, may be null) is recorded in st->n_src.
cudaError_t gn_begin(RegState* st, const double init[16], const u32* n_src, cudaStream_t s);
// One Gauss-Newton iteration = k_gn_lin (search, linearisation, block partials) then
// k_gn_solve (fixed-order FP64 reduction over 32 one-warp blocks, then Cholesky and SE(3)
// update by the last of them); once the state's stop flag is set both skip their work.
cudaError_t gn_iteration(const GnArgs& a, u32 n_upper, cudaStream_t s);
cudaError_t gn_linearise(const GnArgs& a, u32 n_upper, cudaStream_t s, u32* nblocks);
cudaError_t gn_solve(const GnArgs& a, u32 nblocks, cudaStream_t s);
// The Gauss-Newton loop as a CUDA graph with a device-side while loop (conditional node): the
// body is one linearisation and one solve, and the solve ends the loop once the state is done
// or max_iters updates were applied, so no launch follows convergence. Both kernels read the
// arguments from d_args (device memory), so one instantiated graph serves every registration
// with the same grid, lanes per point and precision mode.
struct GnGraph {
    cudaGraphExec_t exec = nullptr;
    u32 grid = 0;
    int tpp = -1;
    bool prec = false;
};
cudaError_t gn_graph_build(const GnArgs* d_args, u32 n_upper, int tpp, bool prec, GnGraph* out);
void gn_graph_destroy(GnGraph* g);

// Distinct map voxels (out2[0]) and their points (out2[1]) probed by the source points at st->T
// (searched in the frame of a.anchor / a.ftile as the linearisation does).
cudaError_t gn_footprint(const GnArgs& a, u32* touched, u32 cap, unsigned long long* out2, u32 n_upper,
                         cudaStream_t s);
// cov36 = H^-1 of the last linearisation in st (zeros when H is not positive definite).
cudaError_t gn_covariance(RegState* st, double* cov36, cudaStream_t s);

}  // namespace far
