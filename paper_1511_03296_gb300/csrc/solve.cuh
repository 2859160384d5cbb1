// Arguments of the solve kernels (passed by value to every launch).
#pragma once

#include "fbs_internal.cuh"

namespace fbs {

struct SolveArgs {
    const VTile* vt;
    int nvt;
    const InstDev* inst;
    int ninst;
    // grid
    const int32_t* nbr;        // 10 x Vtot, global vertex ids, -1 if absent
    int64_t Vtot;
    const double* n64;         // bistochastisation vector n
    const uint32_t* m;         // counts
    const uint32_t* pstart;    // first sorted-pixel slot of each vertex
    const uint32_t* perm;      // sorted slot -> global pixel
    const uint32_t* vid;       // global pixel -> global vertex
    // per-vertex problem data
    float* a;                  // a' = lambda (m - n o Bbar n) + S c (Laplacian-form remainder)
    float2* nm;                // {n, M^-1}
    // vectors, all sum_k C_k V_k floats
    float* y;
    float* r;
    float* d[2];
    float* q;
    // reductions
    Scal* scal;                // sum_k C_k
    double* part;              // sum_k C_k * ntiles_k
    unsigned* cnt;             // 3 x ninst arrival counters (zero between launches)
    uint32_t* err;
};

struct SolvePlan {
    int mode;                  // SplatMode
    int outer_iters;           // 1, or the IRLS count
    int pcg_iters;
    float sigma_gm;
    int chan_block;            // channels per tile pass (1..4)
    int64_t max_pixels;        // largest image
    int64_t max_cv;            // largest C x V block
    bool export_y;
};

cudaError_t launch_solve(const SolveArgs& A, const SolvePlan& P, cudaStream_t s);

}  // namespace fbs
