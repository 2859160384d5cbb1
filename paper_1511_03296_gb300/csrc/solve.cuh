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
    const uint32_t* nbrp;      // 5 x Vtot, packed 16-bit offsets (-1 and +1 per dimension)
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
    float* rlo;                // low part of r (compensated variant)
    float* d[2];
    float* q;
    float* aux[2];             // single-reduction form: s = A p by iteration parity
    // reductions
    Scal* scal;                // sum_k C_k
    float2* part_rs[2];        // sum_k C_k * ntiles_k double-float tile partials of r^T M^-1 r
    float2* part_dq;           // ... of d^T A d
    float2* part_mu[2];        // single-reduction form: partials of w^T u by parity
    uint32_t* err;
};

struct SolvePlan {
    int mode;                  // SplatMode
    int outer_iters;           // 1, or the IRLS count
    int pcg_iters;
    float sigma_gm;
    int chan_block;            // channels per tile pass (1..4)
    int cmax;                  // most channels of any image
    int64_t max_pixels;        // largest image
    int64_t max_cv;            // largest C x V block
    bool export_y;
    int comp;                  // 1: compensated residual / recomputed q variant
    int persistent;            // 1: the whole PCG loop in one cooperative launch when the
                               //    resident form fits (or always, with force_persistent)
    int force_persistent;
    unsigned* barrier;         // kBarrierWords words of grid-barrier state (persistent loop)
    int inject_timeout;        // preset the barrier counter so no wait completes (test)
    int single;                // 1: single-reduction PCG form (FP32, Cp <= 4, per-phase)
    int block_mult;            // per-phase kernels: blocks = min(tiles, SMs x occupancy x this)
};

// A solve runs as segments: for each outer (IRLS) iteration a setup (splat,
// diag(A), flat init, initial residual) and the PCG loop, then the output
// (slice / y export, or the backward adjoints).  `mode` is the splat mode of
// a setup segment.
enum Segment : int { kSegSetup = 0, kSegLoop = 1, kSegOut = 2 };
cudaError_t launch_segment(const SolveArgs& A, const SolvePlan& P, int seg, int mode,
                           cudaStream_t s);

// true when every vertex tile can have its own co-resident block of the
// resident persistent PCG loop and no image has more channels than a pass
bool resident_fits(const SolveArgs& A, const SolvePlan& P);

// the automatic launch policy's choice of the resident loop: it fits and the
// batch has at most one vertex tile per SM (measured: with more tiles the two
// grid barriers per iteration cost more than graph-replayed phase launches)
bool resident_preferred(const SolveArgs& A, const SolvePlan& P);

}  // namespace fbs
