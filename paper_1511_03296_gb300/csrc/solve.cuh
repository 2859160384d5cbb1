// Arguments of the solve kernels (passed by value to every launch).
#pragma once

#include "fbs_internal.cuh"

namespace fbs {

constexpr int kMaxLevels = 16;     // bilateral-space pyramid levels (12-bit fields: at most 13)
constexpr int kPyrMaxNc = 6;       // level-vector values per chunk of a pyramid sum
constexpr int kPyrTailThreads = 1024;

// The bilateral-space pyramid of a grid (supplement) and the per-solve
// arrays of the hierarchical preconditioner (Sec. 4).  Pyramid vertices are
// numbered level by level: level k occupies [off[k], off[k+1]), level 0 is
// the grid's vertices.  Values of levels >= 1 live in buf (W per vertex).
struct PyrDev {
    int K;                     // levels of the deepest image's pyramid (level 0 = the grid)
    int W;                     // channels of a level vector: the widest image's Cp
    int64_t off[kMaxLevels + 1];
    const int64_t* ioff;       // [K * (n_images + 1)]: image i's vertices on level k are
                               //   [ioff[k (n+1) + i], ioff[k (n+1) + i + 1]) (absolute)
    const uint8_t* kimg;       // [n_images]: levels of each image's own pyramid
    const int32_t* parent;     // [off[K-1]]: level-local parent (in level k+1) of each vertex below the top
    const int32_t* child_off;  // [off[K] - off[1] + 1]: children of level >= 1 vertex g are
    const int32_t* child_idx;  //   child_idx[child_off[g - off[1]] .. child_off[g - off[1] + 1])
                               //   (level-local indices in the level below, ascending)
    const uint16_t* vimg;      // [off[K]]: image of each pyramid vertex
    const float* cnt;          // [off[K]]: P(1), grid vertices below each pyramid vertex
                               //   (0 on the vertex an image keeps past its own top)
    const float* cinit;        // [off[K]]: initialisation weight w_init(k) / P(1) (0 likewise)
    float* coef;               // [off[K]]: preconditioner scale w(k) P(1) / P(diag A) (per solve)
    float* dg;                 // [off[1]]: diag(A) (per solve)
    float* scv;                // [off[1]]: S c (per solve)
    float2* lv;                // [(off[K] - off[1]) * nc]: level values (double-float hi,
                               //   lo), nc = W (+ 2 in the set-up) per vertex
    float* z;                  // CG vector layout: z = M_hier^-1 r
};

struct SolveArgs {
    const VTile* vt;
    int nvt;
    const InstDev* inst;
    int ninst;
    // grid
    const int32_t* nbr;        // 10 rows of nbr_stride, global vertex ids, -1 if absent
    int64_t nbr_stride;        // row stride of nbr (>= Vtot: the grid's vertex capacity)
    const uint32_t* nbrp;      // 3 x Vtot, packed offsets (8-bit x, l, u, v; 16-bit y)
    int64_t Vtot;
    const double* n64;         // bistochastisation vector n
    const uint32_t* m;         // counts
    const uint32_t* pstart;    // first sorted-pixel slot of each vertex
    const uint32_t* perm;      // sorted slot -> global pixel
    const uint32_t* vid;       // global pixel -> global vertex
    // per-vertex problem data
    float* a;                  // a' = lambda (m - n o Bbar n) + S c (Laplacian-form remainder)
    float* alo;                // low part of a' as a double-float pair, or nullptr
    float2* nm;                // {n, M^-1}
    // vectors, all sum_k C_k V_k floats
    float* y;
    float* r;
    float* rlo;                // low part of r (compensated variant)
    float* d[2];
    float* q;
    float* aux[2];             // single-reduction form: s = A p by iteration parity
    float* ylo;                // low part of y as a double-float pair (aux[1]), or nullptr:
                               //   the robust solver in compensated precision
    float* zq;                 // z = M^-1 r (aux[0]) for the FP32 Jacobi phase 1, which
                               //   forms A d as A z + beta q_old (per-phase, persistent and
                               //   resident launches); nullptr in the other variants
                               //   (compensated, hierarchical, single reduction)
    const float* nf;           // n in FP32, dense (the neighbour weights of the z form)
    // reductions
    Scal* scal;                // sum_k C_k
    int nscal;                 // entries of scal
    int fin;                   // 1: finalised scalars (the resident loop) -- the block
                               //    that completes a phase's partials reduces them once
                               //    and stores the next phase's scalars; 0: every block
                               //    reduces an image's partials when it starts on it
    float2* part_rs[2];        // sum_k C_k * ntiles_k double-float tile partials of r^T M^-1 r
    float2* part_dq;           // ... of d^T A d
    float2* part_mu[2];        // single-reduction form: partials of w^T u by parity
    uint32_t* err;
    PyrDev pyr;                // hierarchical preconditioner (pyr.K = 0 when off)
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
    int hier;                  // 1: hierarchical preconditioner and initialisation (per-phase)
    int dfy;                   // 1: y and a' held as double-float pairs too (robust solver,
                               //    compensated precision)
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
