/*
 * fbs.h -- C ABI of the GB300 Fast Bilateral Solver library (libfbs.so).
 *
 * The library runs the data-parallel hot path of the bilateral solver
 * (Barron & Poole, "The Fast Bilateral Solver") on one sm_103a GPU:
 *   quantised 5-D keys -> simplified bilateral grid (splat map S, +-1
 *   neighbour tables) -> bistochastisation (D_n, D_m) -> Jacobi-PCG on
 *   A y = b -> slice x = S^T y, plus the robust (IRLS) loop and the
 *   backward pass.
 *
 * Conventions for every call:
 *   - Array arguments are DEVICE pointers owned by the caller, unless a
 *     parameter says "host".  The library never frees caller memory.
 *   - A grid handle owns its own device memory until fbs_grid_destroy.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream).  Calls return once the work is enqueued,
 *     except where a call says it synchronises.
 *   - Argument errors return at once and enqueue nothing.  Errors found on
 *     the device (key field out of range, non-finite input, a bounded wait
 *     that ran out) are latched in the handle; fbs_grid_build reports its
 *     own, and fbs_grid_sync reports any latched error of later calls.
 *   - Images are planar float32: yuv is 3 x H x W (plane 0 luma l, plane 1
 *     u, plane 2 v), targets are C x H x W, confidences H x W, all
 *     row-major with pixel index row * W + col.
 *   - Bilateral-space vectors of image k are C_k x V_k (channel-major);
 *     V_k is reported by fbs_grid_info.
 */
#ifndef FBS_H_
#define FBS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FBS_OK = 0,
    FBS_ERR_ARG = 1,        /* invalid argument (null pointer, bad size, sigma <= 0, ...) */
    FBS_ERR_RANGE = 2,      /* a quantised key field is outside [0, 4095] (or NaN input)  */
    FBS_ERR_OOM = 3,        /* device allocation failed                                    */
    FBS_ERR_CUDA = 4,       /* a CUDA runtime call failed                                  */
    FBS_ERR_TIMEOUT = 5,    /* a bounded device-side wait ran out                          */
    FBS_ERR_NONFINITE = 6,  /* NaN or Inf in a target or confidence                        */
    FBS_ERR_STATE = 7       /* call out of order (e.g. solve before bistochastize)         */
} fbs_status;

typedef struct fbs_grid fbs_grid;   /* opaque; library-owned device memory */

/* One reference image (Sec. 2: "a reference RGB image", affinity of Eq. (2)
 * measured in YUV with spatial, luma and chroma bandwidths). */
typedef struct {
    const float* yuv;     /* device, 3 x height x width float32, planar l, u, v */
    int height;
    int width;
    float sigma_xy;       /* > 0 */
    float sigma_l;        /* > 0 */
    float sigma_uv;       /* > 0 */
} fbs_image_desc;

/* One problem on one image of the grid (Sec. 2: target t, confidence c,
 * smoothness weight lambda; several targets share A, supplement Sec. 4). */
typedef struct {
    const float* t;       /* device, channels x H x W (target)                       */
    const float* c;       /* device, H x W (confidence, >= 0)                        */
    float* x;             /* device, channels x H x W output (sliced solution), or NULL */
    float* y;             /* device, channels x V output (bilateral-space solution y),
                             or NULL; the backward pass reads it as the saved y-hat   */
    int channels;         /* 1 .. 64 */
    float lambda;         /* >= 0 */
} fbs_problem_desc;

/*
 * fbs_grid_build -- simplified bilateral grid of one or more images
 * (Sec. 2, Eq. (3)-(5); supplement Eq. (5): S S^T = D_m).
 *
 * Each pixel gets the integer key floor(p / sigma + 1/2) per coordinate
 * p = (col, row, l, u, v) with sigma = (sigma_xy, sigma_xy, sigma_l,
 * sigma_uv, sigma_uv); vertices are the distinct keys of each image in
 * ascending order of the packed key (row, col, l, u, v), so vertex ids are
 * canonical.  Builds the pixel -> vertex map, the counts m = S 1 and the
 * +-1 neighbour table along each of the 5 dimensions.
 *
 * imgs: host array of n_images descriptors (the yuv buffers are device
 * memory and only need to live until this call returns).  *out receives a
 * new handle.  SYNCHRONISES `stream` once (to size the vertex arrays).
 * Errors: FBS_ERR_ARG (null, n_images outside 1 .. 65535, non-positive
 * size or sigma, a grid cell of more than 16384 pixels, i.e. sigma_xy >
 * 127), FBS_ERR_RANGE
 * (a key field out of [0, 4095], including NaN / negative colours),
 * FBS_ERR_OOM, FBS_ERR_CUDA.  On error *out is NULL.
 */
fbs_status fbs_grid_build(const fbs_image_desc* imgs, int n_images, void* stream,
                          fbs_grid** out);

/*
 * fbs_bistochastize -- supplement Alg. 1: n <- sqrt(n o m / (Bbar n))
 * repeated `iters` times (iters >= 1) from n = 1, in FP64, where
 * Bbar = 10 I + (sum over the +-1 neighbours), the [1, 2, 1] blur summed over
 * the 5 dimensions.  Stores D_n in the handle.  Must precede any solve.
 */
fbs_status fbs_bistochastize(fbs_grid* g, int iters, void* stream);

/*
 * fbs_solve -- the bilateral solver forward pass (Sec. 2, Eq. (6)-(8);
 * Sec. 4 Jacobi preconditioner and flat initialisation; supplement Alg. 2).
 * For each image k: b = S(c o t), A = lambda (D_m - D_n Bbar D_n) + diag(S c),
 * y0 = b / S c, then `pcg_iters` PCG iterations per channel (all channels
 * and all images advance together, one launch per CG phase), then
 * x = S^T y.  probs: host array with one entry per image of the grid.
 * FP32 vectors; dot products reduced with FP64 accuracy.
 */
fbs_status fbs_solve(fbs_grid* g, const fbs_problem_desc* probs, int pcg_iters, void* stream);

/*
 * fbs_solve_lowrank -- the forward pass of a wide target through the
 * low-rank reduction of the supplement (multiple output channels):
 * for each image, B = S(c o t) (V x C) is factored by a column-pivoted QR
 * B P = Q R; the rows of R P^T are ranked by their squared norm ("mass",
 * ties in pivot order) and the fewest leading rows whose mass reaches
 * (1 - eps) of |B|_F^2 are kept (t of them, the image's rank); the reduced
 * system A Y~ = Q~ (the kept columns of Q) is solved with `pcg_iters`
 * PCG iterations per column, exactly as fbs_solve solves a t-channel target
 * (with the grid's preconditioner option), and x = S^T (Y~ R~) with R~ the
 * kept rows.  R and P are formed on
 * the host from the pivoted Cholesky factorisation of the Gram matrix
 * B^T B (accumulated on the GPU with FP64 accuracy); a pivot at or below
 * 1e-13 of the largest column mass ends the factorisation (numerically
 * dependent columns have mass 0).  probs[k].x (C x N, device) receives x;
 * probs[k].y must be NULL.  eps in [1e-12, 1); the paper uses 0.01.
 * ranks: host array of n_images receiving t per image (0 when B = 0, then
 * x = 0), or NULL.  SYNCHRONISES `stream` (twice: to read the Gram matrices
 * back and at the end).  Errors: FBS_ERR_ARG (as fbs_solve, plus eps out of
 * range, a NULL x or a non-NULL y), FBS_ERR_STATE (inside a stream capture,
 * or before fbs_bistochastize), FBS_ERR_OOM, FBS_ERR_CUDA.
 */
fbs_status fbs_solve_lowrank(fbs_grid* g, const fbs_problem_desc* probs, int pcg_iters,
                             double eps, int* ranks, void* stream);

/*
 * fbs_domain_transform -- the edge-aware post-filter the paper runs on the
 * solver's output (Sec. 5: it smooths the blocky artefacts of the
 * simplified grid; Gastal and Oliveira 2011, recursive formulation).
 * guide: 3 x height x width (device, planar; its values set the edges, in
 * the units sigma_r is given in), x: channels x height x width (device),
 * filtered in place.  With d = 1 + (sigma_s / sigma_r) sum_c |dI_c| the
 * step length between horizontally (vertically) adjacent pixels, iteration
 * i = 1 .. iterations filters every row and then every column forward and
 * backward with J[k] <- (1 - a^d) J[k] + a^d J[k -/+ 1], a = exp(-sqrt(2) /
 * sigma_i), sigma_i = sigma_s sqrt(3) 2^(iterations - i) /
 * sqrt(4^iterations - 1).  FP32.  Errors: FBS_ERR_ARG (NULL buffers,
 * non-positive sizes or sigmas, iterations outside 1 .. 16, width above
 * 28000), FBS_ERR_OOM, FBS_ERR_CUDA.
 */
fbs_status fbs_domain_transform(const float* guide, int height, int width, float* x, int channels,
                                float sigma_s, float sigma_r, int iterations, void* stream);

/*
 * fbs_solve_robust -- robust bilateral solver with the Geman-McClure loss
 * (supplement Sec. 3, Alg. 3): c <- c_init (probs[k].c); repeat irls_iters
 * times { x <- solve(t, c); e <- x - t; c <- 2 s^2 / (s^2 + e^2)^2 } with
 * s = sigma_gm; each solve starts from the flat initialisation of the
 * current weights.  channels must be 1.  probs[k].x / .y receive the last
 * solve's x / y.
 */
fbs_status fbs_solve_robust(fbs_grid* g, const fbs_problem_desc* probs, float sigma_gm,
                            int irls_iters, int pcg_iters, void* stream);

/*
 * fbs_solve_backward -- backward pass through the solver (Sec. 3):
 *   dL/db = A^-1 (S dL/dx)            (PCG, same A, flat-initialised)
 *   dL/dt = c o S^T dL/db
 *   dL/dc = sum over channels [ S^T(-dL/db o y) + (S^T dL/db) o t ]
 * probs[k].y must hold the forward solution y-hat (channels x V).
 * dL_dx[k], dL_dt[k]: device, channels x H x W; dL_dc[k]: device, H x W.
 * The host arrays dL_dx, dL_dt, dL_dc have one entry per image.
 */
fbs_status fbs_solve_backward(fbs_grid* g, const fbs_problem_desc* probs,
                              const float* const* dL_dx, float* const* dL_dt,
                              float* const* dL_dc, int pcg_iters, void* stream);

/*
 * fbs_set_option -- per-grid settings for later solves (host-side; no
 * device work).  Errors: FBS_ERR_ARG for an unknown option or value.
 *
 * FBS_OPT_VECTOR_PRECISION: how the CG state is held (the paper fixes no
 * precision; every variant keeps the CG inner products FP64-accurate):
 *   FBS_VECTORS_FP32         y, r, d, q in FP32; A d computed in FP32 (with
 *                            the Jacobi preconditioner, from the second PCG
 *                            iteration as A z + beta q_old with z = M^-1 r,
 *                            equal to A d up to rounding).
 *   FBS_VECTORS_COMPENSATED  y, d in FP32; the residual r as a pair of FP32
 *                            values (double-float) and q = A d recomputed in
 *                            the update phase with error-free products, so
 *                            r <- r - alpha A d carries no rounding of q
 *                            (the FP32 A d of the first phase only enters
 *                            d^T q, i.e. the step length).  Same vector bytes
 *                            per channel, one more neighbour-table pass per
 *                            iteration.  In
 *                            fbs_solve_robust y and the diagonal remainder of
 *                            A are double-float pairs too (the IRLS loop
 *                            amplifies their float32 rounding): 4 more bytes
 *                            per vertex and 8 per vertex and channel moved per
 *                            iteration.
 *   FBS_VECTORS_AUTO         (default) compensated for fbs_solve_backward,
 *                            FP32 for fbs_solve and fbs_solve_robust.
 * FBS_OPT_PCG_LAUNCH: how the PCG iterations are launched:
 *   FBS_PCG_AUTO             (default) FBS_PCG_PERSISTENT when the batch has
 *                            at most one vertex tile per SM and no image has
 *                            more than 4 channels (every tile then gets its
 *                            own co-resident block and its topology stays in
 *                            shared memory for the whole loop), else
 *                            FBS_PCG_PER_PHASE.
 *   FBS_PCG_PERSISTENT       all iterations in one cooperative launch whose
 *                            blocks meet at grid barriers (each wait bounded;
 *                            on time-out the solve stops and FBS_ERR_TIMEOUT
 *                            is latched).  Falls back to FBS_PCG_PER_PHASE when
 *                            the cooperative launch is refused or the stream
 *                            is being captured.
 *   FBS_PCG_PER_PHASE        two launches per iteration (replayed from a CUDA
 *                            graph when the same solve repeats).
 * FBS_OPT_PCG_FORM: which form of the Jacobi PCG (supplement Alg. 2) runs:
 *   FBS_PCG_FORM_STANDARD    (default) Alg. 2: two phases, two global
 *                            reductions per iteration.
 *   FBS_PCG_FORM_SINGLE      the single-reduction (Chronopoulos-Gear) form,
 *                            with the same iterates in exact arithmetic: u =
 *                            M^-1 r, w = A u and s = A p are carried along and
 *                            both inner products of an iteration are taken
 *                            together, so an iteration is one launch, or,
 *                            with the persistent style where every tile has a
 *                            co-resident block, one grid barrier.  Used for
 *                            FP32 vectors when no image has more than 4
 *                            channels; other solves keep the standard form.
 * FBS_OPT_PRECONDITIONER: the preconditioner and initial state (Sec. 4):
 *   FBS_PRECOND_JACOBI        (default) M^-1 = diag(A)^-1 and the flat
 *                             initialisation y0 = S(c o t) / S c.
 *   FBS_PRECOND_HIERARCHICAL  the bilateral-space pyramid (supplement):
 *                             M^-1 = P^T(w o P(1) o P(.) / P(diag A)) with
 *                             (alpha, beta) = (2, 5) and the push-pull
 *                             initialisation with (4, 0).  The pyramid is
 *                             built on the GPU on first use (one
 *                             synchronisation per level to read its size;
 *                             FBS_ERR_STATE if that first use is inside a
 *                             stream capture).  Any channel count;
 *                             per-phase launches, standard PCG form.
 * FBS_OPT_PHASE_BLOCKS: 1 (default), 2 or 4 -- the per-phase PCG kernels
 *   launch min(tiles, SMs x resident blocks per SM x value) blocks; above 1
 *   the blocks take shorter runs of tiles in several waves.
 * FBS_OPT_INJECT_BARRIER_TIMEOUT: value 1 makes the next persistent PCG
 *   loop start with its barrier counter preset so that no barrier can
 *   complete; every block waits out its bounded spin, latches
 *   FBS_ERR_TIMEOUT and returns (a test of the failure path; one-shot).
 * FBS_OPT_TUNE_SINGLE_SOLVE: 0 (default) or 1 -- what fbs_autotune times.
 *   0: repeated solves on this grid, whose per-phase launches are replayed
 *   from a CUDA graph captured on the second solve of a shape.  1: the
 *   first solve on a grid (the graphs are dropped before every timed
 *   solve, so per-phase launches go out one by one), for callers that
 *   build a new grid for every solve.
 */
enum { FBS_OPT_VECTOR_PRECISION = 1, FBS_OPT_PCG_LAUNCH = 2, FBS_OPT_INJECT_BARRIER_TIMEOUT = 3,
       FBS_OPT_PCG_FORM = 4, FBS_OPT_PHASE_BLOCKS = 5, FBS_OPT_PRECONDITIONER = 6,
       FBS_OPT_TUNE_SINGLE_SOLVE = 7 };
enum { FBS_PRECOND_JACOBI = 0, FBS_PRECOND_HIERARCHICAL = 1 };
enum { FBS_VECTORS_AUTO = 0, FBS_VECTORS_FP32 = 1, FBS_VECTORS_COMPENSATED = 2 };
enum { FBS_PCG_AUTO = 0, FBS_PCG_PERSISTENT = 1, FBS_PCG_PER_PHASE = 2 };
enum { FBS_PCG_FORM_STANDARD = 0, FBS_PCG_FORM_SINGLE = 1 };
fbs_status fbs_set_option(fbs_grid* g, int option, int value);

/*
 * fbs_autotune -- picks the PCG launch configuration for this grid and
 * problem shape by timing it.  The paper has no counterpart (it runs one CPU
 * configuration); it serves the batched solves (tile and block shapes
 * chosen by measurement rather than fixed).
 *
 * Runs fbs_solve(g, probs, pcg_iters) under each candidate -- launch style
 * (per-phase launches, or the persistent loop where its cooperative launch
 * fits; with the single-reduction form, the resident loop of that form),
 * PCG form (standard or single-reduction) and the per-phase block
 * count (FBS_OPT_PHASE_BLOCKS 1, 2, 4) -- each warmed up twice (so graph
 * replay is what gets timed; with FBS_OPT_TUNE_SINGLE_SOLVE set, the graphs
 * are dropped before each solve instead) and timed over three solves with
 * CUDA events on `stream`, then leaves the fastest set on the grid (fbs_set_option values)
 * and solves once more with it, so the output buffers in probs hold that
 * configuration's result.  *out, if not null, receives the choice and its
 * median solve time.  Synchronises `stream`.  Errors: as fbs_solve;
 * FBS_ERR_STATE while `stream` is being captured.
 */
typedef struct {
    int pcg_launch;        /* FBS_PCG_PER_PHASE or FBS_PCG_PERSISTENT */
    int pcg_form;          /* FBS_PCG_FORM_* */
    int phase_blocks;      /* FBS_OPT_PHASE_BLOCKS value */
    float solve_ms;        /* median time of one solve with this choice */
    int candidates;        /* configurations timed */
} fbs_tune_result;
fbs_status fbs_autotune(fbs_grid* g, const fbs_problem_desc* probs, int pcg_iters, void* stream,
                        fbs_tune_result* out);

/*
 * fbs_solve_static -- fbs_solve for callers that cannot allocate device
 * memory (a fixed memory budget handed over up front, a real-time loop that
 * must never enter an allocator, an embedding runtime whose own allocator
 * owns the device).  There is no counterpart in the paper: it is the same
 * forward solve, but every piece of scratch (CG vectors, diag(A), inner
 * product partials, grid-barrier words, image descriptors) comes from one
 * 64 MiB array compiled into the library, and the call allocates nothing.
 * The grid (built earlier by fbs_grid_build) and all inputs and outputs
 * are the caller's, with the same meaning as for fbs_solve; the CG state is
 * FP32 unless FBS_OPT_VECTOR_PRECISION selects the compensated variant, and
 * no CUDA graph is used.  It always solves with the Jacobi preconditioner
 * and the flat initialisation in the standard PCG form
 * (FBS_OPT_PRECONDITIONER and FBS_OPT_PCG_FORM do not apply: the pyramid
 * needs its own device arrays).
 *
 * Launch options set on the grid (FBS_OPT_PCG_LAUNCH, FBS_OPT_PHASE_BLOCKS,
 * or fbs_autotune's choice) apply as they do to fbs_solve.
 *
 * Limits and sharing: the array is 64 MiB (67,108,864 bytes).  A problem
 * needs, with V_k the vertex count and C_k the channel count of image k,
 * Cp_k = C_k for C_k <= 2 and C_k rounded up to a multiple of 4 otherwise,
 * and T_k = ceil(V_k / 256) vertex tiles:
 *     32 B x sum_k roundup32(Cp_k V_k)    eight CG vectors (y, r, r_lo, two
 *                                         search directions, q, two spares)
 *   + 12 B x sum_k V_k                    diag(A) remainder and {n, M^-1}
 *   + 32 B x sum_k C_k T_k                inner-product partials
 *   + 144 B per image + 72 B per (image, channel) + 4,224 B of barrier words,
 * each of these seven pieces rounded up to 256 bytes.  (One 3-channel image
 * fits up to about 478,000 vertices, a 1-channel image about 1.5 million.)
 * A problem that does not fit returns FBS_ERR_ARG before any device work.
 * Every GPU that loads the library holds the array
 * until the process exits.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) -- make that first call
 * before any stream capture.  All calls share the array and it keeps the
 * last call's contents: calls whose work overlaps on the GPU race, so
 * serialise them (one stream, or events).
 */
fbs_status fbs_solve_static(fbs_grid* g, const fbs_problem_desc* probs, int pcg_iters,
                            void* stream);

/* Vertex count and offset (in the concatenated vertex order) of one image.
 * Host outputs; no device work. */
fbs_status fbs_grid_info(const fbs_grid* g, int image, int64_t* n_vertices,
                         int64_t* vertex_offset);

/*
 * fbs_grid_export -- copy one image's grid to HOST buffers for inspection
 * (parity checks).  Any output may be NULL.  Synchronises `stream`.
 *   host_keys  uint64[V]   packed keys (row<<48 | col<<36 | l<<24 | u<<12 | v)
 *   host_vid   uint32[N]   pixel -> vertex id (local to the image)
 *   host_counts uint32[V]  m = S 1
 *   host_nbr   int32[V*10] neighbour ids (local), order x-, x+, y-, y+, l-, l+,
 *                          u-, u+, v-, v+; -1 if absent
 *   host_n     double[V]   bistochastisation vector n (needs fbs_bistochastize)
 */
fbs_status fbs_grid_export(const fbs_grid* g, int image, void* stream, uint64_t* host_keys,
                           uint32_t* host_vid, uint32_t* host_counts, int32_t* host_nbr,
                           double* host_n);

/*
 * fbs_pyramid_export -- copy one level of one image's bilateral-space
 * pyramid (the hierarchical preconditioner's, supplement) to HOST buffers
 * for inspection (parity checks).  Builds the pyramid first if no
 * hierarchical solve has (SYNCHRONISES `stream`; FBS_ERR_STATE inside a
 * stream capture).  *levels receives the number of levels K of the grid's
 * deepest image (an image past its own top keeps one vertex, with count 0).
 * Level 0 is the grid.  Outputs (any may be NULL):
 *   *n_vertices      the image's vertex count on that level (V_level)
 *   host_keys        uint64[V_level]  packed keys, fields floor-halved
 *                                     `level` times; vertices in the
 *                                     library's order (first occurrence)
 *   host_parent      int32[V_level]   index of each vertex's parent among
 *                                     the image's vertices of level + 1
 *                                     (-1 on the top level)
 *   host_count       float[V_level]   P(1): grid vertices below each vertex
 * Errors: FBS_ERR_ARG (bad image or level), FBS_ERR_STATE, FBS_ERR_OOM,
 * FBS_ERR_CUDA.
 */
fbs_status fbs_pyramid_export(fbs_grid* g, int image, int level, void* stream, int* levels,
                              int64_t* n_vertices, uint64_t* host_keys, int32_t* host_parent,
                              float* host_count);

/* Wait for the handle's work on `stream` and return (then clear) any latched
 * device-side error. */
fbs_status fbs_grid_sync(fbs_grid* g, void* stream);

/* Release the handle and its device memory (stream-ordered on `stream`). */
fbs_status fbs_grid_destroy(fbs_grid* g, void* stream);

/* Static description of a status code. */
const char* fbs_status_string(fbs_status s);

/*
 * Device timing with CUDA events on the launching stream (no kernels are
 * added).  fbs_profile_enable(level) clears the totals and records:
 * level 0 nothing, level 1 every kernel family (one event pair around each
 * launch), level 2 regions spanning several launches ("region:grid_build",
 * "region:bistochastize", "region:solve_setup", "region:pcg_loop",
 * "region:slice").  Nothing is recorded while a stream is being captured.
 * fbs_profile_read fills, for family index i < *count, the name, number of
 * recorded intervals and total milliseconds (host arrays of length *count on
 * entry; on return *count is the number of families); it waits for the
 * recorded events.
 */
fbs_status fbs_profile_enable(int on);
fbs_status fbs_profile_read(int* count, const char** names, int64_t* launches, double* total_ms);

#ifdef __cplusplus
}
#endif

#endif /* FBS_H_ */
