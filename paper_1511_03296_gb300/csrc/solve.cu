// Solve kernels: splat (b = S(c o t), S c, diag(A), Jacobi M^-1 and the flat
// initialisation), the initial residual, the two phases of each PCG
// iteration, the slice, and the backward adjoints.
//
// Every vertex kernel walks a table of CTA-sized vertex tiles; each tile
// belongs to one image ("instance"), so one launch advances every (image,
// channel) problem of a batch.  Each block takes a contiguous chunk of tiles.
//
// Vector layout: the CG vectors of an image are vertex-major with each
// vertex's channels padded to Cp (1, 2, or a multiple of 4), so a vertex's
// channels -- its own and, above all, a neighbour's in a gather -- move as
// one aligned float, float2 or float4 per pass of W = min(Cp, 4) channels.
// Padding entries are kept at zero.
//
// CG inner products: every tile (or, when an image's channels fit one pass,
// every block's run of tiles of that image) writes per channel the sum of its
// exact FP32 products as a double-float pair.  The next phase's blocks each
// reduce the partials of the images they touch, in a fixed order, and form
// the CG scalar they need (alpha or beta) in FP64 -- every block obtains the
// same value, so there is no grid-wide serial step, no atomic and no fence,
// and results are bitwise reproducible.
#include "fbs_internal.cuh"
#include "solve.cuh"

namespace fbs {

namespace {

// element (ch, v) of image I
__device__ __forceinline__ int64_t vec_index(const InstDev& I, int ch, int64_t v)
{
    return I.vec_base + (v - I.voff) * I.Cp + ch;
}

// element (cb, v) is at pass_base(I, cb) + v * I.Cp
__device__ __forceinline__ int64_t pass_base(const InstDev& I, int cb)
{
    return I.vec_base - I.voff * I.Cp + cb;
}

__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

// contiguous chunk of tiles for this block
__device__ __forceinline__ void block_chunk(int nvt, int& t0, int& t1)
{
    const int chunk = (nvt + gridDim.x - 1) / gridDim.x;
    t0 = blockIdx.x * chunk;
    t1 = min(t0 + chunk, nvt);
}

// ---------------------------------------------------- vector load/store ---
// W consecutive floats at p (W-aligned); CO: through L2 (ld.cg), for data
// that other blocks rewrite within the same launch.
template <int W, bool CO>
__device__ __forceinline__ void ldw(const float* p, float (&o)[W])
{
    if (W == 4) {
        const float4 v = CO ? __ldcg(reinterpret_cast<const float4*>(p))
                            : *reinterpret_cast<const float4*>(p);
        o[0] = v.x;
        o[1 % W] = v.y;
        o[2 % W] = v.z;
        o[3 % W] = v.w;
    } else if (W == 2) {
        const float2 v = CO ? __ldcg(reinterpret_cast<const float2*>(p))
                            : *reinterpret_cast<const float2*>(p);
        o[0] = v.x;
        o[1 % W] = v.y;
    } else {
        o[0] = CO ? __ldcg(p) : *p;
    }
}

template <int W>
__device__ __forceinline__ void stw(float* p, const float (&v)[W])
{
    if (W == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1 % W], v[2 % W], v[3 % W]);
    } else if (W == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1 % W]);
    } else {
        *p = v[0];
    }
}

// The ten neighbours of vertex v (order: -1, +1 per dimension x, y, l, u, v)
// from the packed table (8-bit offsets for x, l, u, v and 16-bit for y;
// absent: v itself, whose Laplacian term is exactly 0).  Escaped offsets are
// rare (a cell with more than 127 vertices between neighbours, or more than
// 32767 vertices between a vertex and its y neighbour): the 32-bit table is
// read only in a warp-uniform branch when some lane of the warp has one, so
// the common path has no load in the id chain.  All lanes of the warp must
// call it.
__device__ __forceinline__ void load_neighbours(const SolveArgs& A, int v, int (&nb)[10])
{
    const uint32_t w0 = A.nbrp[v];
    const uint32_t w1 = A.nbrp[A.Vtot + v];
    const uint32_t w2 = A.nbrp[2 * A.Vtot + v];
    int o[10];
    o[0] = (int)(int8_t)(w0 & 0xffu);
    o[1] = (int)(int8_t)((w0 >> 8) & 0xffu);
    o[4] = (int)(int8_t)((w0 >> 16) & 0xffu);
    o[5] = (int)(int8_t)(w0 >> 24);
    o[6] = (int)(int8_t)(w1 & 0xffu);
    o[7] = (int)(int8_t)((w1 >> 8) & 0xffu);
    o[8] = (int)(int8_t)((w1 >> 16) & 0xffu);
    o[9] = (int)(int8_t)(w1 >> 24);
    o[2] = (int)(int16_t)(w2 & 0xffffu);
    o[3] = (int)(int16_t)(w2 >> 16);
    bool esc = (o[2] == kNbrEscape) | (o[3] == kNbrEscape);
#pragma unroll
    for (int j = 0; j < 10; ++j) {
        nb[j] = v + o[j];
        if (j != 2 && j != 3) esc |= o[j] == kNbrEscape8;
    }
    if (__any_sync(0xffffffffu, esc)) {
#pragma unroll
        for (int j = 0; j < 10; ++j) {
            const bool e = (j == 2 || j == 3) ? o[j] == kNbrEscape : o[j] == kNbrEscape8;
            if (e) nb[j] = A.nbr[(int64_t)j * A.nbr_stride + v];
        }
    }
}

// -------------------------------------------------------- inner products ---
struct PhaseSmem {
    DF red[4][kVTile / 32];
    double sd[kMaxChannels];     // reduced inner products
    double sd2[kMaxChannels];    // second inner product (single-reduction form)
    float sf[kMaxChannels];      // beta (phase 1)
    double sa[kMaxChannels];     // alpha (phase 2)
    int last;                    // this block completed an image's partials
};

// scratch of the per-channel reduction of wide images (Cp > 4)
struct WideSmem {
    DF lane[kVTile][4];          // each thread's four channel sums
    DF group[kVTile];            // [group][channel] partial sums
};

// Block-reduce W double-float partials (channels cb .. cb+W-1) and store each
// in partial slot `slot` of its channel.
template <int W>
__device__ void store_partials(DF (&acc)[W], int C, int ntiles, int64_t part_base, int cb,
                               int slot, float2* __restrict__ part, DF (*red)[kVTile / 32])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        DF s = df_warp_sum(acc[k]);
        if (lane == 0) red[k][w] = s;
        acc[k] = {0.0f, 0.0f};
    }
    __syncthreads();
    if ((int)threadIdx.x < W && cb + (int)threadIdx.x < C) {
        const int k = threadIdx.x, ch = cb + k;
        DF t = red[k][0];
        for (int j = 1; j < (int)(blockDim.x >> 5); ++j) t = df_add(t, red[k][j]);
        part[part_base + (int64_t)ch * ntiles + slot] = make_float2(t.hi, t.lo);
    }
    __syncthreads();
}

// Sum, per channel, the partials of one instance (fixed order: lane j takes
// slots j, j+32, ... in groups of 8 loads issued together; then the warp
// tree) into out[ch] (FP64).  Warps take channels round-robin.  Whole block.
// Partials written earlier in the same launch by other blocks are read
// through L2 (ld.cg).
__device__ void reduce_instance_partials(const float2* __restrict__ part, const InstDev& I,
                                         double* out)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int ch = w; ch < I.C; ch += nw) {
        const float2* p = part + I.part_base + (int64_t)ch * I.ntiles;
        DF t = {0.0f, 0.0f};
        for (int j0 = lane; j0 < I.ntiles; j0 += 32 * 8) {
            float2 v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int j = j0 + 32 * k;
                v[k] = j < I.ntiles ? __ldcg(p + j) : make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) t = df_add(t, DF{v[k].x, v[k].y});
        }
        t = df_warp_sum(t);
        if (lane == 0) out[ch] = df_to_double(t);
    }
}

// All threads sum the partials of one instance for all its (<= W) channels
// (thread t takes slots t, t + blockDim, ..., H of them per channel in
// flight), then a block tree; out[ch].  Whole block; ends with a barrier.
template <int W, int H = (W == 4 ? 1 : 2)>
__device__ void reduce_partials_all(const float2* __restrict__ part, const InstDev& I,
                                    double* out, DF (*red)[kVTile / 32])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    DF acc[W];
#pragma unroll
    for (int k = 0; k < W; ++k) acc[k] = {0.0f, 0.0f};
    for (int j0 = threadIdx.x; j0 < I.ntiles; j0 += H * blockDim.x) {
        float2 v[W][H];
#pragma unroll
        for (int k = 0; k < W; ++k)
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const int j = j0 + h * blockDim.x;
                v[k][h] = (k < I.C && j < I.ntiles)
                              ? __ldcg(part + I.part_base + (int64_t)k * I.ntiles + j)
                              : make_float2(0.0f, 0.0f);
            }
#pragma unroll
        for (int k = 0; k < W; ++k)
#pragma unroll
            for (int h = 0; h < H; ++h) acc[k] = df_add(acc[k], DF{v[k][h].x, v[k][h].y});
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const DF t = df_warp_sum(acc[k]);
        if (lane == 0) red[k][w] = t;
    }
    __syncthreads();
    if ((int)threadIdx.x < W && (int)threadIdx.x < I.C) {
        const int k = threadIdx.x;
        DF t = red[k][0];
        for (int j = 1; j < nw; ++j) t = df_add(t, red[k][j]);
        out[k] = df_to_double(t);
    }
    __syncthreads();
}

// Finalised CG scalars (A.fin): the block that completes an image's tile
// partials of a phase reduces them -- in the same fixed order as any block
// would -- and stores the scalars the next phase needs, so the blocks of the
// next phase read a few words instead of each reducing every partial of the
// image.  kind 0: the partials are r^T M^-1 r of iteration `it` (initial
// residual, or phase 2 of iteration it - 1): delta_it and beta_it.  kind 1:
// d^T A d of iteration `it` (phase 1): alpha_it.  `ntiles`: the image's tiles
// whose partials this block has stored since its last call.  The counter is
// the image's first Scal entry; the completing block resets it.  Whole block.
__device__ void finish_image(const SolveArgs& A, const InstDev& I, int ntiles,
                             const float2* __restrict__ part, int kind, int it, PhaseSmem& S)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned old = atomicAdd(&A.scal[I.pc].done, (unsigned)ntiles);
        const int last = old + (unsigned)ntiles == (unsigned)I.ntiles;
        if (last) __threadfence();
        S.last = last;
    }
    __syncthreads();
    if (!S.last) return;
    if (I.Cp == 1) reduce_partials_all<1, 8>(part, I, S.sd, S.red);
    else if (I.Cp == 2) reduce_partials_all<2, 4>(part, I, S.sd, S.red);
    else if (I.Cp == 4) reduce_partials_all<4, 2>(part, I, S.sd, S.red);
    else {
        reduce_instance_partials(part, I, S.sd);
        __syncthreads();
    }
    for (int ch = threadIdx.x; ch < I.C; ch += blockDim.x) {
        Scal* sc = &A.scal[I.pc + ch];
        const double d0 = __ldcg(&sc->delta0);
        if (kind == 0) {
            const int slot = it & 1;
            const double dnow = S.sd[ch];
            double beta = 0.0;
            if (it > 0) {
                const double dprev = __ldcg(&sc->delta[slot ^ 1]);
                beta = dprev != 0.0 && !cg_stalled(dnow, d0) ? dnow / dprev : 0.0;
            } else {
                sc->delta0 = dnow;
            }
            sc->delta[slot] = dnow;
            sc->beta = (float)beta;
        } else {
            const double delta = __ldcg(&sc->delta[it & 1]);
            const double dq = S.sd[ch];
            sc->alpha = (dq > 0.0 && !cg_stalled(delta, d0)) ? delta / dq : 0.0;
        }
    }
    if (threadIdx.x == 0) A.scal[I.pc].done = 0u;
    __syncthreads();
}

// The finalised scalars of image I for a phase (A.fin): beta (phase 1) or
// alpha (phase 2); padding channels 0.  Whole block; ends with a barrier.
template <int PHASE>
__device__ __forceinline__ void load_scalars(const SolveArgs& A, const InstDev& I, PhaseSmem& S)
{
    __syncthreads();
    for (int ch = threadIdx.x; ch < I.Cp; ch += blockDim.x) {
        const bool on = ch < I.C;
        if (PHASE == 1) S.sf[ch] = on ? __ldcg(&A.scal[I.pc + ch].beta) : 0.0f;
        else S.sa[ch] = on ? __ldcg(&A.scal[I.pc + ch].alpha) : 0.0;
    }
    __syncthreads();
}

// The CG scalars a block needs for image I at the start of a phase, from the
// previous phase's partials (every block forms the same values): phase 1
// delta_it = r^T M^-1 r and beta = delta_it / delta_(it-1) (delta_it is also
// stored); phase 2 alpha = delta_it / d^T q.  Padding channels get 0.
// Whole block; ends with a barrier.
template <int PHASE, bool CO, int WMAX>
__device__ void phase_scalars(const SolveArgs& A, const InstDev& I, const float2* in, int it,
                              PhaseSmem& S)
{
    const int slot = it & 1;
    __syncthreads();
    if (WMAX == 1 || I.Cp == 1) reduce_partials_all<1, 8>(in, I, S.sd, S.red);
    else if (WMAX == 2 || I.Cp == 2) reduce_partials_all<2, 4>(in, I, S.sd, S.red);
    else if (I.Cp == 4) reduce_partials_all<4, 2>(in, I, S.sd, S.red);
    else {
        reduce_instance_partials(in, I, S.sd);
        __syncthreads();
    }
    for (int ch = threadIdx.x; ch < I.Cp; ch += blockDim.x) {
        if (ch >= I.C) {            // padding channels: scalars 0 keep them at 0
            S.sf[ch] = 0.0f;
            S.sa[ch] = 0.0;
        } else if (PHASE == 1) {
            const double dnow = S.sd[ch];
            double beta = 0.0;
            if (it > 0) {
                const double dprev = CO ? __ldcg(&A.scal[I.pc + ch].delta[slot ^ 1])
                                        : A.scal[I.pc + ch].delta[slot ^ 1];
                const double d0 = CO ? __ldcg(&A.scal[I.pc + ch].delta0) : A.scal[I.pc + ch].delta0;
                beta = dprev != 0.0 && !cg_stalled(dnow, d0) ? dnow / dprev : 0.0;
            } else {
                A.scal[I.pc + ch].delta0 = dnow;
            }
            S.sf[ch] = (float)beta;
            A.scal[I.pc + ch].delta[slot] = dnow;   // same value from every block
        } else {
            const double delta = CO ? __ldcg(&A.scal[I.pc + ch].delta[slot])
                                    : A.scal[I.pc + ch].delta[slot];
            const double d0 = CO ? __ldcg(&A.scal[I.pc + ch].delta0) : A.scal[I.pc + ch].delta0;
            const double dq = S.sd[ch];
            S.sa[ch] = (dq > 0.0 && !cg_stalled(delta, d0)) ? delta / dq : 0.0;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- splat ---
// A is applied in Laplacian form,
//   (A z)_v = a'_v z_v + lambda n_v sum_u n_u (z_v - z_u),
//   a'_v    = lambda (m_v - n_v (Bbar n)_v) + (S c)_v,
// which equals a_v z_v - lambda n_v sum_u n_u z_u with
// a_v = diag(A)_v = lambda (m_v - 10 n_v^2) + (S c)_v.  a' is formed in FP64
// here; the off-diagonal part has zero row sums whatever the rounding of n,
// so FP32 vectors keep the data term intact.  A vertex without neighbours
// has smoothness part 0 (its row of lambda (D_m - D_n Bbar D_n) vanishes once
// n^2 = m / 10).  M^-1 = 1 / diag(A), 0 where diag(A) <= 0.
__device__ __forceinline__ void vertex_epilogue(const SolveArgs& A, const InstDev& I, int64_t v,
                                                uint32_t cnt, DF sc)
{
    bool has_nbr = false;
    double sum_n = 0.0;
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        const int32_t u = A.nbr[(int64_t)k * A.nbr_stride + v];
        if (u >= 0) {
            has_nbr = true;
            sum_n += A.n64[u];
        }
    }
    const double nv = A.n64[v];
    const double scd = (double)sc.hi + (double)sc.lo;
    const double lam = (double)I.lam;
    const double rem = has_nbr ? lam * ((double)cnt - nv * (10.0 * nv + sum_n)) : 0.0;
    const double diag = has_nbr ? lam * ((double)cnt - 10.0 * nv * nv) + scd : scd;
    if (A.alo) {                        // a' as a double-float pair
        const DF ap = df_from_double(rem + scd);
        A.a[v] = ap.hi;
        A.alo[v] = ap.lo;
    } else {
        A.a[v] = (float)(rem + scd);
    }
    A.nm[v] = make_float2((float)nv, diag > 0.0 ? (float)(1.0 / diag) : 0.0f);
    if (A.pyr.K > 0) {                  // hierarchical preconditioner: diag(A) and S c
        A.pyr.dg[v] = (float)diag;
        A.pyr.scv[v] = (float)scd;
    }
}

// Splat weight and value of one pixel (index i within its image) for channel
// ch: robust weights are Geman-McClure of the residual against the vertex's
// current solution yv (+ ylo, its low part when y is a double-float pair:
// yv - t is exact when they are close, so the residual keeps y's accuracy).
__device__ __forceinline__ float splat_weight(const InstDev& I, int mode, int64_t i, float yv,
                                              float ylo, float s2)
{
    if (mode == kSplatRobust) {
        const float e = (yv - I.t[i]) + ylo;
        const float den = s2 + e * e;
        return (2.0f * s2) / (den * den);
    }
    return I.c[i];
}

__device__ __forceinline__ float splat_value(const InstDev& I, int mode, int ch, int64_t i)
{
    return mode == kSplatBackward ? I.dx[(int64_t)ch * I.N + i] : I.t[(int64_t)ch * I.N + i];
}

__device__ __forceinline__ DF df_shfl_idx(DF v, int src)
{
    return {__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

// Write b (into r, or the double-float pair r, r_lo when comp) and the flat
// initialisation y0 = b / S c for channels cb .. cb+CB-1 of vertex v.
template <int CB>
__device__ __forceinline__ void splat_store(const SolveArgs& A, const InstDev& I, int64_t v,
                                            int cb, const DF (&acc)[CB], DF sc, int comp)
{
    const float scf = sc.hi + sc.lo;
#pragma unroll
    for (int k = 0; k < CB; ++k) {
        const int ch = cb + k;
        if (ch < I.C) {
            const float b = acc[k].hi + acc[k].lo;
            const int64_t idx = vec_index(I, ch, v);
            if (comp) {
                const DF bn = df_fast_two_sum(acc[k].hi, acc[k].lo);
                A.r[idx] = bn.hi;
                A.rlo[idx] = bn.lo;
            } else {
                A.r[idx] = b;
            }
            A.y[idx] = scf > 0.0f ? b / scf : 0.0f;
            if (A.ylo) A.ylo[idx] = 0.0f;
        }
    }
}

// Padding channels zero, non-finite flag, diagonal and preconditioner.
__device__ __forceinline__ void splat_finish(const SolveArgs& A, const InstDev& I, int64_t v,
                                             uint32_t cnt, DF sc)
{
    for (int ch = I.C; ch < I.Cp; ++ch) {
        const int64_t idx = vec_index(I, ch, v);
        A.r[idx] = 0.0f;
        A.rlo[idx] = 0.0f;
        A.y[idx] = 0.0f;
        A.d[0][idx] = 0.0f;
        A.d[1][idx] = 0.0f;
        A.q[idx] = 0.0f;
        A.aux[0][idx] = 0.0f;
        A.aux[1][idx] = 0.0f;
    }
    vertex_epilogue(A, I, v, cnt, sc);
}

// Pixels of a vertex with more than this many are summed by the whole warp.
constexpr uint32_t kSplatWarpMin = 24;

// One warp unit (32 consecutive vertices of one tile): a vertex with at most
// kSplatWarpMin pixels is summed by its own thread, walking its pixels in the
// sorted order; a larger vertex is summed by the whole warp (lane j takes
// pixels j, j + 32, ..., then a fixed-order warp reduction).
template <int CB>
__device__ __forceinline__ void splat_unit(const SolveArgs& A, const InstDev& I, int64_t v,
                                           bool valid, int mode, float s2, int comp)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t p0 = valid ? A.pstart[v] : 0u, cnt = valid ? A.m[v] : 0u;
    const bool big = cnt > kSplatWarpMin;
    const uint32_t own = big ? 0u : cnt;
    // robust weights: the robust solver has one channel (CB = 1)
    float yv = 0.0f, ylv = 0.0f;
    if (mode == kSplatRobust && valid) {
        yv = A.y[vec_index(I, 0, v)];
        if (CB == 1 && A.ylo) ylv = A.ylo[vec_index(I, 0, v)];
    }
    DF sc = {0.0f, 0.0f};
    bool bad = false;
    for (int cb = 0; cb < I.C; cb += CB) {
        DF acc[CB];
#pragma unroll
        for (int k = 0; k < CB; ++k) acc[k] = {0.0f, 0.0f};
        for (uint32_t j0 = 0; j0 < own; j0 += 8) {
            int64_t ii[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                ii[u] = j0 + u < own ? (int64_t)A.perm[p0 + j0 + u] - I.pix_base : -1;
            float wv[8], val[CB][8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t i = ii[u] >= 0 ? ii[u] : 0;
                wv[u] = splat_weight(I, mode, i, yv, ylv, s2);
#pragma unroll
                for (int k = 0; k < CB; ++k)
                    val[k][u] = splat_value(I, mode, min(cb + k, I.C - 1), i);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (ii[u] < 0) break;
                const float w = wv[u];
                if (cb == 0) {
                    sc = df_add(sc, DF{w, 0.0f});
                    bad |= !isfinite(w);
                }
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    if (cb + k < I.C) {
                        const float x = val[k][u];
                        acc[k] = df_add(acc[k], mode == kSplatBackward ? DF{x, 0.0f}
                                                                       : df_mul_exact(w, x));
                        bad |= !isfinite(x);
                    }
                }
            }
        }
        unsigned bigmask = __ballot_sync(FULL, big);
        while (bigmask) {
            const int owner = __ffs(bigmask) - 1;
            bigmask &= bigmask - 1;
            const uint32_t q0 = __shfl_sync(FULL, p0, owner);
            const uint32_t qn = __shfl_sync(FULL, cnt, owner);
            const float qy = __shfl_sync(FULL, yv, owner);
            const float qyl = CB == 1 ? __shfl_sync(FULL, ylv, owner) : 0.0f;
            DF wacc[CB], wsc = {0.0f, 0.0f};
#pragma unroll
            for (int k = 0; k < CB; ++k) wacc[k] = {0.0f, 0.0f};
            bool wbad = false;
            for (uint32_t j0 = 0; j0 < qn; j0 += 4 * 32) {
                int64_t ii[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t j = j0 + 32 * u + lane;
                    ii[u] = j < qn ? (int64_t)A.perm[q0 + j] - I.pix_base : -1;
                }
                float wv[4], val[CB][4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t i = ii[u] >= 0 ? ii[u] : 0;
                    wv[u] = splat_weight(I, mode, i, qy, qyl, s2);
#pragma unroll
                    for (int k = 0; k < CB; ++k)
                        val[k][u] = splat_value(I, mode, min(cb + k, I.C - 1), i);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (ii[u] < 0) continue;
                    const float w = wv[u];
                    if (cb == 0) {
                        wsc = df_add(wsc, DF{w, 0.0f});
                        wbad |= !isfinite(w);
                    }
#pragma unroll
                    for (int k = 0; k < CB; ++k) {
                        if (cb + k < I.C) {
                            const float x = val[k][u];
                            wacc[k] = df_add(wacc[k], mode == kSplatBackward ? DF{x, 0.0f}
                                                                             : df_mul_exact(w, x));
                            wbad |= !isfinite(x);
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                const DF t = df_warp_sum(wacc[k]);
                const DF g = df_shfl_idx(t, 0);
                if (lane == owner) acc[k] = g;
            }
            if (cb == 0) {
                const DF t = df_warp_sum(wsc);
                const DF g = df_shfl_idx(t, 0);
                if (lane == owner) sc = g;
            }
            if (__any_sync(FULL, wbad) && lane == owner) bad = true;
        }
        if (valid) splat_store<CB>(A, I, v, cb, acc, sc, comp);
    }
    if (bad) atomicOr(A.err, kErrNonFinite);
    if (valid) splat_finish(A, I, v, cnt, sc);
}

// b = S(c o t) (or its robust / backward form), S c, the flat initialisation
// y0 = b / S c (zero in the padding channels), the diagonal remainder a' and
// {n, M^-1}.  Work is split in warp units of 32 consecutive vertices of one
// tile, which warps claim from a counter (*work, zero at launch): the pixel
// counts of vertices differ by orders of magnitude between images (a grey
// colourisation reference puts whole cells in one vertex), so a static split
// leaves most blocks idle behind a few.  Products are exact and accumulated
// as double-float pairs in a fixed order, so results do not depend on which
// warp takes which unit.
template <int CB>
__global__ void __launch_bounds__(kVTile)
splat_kernel(SolveArgs A, int mode, float sigma_gm, int comp, unsigned* work)
{
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int kUnits = kVTile / 32;
    const float s2 = sigma_gm * sigma_gm;
    const int lane = threadIdx.x & 31;
    const int nunits = A.nvt * kUnits;
    int unit = 0;
    if (lane == 0) unit = (int)atomicAdd(work, 1u);
    unit = __shfl_sync(FULL, unit, 0);
    while (unit < nunits) {
        int next = 0;
        if (lane == 0) next = (int)atomicAdd(work, 1u);   // overlaps this unit
        const int tile = unit / kUnits;
        const VTile vt = A.vt[tile];
        const int64_t v = vt.v0 + (unit - tile * kUnits) * 32 + lane;
        if (vt.v0 + (unit - tile * kUnits) * 32 < vt.v1) {       // warp-uniform
            const InstDev I = A.inst[vt.inst];
            splat_unit<CB>(A, I, v, v < vt.v1, mode, s2, comp);
        }
        unit = __shfl_sync(FULL, next, 0);
    }
}

// ------------------------------------------------- Laplacian-form apply ---
// Accumulates, for W channels, sum_u n_u (z_v - z_u) over the neighbours.
// COMP: each product n_u (z_v - z_u) is split exactly into p + e; p enters
// the running high part through an error-free two-sum and both errors are
// added to the low part (the cascaded "Sum2" scheme of Ogita, Rump and
// Oishi, 2005: as accurate as summing in twice the working precision); the
// pair is renormalised in lap_finish.
template <int W, bool COMP>
__device__ __forceinline__ void lap_acc(DF (&s)[W], float nu, const float (&zv)[W],
                                        const float (&zu)[W])
{
#pragma unroll
    for (int k = 0; k < W; ++k) {
        if (COMP) {
            const float dz = zv[k] - zu[k];
            const float p = __fmul_rn(nu, dz);
            const float e = __fmaf_rn(nu, dz, -p);
            const DF t = df_two_sum(s[k].hi, p);
            s[k].hi = t.hi;
            s[k].lo = __fadd_rn(s[k].lo, __fadd_rn(t.lo, e));
        } else {
            s[k].hi = fmaf(nu, zv[k] - zu[k], s[k].hi);
        }
    }
}

// (A z)_v = a'_v z_v + lambda n_v s
template <bool COMP>
__device__ __forceinline__ DF lap_finish(float av, float lam_n, float zv, DF s, float alv = 0.0f)
{
    // COMP: a' z exactly (plus alv z when a' is a double-float pair a' = av + alv)
    return COMP ? df_add(df_add_f(df_mul_exact(av, zv), alv * zv),
                         df_mul_f(df_two_sum(s.hi, s.lo), lam_n))
                : DF{fmaf(av, zv, lam_n * s.hi), 0.0f};
}

// ------------------------------------------------------- initial residual ---
// r = b - A y0 (b is in r, and in r_lo too when COMP); tile partials of
// r^T M^-1 r (delta_0) into rs slot 0.
template <int W, bool COMP>
__device__ __forceinline__ void residual_tile(const SolveArgs& A, const InstDev& I,
                                              const VTile& vt, PhaseSmem& S)
{
    const int64_t v = vt.v0 + threadIdx.x;
    const bool valid = v < vt.v1;
    const int64_t vs = valid ? v : vt.v0;
    const float2 nmv = valid ? A.nm[v] : make_float2(0.0f, 0.0f);
    const float av = valid ? A.a[v] : 0.0f;
    const float alv = COMP && A.alo && valid ? A.alo[v] : 0.0f;
    const float lam_n = I.lam * nmv.x;
    int32_t nb[10];
#pragma unroll
    for (int j = 0; j < 10; ++j) nb[j] = valid ? A.nbr[(int64_t)j * A.nbr_stride + v] : -1;
    for (int cb = 0; cb < I.C; cb += W) {
        const int64_t base = pass_base(I, cb);
        float yv[W];
        ldw<W, false>(A.y + base + vs * I.Cp, yv);
        DF s[W];
#pragma unroll
        for (int k = 0; k < W; ++k) s[k] = {0.0f, 0.0f};
#pragma unroll
        for (int j = 0; j < 10; ++j) {
            const int64_t u = nb[j] >= 0 ? nb[j] : vs;
            const float nu = nb[j] >= 0 ? A.nm[u].x : 0.0f;
            float yu[W];
            ldw<W, false>(A.y + base + u * I.Cp, yu);
            lap_acc<W, COMP>(s, nu, yv, yu);
        }
        float rv[W];
        ldw<W, false>(A.r + base + vs * I.Cp, rv);
        float rl[W];
        if (COMP) ldw<W, false>(A.rlo + base + vs * I.Cp, rl);
        DF acc[W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const DF Ay = lap_finish<COMP>(av, lam_n, yv[k], s[k], alv);
            if (COMP) {
                const DF r = df_add(DF{rv[k], rl[k]}, df_neg(Ay));
                rv[k] = r.hi;
                rl[k] = r.lo;
            } else {
                rv[k] = rv[k] - Ay.hi;
            }
            acc[k] = valid && cb + k < I.C ? df_mul_exact(rv[k], nmv.y * rv[k]) : DF{0.0f, 0.0f};
        }
        if (valid) {
            stw<W>(A.r + base + v * I.Cp, rv);
            if (COMP) stw<W>(A.rlo + base + v * I.Cp, rl);
        }
        store_partials<W>(acc, I.C, I.ntiles, I.part_base, cb, vt.t_in_inst, A.part_rs[0], S.red);
    }
}

template <bool COMP>
__global__ void __launch_bounds__(kVTile)
residual_kernel(SolveArgs A)
{
    __shared__ PhaseSmem S;
    int t0, t1;
    block_chunk(A.nvt, t0, t1);
    for (int tile = t0; tile < t1; ++tile) {
        const VTile vt = A.vt[tile];
        const InstDev I = A.inst[vt.inst];
        if (I.Cp == 1) residual_tile<1, COMP>(A, I, vt, S);
        else if (I.Cp == 2) residual_tile<2, COMP>(A, I, vt, S);
        else residual_tile<4, COMP>(A, I, vt, S);
        if (A.fin) finish_image(A, I, 1, A.part_rs[0], 0, 0, S);
    }
}

// -------------------------------------------------- PCG phase bodies ---
// FP32 phase 1 of iterations >= 1 with the preconditioned residual
// z = M^-1 r stored by the previous update: since d = z + beta d_old is
// linear, A d = A z + beta q_old, so a neighbour contributes only n_u and z_u
// (two dense gathers instead of {n, M^-1}, r and d_old) and the vertex's own
// q_old is a streamed read.  d and d^T q are formed as in apply_tile; q
// differs from A d by rounding only.  (Iteration 0 takes apply_tile's path,
// whose q = A d = A z starts the recurrence.)
template <int W, bool CO>
__device__ __forceinline__ void apply_tile_z(const SolveArgs& A, const InstDev& I,
                                             const VTile& vt, const float* __restrict__ dold,
                                             float* __restrict__ dnew, PhaseSmem& S,
                                             DF (&run)[4], bool fetch, const float2* in, int it)
{
    const int v = (int)vt.v0 + (int)threadIdx.x;
    const bool valid = v < (int)vt.v1;
    const int vs = valid ? v : (int)vt.v0;
    const int64_t off = I.vec_base - I.voff * W;
    const float* __restrict__ zb = A.zq + off;
    int nb[10];
    load_neighbours(A, vs, nb);
    float zv[W], ov[W], qo[W];
    ldw<W, CO>(zb + vs * W, zv);
    ldw<W, CO>(dold + off + vs * W, ov);
    ldw<W, CO>(A.q + off + vs * W, qo);
    const float nv = valid ? A.nf[v] : 0.0f;
    const float av = valid ? A.a[v] : 0.0f;
    if (fetch) phase_scalars<1, CO, W>(A, I, in, it, S);
    float sacc[W];
#pragma unroll
    for (int k = 0; k < W; ++k) sacc[k] = 0.0f;
#pragma unroll
    for (int j = 0; j < 10; ++j) {
        const int u = nb[j];
        const float nu = A.nf[u];
        float zu[W];
        ldw<W, CO>(zb + u * W, zu);
#pragma unroll
        for (int k = 0; k < W; ++k) sacc[k] = fmaf(nu, zv[k] - zu[k], sacc[k]);
    }
    const float lam_n = I.lam * nv;
    float dv[W], qh[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const float beta = S.sf[k];
        const float az = fmaf(av, zv[k], lam_n * sacc[k]);
        dv[k] = fmaf(beta, ov[k], zv[k]);
        qh[k] = fmaf(beta, qo[k], az);
        if (valid && k < I.C) run[k] = df_add(run[k], df_mul_exact(dv[k], qh[k]));
    }
    if (valid) {
        stw<W>(dnew + off + v * W, dv);
        stw<W>(A.q + off + v * W, qh);
    }
}

// Phase 1 of iteration `it` on one tile of an image with Cp = W <= 4 (one
// pass; the row stride is the compile-time W, and vertex ids are 32-bit):
// d = M^-1 r + beta d_old (own vertex and, on the fly, its neighbours),
// q = A d, products d q into run[].  q is formed in FP32 in both precisions;
// FP32 stores it for phase 2, while COMP uses it only in d^T q (the step
// length) and phase 2 recomputes it exactly from d.  With fetch (the tile starts the
// block's run over an image) the CG scalars are formed first, after the
// tile's neighbour ids and own values have been requested.
// Z: the z form (FP32, Jacobi, iterations >= 1; z stored by the last update)
template <int W, bool COMP, bool CO, bool HIER = false, bool Z = false>
__device__ __forceinline__ void apply_tile(const SolveArgs& A, const InstDev& I, const VTile& vt,
                                           const float* __restrict__ dold,
                                           float* __restrict__ dnew, bool first, PhaseSmem& S,
                                           DF (&run)[4], bool fetch, const float2* in, int it)
{
    static_assert(!Z || (!COMP && !HIER), "the z form is the FP32 Jacobi phase 1");
    if (Z) {
        apply_tile_z<W, CO>(A, I, vt, dold, dnew, S, run, fetch, in, it);
        return;
    }
    // HIER: the preconditioned residual z = M_hier^-1 r is a vector of its own
    // (the pyramid passes after each update), read in place of M^-1 r
    const int v = (int)vt.v0 + (int)threadIdx.x;
    const bool valid = v < (int)vt.v1;
    const int vs = valid ? v : (int)vt.v0;
    const int64_t off = I.vec_base - I.voff * W;        // element (ch, u) at off + u W + ch
    const float* __restrict__ rb = (HIER ? A.pyr.z : A.r) + off;
    const float* __restrict__ ob = dold + off;
    const float2 nmv = valid ? A.nm[v] : make_float2(0.0f, 0.0f);
    const float av = valid ? A.a[v] : 0.0f;
    // neighbour ids (an absent neighbour is replaced by the vertex itself:
    // its term n_u (d_v - d_u) is then exactly 0, so no masking is needed)
    int nb[10];
    load_neighbours(A, vs, nb);
    float rv[W], ov[W];
    ldw<W, CO>(rb + vs * W, rv);
    if (!first) ldw<W, CO>(ob + vs * W, ov);
    if (fetch) phase_scalars<1, CO, W>(A, I, in, it, S);
    float beta[W], dv[W];
    const float mv = HIER ? 1.0f : nmv.y;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        beta[k] = S.sf[k];
        dv[k] = first ? mv * rv[k] : fmaf(beta[k], ov[k], mv * rv[k]);
    }
    float sacc[W];
#pragma unroll
    for (int k = 0; k < W; ++k) sacc[k] = 0.0f;
#pragma unroll
    for (int j = 0; j < 10; ++j) {
        const int u = nb[j];
        const float2 nm = A.nm[u];
        float ru[W], ou[W];
        ldw<W, CO>(rb + u * W, ru);
        if (!first) ldw<W, CO>(ob + u * W, ou);
        const float mu = HIER ? 1.0f : nm.y;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const float du = first ? mu * ru[k] : fmaf(beta[k], ou[k], mu * ru[k]);
            sacc[k] = fmaf(nm.x, dv[k] - du, sacc[k]);
        }
    }
    const float lam_n = I.lam * nmv.x;
    float qh[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
        qh[k] = fmaf(av, dv[k], lam_n * sacc[k]);
        if (valid && k < I.C) run[k] = df_add(run[k], df_mul_exact(dv[k], qh[k]));
    }
    if (valid) {
        stw<W>(dnew + off + v * W, dv);
        if (!COMP) stw<W>(A.q + off + v * W, qh);
    }
}

// Phase 2 on one tile of an image with Cp = W <= 4: y += alpha d;
// r -= alpha q; products r M^-1 r into run[].  COMP: q = A d is recomputed
// here with compensated arithmetic and the residual is kept as a
// double-float pair (r, r_lo), so the recurrence r <- r - alpha A d carries
// no rounding of q.  With fetch, the CG scalars are formed after the tile's
// own loads have been requested.
template <int W, bool COMP, bool CO>
__device__ __forceinline__ void update_tile(const SolveArgs& A, const InstDev& I, const VTile& vt,
                                            const float* __restrict__ d, PhaseSmem& S,
                                            DF (&run)[4], bool fetch, const float2* in, int it)
{
    const int v = (int)vt.v0 + (int)threadIdx.x;
    const bool valid = v < (int)vt.v1;
    const int vs = valid ? v : (int)vt.v0;
    const int64_t off = I.vec_base - I.voff * W;
    const float2 nmv = valid ? A.nm[v] : make_float2(0.0f, 0.0f);
    float dv[W], yv[W], rv[W], rl[W], qv[W];
    ldw<W, CO>(d + off + vs * W, dv);
    ldw<W, CO>(A.y + off + vs * W, yv);
    ldw<W, CO>(A.r + off + vs * W, rv);
    if (COMP) ldw<W, CO>(A.rlo + off + vs * W, rl);
    else ldw<W, CO>(A.q + off + vs * W, qv);
    // COMP with a double-float y (A.ylo): y's low part, updated exactly
    const bool ydf = COMP && A.ylo != nullptr;
    float yl[W];
    if (ydf) ldw<W, CO>(A.ylo + off + vs * W, yl);
    if (fetch) phase_scalars<2, CO, W>(A, I, in, it, S);
    DF sacc[W];
    float av = 0.0f, alv = 0.0f;
    if (COMP) {
        av = valid ? A.a[v] : 0.0f;
        alv = A.alo && valid ? A.alo[v] : 0.0f;
#pragma unroll
        for (int k = 0; k < W; ++k) sacc[k] = {0.0f, 0.0f};
        int nb[10];
        load_neighbours(A, vs, nb);
#pragma unroll
        for (int j = 0; j < 10; ++j) {
            const int u = nb[j];
            const float nu = A.nm[u].x;
            float du[W];
            ldw<W, CO>(d + off + u * W, du);
            lap_acc<W, true>(sacc, nu, dv, du);
        }
    }
    const float lam_n = I.lam * nmv.x;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const double alpha = S.sa[k];
        if (ydf) {
            const DF yy = df_add(DF{yv[k], yl[k]}, df_mul_f(df_from_double(alpha), dv[k]));
            yv[k] = yy.hi;
            yl[k] = yy.lo;
        } else {
            yv[k] = fmaf((float)alpha, dv[k], yv[k]);
        }
        if (COMP) {
            const DF q = lap_finish<true>(av, lam_n, dv[k], sacc[k], alv);
            const DF r = df_add(DF{rv[k], rl[k]}, df_neg(df_mul(df_from_double(alpha), q)));
            rv[k] = r.hi;
            rl[k] = r.lo;
        } else {
            rv[k] = fmaf(-(float)alpha, qv[k], rv[k]);
        }
        if (valid && k < I.C) run[k] = df_add(run[k], df_mul_exact(rv[k], nmv.y * rv[k]));
    }
    if (valid) {
        stw<W>(A.y + off + v * W, yv);
        stw<W>(A.r + off + v * W, rv);
        if (COMP) stw<W>(A.rlo + off + v * W, rl);
        if (ydf) stw<W>(A.ylo + off + v * W, yl);
        if (!COMP && A.zq) {
            float zv[W];
#pragma unroll
            for (int k = 0; k < W; ++k) zv[k] = nmv.y * rv[k];
            stw<W>(A.zq + off + v * W, zv);
        }
    }
}

// FP32 phase 2 on two consecutive tiles of one image (Cp = W <= 4): the same
// arithmetic as update_tile, with the loads of both tiles issued together
// (a streaming pass; this doubles the loads in flight per thread).  The
// products enter run[] tile by tile, in the same order as two single calls.
template <int W, bool CO>
__device__ __forceinline__ void update_pair(const SolveArgs& A, const InstDev& I,
                                            const VTile& va, const VTile& vb,
                                            const float* __restrict__ d, PhaseSmem& S,
                                            DF (&run)[4], bool fetch, const float2* in, int it)
{
    const int64_t off = I.vec_base - I.voff * W;
    int v[2], vs[2];
    bool valid[2];
    float2 nmv[2];
    float dv[2][W], yv[2][W], rv[2][W], qv[2][W];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const VTile& vt = t == 0 ? va : vb;
        v[t] = (int)vt.v0 + (int)threadIdx.x;
        valid[t] = v[t] < (int)vt.v1;
        vs[t] = valid[t] ? v[t] : (int)vt.v0;
        nmv[t] = A.nm[vs[t]];
        ldw<W, CO>(d + off + vs[t] * W, dv[t]);
        ldw<W, CO>(A.y + off + vs[t] * W, yv[t]);
        ldw<W, CO>(A.r + off + vs[t] * W, rv[t]);
        ldw<W, CO>(A.q + off + vs[t] * W, qv[t]);
    }
    if (fetch) phase_scalars<2, CO, W>(A, I, in, it, S);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const float alpha = (float)S.sa[k];
            yv[t][k] = fmaf(alpha, dv[t][k], yv[t][k]);
            rv[t][k] = fmaf(-alpha, qv[t][k], rv[t][k]);
            if (valid[t] && k < I.C)
                run[k] = df_add(run[k], df_mul_exact(rv[t][k], nmv[t].y * rv[t][k]));
        }
        if (valid[t]) {
            stw<W>(A.y + off + v[t] * W, yv[t]);
            stw<W>(A.r + off + v[t] * W, rv[t]);
            if (A.zq) {
                float zv[W];
#pragma unroll
                for (int k = 0; k < W; ++k) zv[k] = nmv[t].y * rv[t][k];
                stw<W>(A.zq + off + v[t] * W, zv);
            }
        }
    }
}

// ------------------------------------------------ wide images (Cp > 4) ---
// The Cp / 4 consecutive threads of a vertex each take one float4 of its
// channel row (thread p: channels 4p .. 4p+3), so a neighbour's whole row is
// one coalesced request and the topology loads are shared (same address)
// by the vertex's threads.  A tile is walked in chunks of kVTile / P
// vertices.  A thread's channels stay fixed, so its products accumulate in
// run[] over the block's whole run of the image's tiles.
__device__ __forceinline__ void wide_lane(const InstDev& I, int& P, int& nvc, int& lv, int& p)
{
    P = I.Cp >> 2;
    nvc = kVTile / P;
    lv = threadIdx.x / P;
    p = threadIdx.x - lv * P;
}

// The z form of apply_tile_z for wide images: a neighbour contributes n_u
// and its z row (one float4 per lane) in place of {n, M^-1}, r and d_old.
template <bool CO>
__device__ __forceinline__ void apply_wide_z(const SolveArgs& A, const InstDev& I,
                                             const VTile& vt, const float* __restrict__ dold,
                                             float* __restrict__ dnew, PhaseSmem& S,
                                             DF (&run)[4])
{
    int P, nvc, lv, p;
    wide_lane(I, P, nvc, lv, p);
    const int cb = 4 * p, Cp = I.Cp;
    const int64_t base = pass_base(I, cb);
    const float* __restrict__ zb = A.zq + base;
    float beta[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) beta[k] = S.sf[min(cb + k, kMaxChannels - 1)];
    const int nverts = (int)(vt.v1 - vt.v0);
    for (int c0 = 0; c0 < nverts; c0 += nvc) {
        const int v = (int)vt.v0 + c0 + lv;
        const bool valid = lv < nvc && c0 + lv < nverts;
        const int vs = valid ? v : (int)vt.v0;
        int nb[10];
        load_neighbours(A, vs, nb);
        float zv[4], ov[4], qo[4];
        ldw<4, CO>(zb + vs * Cp, zv);
        ldw<4, CO>(dold + base + vs * Cp, ov);
        ldw<4, CO>(A.q + base + vs * Cp, qo);
        const float nv = valid ? A.nf[v] : 0.0f;
        const float av = valid ? A.a[v] : 0.0f;
        float sacc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) sacc[k] = 0.0f;
#pragma unroll
        for (int j = 0; j < 10; ++j) {
            const int u = nb[j];
            const float nu = A.nf[u];
            float zu[4];
            ldw<4, CO>(zb + u * Cp, zu);
#pragma unroll
            for (int k = 0; k < 4; ++k) sacc[k] = fmaf(nu, zv[k] - zu[k], sacc[k]);
        }
        const float lam_n = I.lam * nv;
        float dv[4], qh[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float az = fmaf(av, zv[k], lam_n * sacc[k]);
            dv[k] = fmaf(beta[k], ov[k], zv[k]);
            qh[k] = fmaf(beta[k], qo[k], az);
            if (valid && cb + k < I.C) run[k] = df_add(run[k], df_mul_exact(dv[k], qh[k]));
        }
        if (valid) {
            stw<4>(dnew + base + v * Cp, dv);
            stw<4>(A.q + base + v * Cp, qh);
        }
    }
}

template <bool COMP, bool CO, bool HIER = false, bool Z = false>
__device__ __forceinline__ void apply_wide(const SolveArgs& A, const InstDev& I, const VTile& vt,
                                           const float* __restrict__ dold,
                                           float* __restrict__ dnew, bool first, PhaseSmem& S,
                                           DF (&run)[4])
{
    static_assert(!Z || (!COMP && !HIER), "the z form is the FP32 Jacobi phase 1");
    if (Z) {
        apply_wide_z<CO>(A, I, vt, dold, dnew, S, run);
        return;
    }
    // HIER: z = M_hier^-1 r read in place of M^-1 r (as apply_tile)
    int P, nvc, lv, p;
    wide_lane(I, P, nvc, lv, p);
    const int cb = 4 * p, Cp = I.Cp;
    const float* __restrict__ rb = (HIER ? A.pyr.z : A.r) + pass_base(I, cb);
    const float* __restrict__ ob = dold + pass_base(I, cb);
    float beta[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) beta[k] = S.sf[min(cb + k, kMaxChannels - 1)];
    const int nverts = (int)(vt.v1 - vt.v0);
    for (int c0 = 0; c0 < nverts; c0 += nvc) {
        const int v = (int)vt.v0 + c0 + lv;
        const bool valid = lv < nvc && c0 + lv < nverts;
        const int vs = valid ? v : (int)vt.v0;
        const float2 nmv = valid ? A.nm[v] : make_float2(0.0f, 0.0f);
        const float av = valid ? A.a[v] : 0.0f;
        const float lam_n = I.lam * nmv.x;
        int nb[10];
        load_neighbours(A, vs, nb);
        float rv[4], dv[4];
        ldw<4, CO>(rb + vs * Cp, rv);
        const float mv = HIER ? 1.0f : nmv.y;
        if (first) {
#pragma unroll
            for (int k = 0; k < 4; ++k) dv[k] = mv * rv[k];
        } else {
            float ov[4];
            ldw<4, CO>(ob + vs * Cp, ov);
#pragma unroll
            for (int k = 0; k < 4; ++k) dv[k] = fmaf(beta[k], ov[k], mv * rv[k]);
        }
        DF sacc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) sacc[k] = {0.0f, 0.0f};
#pragma unroll
        for (int j = 0; j < 10; ++j) {
            const int u = nb[j];
            const float2 nmu = A.nm[u];
            float ru[4], du[4];
            ldw<4, CO>(rb + u * Cp, ru);
            const float mu = HIER ? 1.0f : nmu.y;
            if (first) {
#pragma unroll
                for (int k = 0; k < 4; ++k) du[k] = mu * ru[k];
            } else {
                float ou[4];
                ldw<4, CO>(ob + u * Cp, ou);
#pragma unroll
                for (int k = 0; k < 4; ++k) du[k] = fmaf(beta[k], ou[k], mu * ru[k]);
            }
            lap_acc<4, false>(sacc, nmu.x, dv, du);
        }
        float qh[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const DF q = lap_finish<false>(av, lam_n, dv[k], sacc[k]);
            qh[k] = q.hi;
            if (valid && cb + k < I.C)
                run[k] = df_add(run[k], df_mul_exact(dv[k], q.hi));
        }
        if (valid) {
            stw<4>(dnew + pass_base(I, cb) + v * Cp, dv);
            if (!COMP) stw<4>(A.q + pass_base(I, cb) + v * Cp, qh);
        }
    }
}

template <bool COMP, bool CO>
__device__ __forceinline__ void update_wide(const SolveArgs& A, const InstDev& I, const VTile& vt,
                                            const float* __restrict__ d, PhaseSmem& S,
                                            DF (&run)[4])
{
    int P, nvc, lv, p;
    wide_lane(I, P, nvc, lv, p);
    const int cb = 4 * p, Cp = I.Cp;
    const int64_t base = pass_base(I, cb);
    double alpha[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) alpha[k] = S.sa[min(cb + k, kMaxChannels - 1)];
    const int nverts = (int)(vt.v1 - vt.v0);
    for (int c0 = 0; c0 < nverts; c0 += nvc) {
        const int v = (int)vt.v0 + c0 + lv;
        const bool valid = lv < nvc && c0 + lv < nverts;
        const int vs = valid ? v : (int)vt.v0;
        const float2 nmv = valid ? A.nm[v] : make_float2(0.0f, 0.0f);
        float dv[4], yv[4], rv[4], rl[4], qv[4], yl[4];
        ldw<4, CO>(d + base + vs * Cp, dv);
        ldw<4, CO>(A.y + base + vs * Cp, yv);
        ldw<4, CO>(A.r + base + vs * Cp, rv);
        const bool ydf = COMP && A.ylo != nullptr;     // y as a double-float pair
        if (ydf) ldw<4, CO>(A.ylo + base + vs * Cp, yl);
        DF sacc[4];
        float av = 0.0f, lam_n = 0.0f, alv = 0.0f;
        if (COMP) {
            av = valid ? A.a[v] : 0.0f;
            alv = A.alo && valid ? A.alo[v] : 0.0f;
            lam_n = I.lam * nmv.x;
            ldw<4, CO>(A.rlo + base + vs * Cp, rl);
#pragma unroll
            for (int k = 0; k < 4; ++k) sacc[k] = {0.0f, 0.0f};
            int nb[10];
            load_neighbours(A, vs, nb);
#pragma unroll
            for (int j = 0; j < 10; ++j) {
                const int u = nb[j];
                const float nu = A.nm[u].x;
                float du[4];
                ldw<4, CO>(d + base + u * Cp, du);
                lap_acc<4, true>(sacc, nu, dv, du);
            }
        } else {
            ldw<4, CO>(A.q + base + vs * Cp, qv);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (ydf) {
                const DF yy = df_add(DF{yv[k], yl[k]}, df_mul_f(df_from_double(alpha[k]), dv[k]));
                yv[k] = yy.hi;
                yl[k] = yy.lo;
            } else {
                yv[k] = fmaf((float)alpha[k], dv[k], yv[k]);
            }
            if (COMP) {
                const DF q = lap_finish<true>(av, lam_n, dv[k], sacc[k], alv);
                const DF r = df_add(DF{rv[k], rl[k]}, df_neg(df_mul(df_from_double(alpha[k]), q)));
                rv[k] = r.hi;
                rl[k] = r.lo;
            } else {
                rv[k] = fmaf(-(float)alpha[k], qv[k], rv[k]);
            }
            if (valid && cb + k < I.C) run[k] = df_add(run[k], df_mul_exact(rv[k], nmv.y * rv[k]));
        }
        if (valid) {
            stw<4>(A.y + base + v * Cp, yv);
            stw<4>(A.r + base + v * Cp, rv);
            if (COMP) stw<4>(A.rlo + base + v * Cp, rl);
            if (ydf) stw<4>(A.ylo + base + v * Cp, yl);
            if (!COMP && A.zq) {
                float zv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) zv[k] = nmv.y * rv[k];
                stw<4>(A.zq + base + v * Cp, zv);
            }
        }
    }
}

// Per-channel sums of the block's run over a wide image, into the run's
// slot: thread sums first go to shared memory; G = kVTile / Cp threads per
// channel each add every G-th vertex lane in order, then one thread per
// channel adds the G group sums in order.
__device__ void flush_wide(DF (&run)[4], int Cp, int C, int ntiles, int64_t part_base, int slot,
                           float2* part, WideSmem& Wd)
{
    const int P = Cp >> 2, nvc = kVTile / P, lv = threadIdx.x / P;
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        Wd.lane[t][k] = lv < nvc ? run[k] : DF{0.0f, 0.0f};
        run[k] = {0.0f, 0.0f};
    }
    __syncthreads();
    const int G = kVTile / Cp;
    if (t < G * Cp) {
        const int ch = t % Cp, g = t / Cp;
        DF acc = {0.0f, 0.0f};
        for (int l = g; l < nvc; l += G) acc = df_add(acc, Wd.lane[l * P + (ch >> 2)][ch & 3]);
        Wd.group[g * Cp + ch] = acc;
    }
    __syncthreads();
    if (t < C) {
        DF acc = Wd.group[t];
        for (int g = 1; g < G; ++g) acc = df_add(acc, Wd.group[g * Cp + t]);
        part[part_base + (int64_t)t * ntiles + slot] = make_float2(acc.hi, acc.lo);
    }
    __syncthreads();
}

// Store the block's run partial (channels of one pass) in the slot of the
// first tile of the run; the other slots of the run were written as exact
// zeros as their tiles were visited, so the reducers' sums are unchanged.
__device__ __forceinline__ void flush_run(DF (&run)[4], int W, int C, int ntiles,
                                          int64_t part_base, int slot, float2* part,
                                          PhaseSmem& S)
{
    if (W == 1) {
        DF r1[1] = {run[0]};
        store_partials<1>(r1, C, ntiles, part_base, 0, slot, part, S.red);
    } else if (W == 2) {
        DF r2[2] = {run[0], run[1]};
        store_partials<2>(r2, C, ntiles, part_base, 0, slot, part, S.red);
    } else {
        store_partials<4>(run, C, ntiles, part_base, 0, slot, part, S.red);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) run[k] = {0.0f, 0.0f};
}

// Loop over a block's chunk of tiles for one phase.  At each new image the
// block reduces the previous phase's partials of that image and forms the CG
// scalars (phase 1: delta_it and beta; phase 2: alpha), then dispatches each
// tile on the image's pass width.  When an image's channels fit one pass the
// products are accumulated over the run of its tiles in this chunk.
template <int PHASE, bool COMP, bool CO, int WMAX, bool HIER = false, bool Z = false>
__device__ void phase_run(const SolveArgs& A, const float* __restrict__ dsrc,
                          float* __restrict__ ddst, int it, int t0, int t1, PhaseSmem& S,
                          WideSmem& Wd)
{
    const int slot = it & 1;
    const bool first = it == 0;
    float2* const out = PHASE == 1 ? A.part_dq : A.part_rs[slot ^ 1];
    const float2* const in = PHASE == 1 ? A.part_rs[slot] : A.part_dq;
    int cur = -1, run_tile = 0, run_C = 0, run_Cp = 1, run_W = 1, run_ntiles = 0;
    int64_t run_base = 0;
    bool fetch = false;
    DF run[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) run[k] = {0.0f, 0.0f};
    for (int tile = t0; tile < t1; ++tile) {
        const VTile vt = A.vt[tile];
        const InstDev I = A.inst[vt.inst];
        if (vt.inst != cur) {
            if (cur >= 0) {
                if (WMAX == 4 && run_Cp > 4)
                    flush_wide(run, run_Cp, run_C, run_ntiles, run_base, run_tile, out, Wd);
                else
                    flush_run(run, run_W, run_C, run_ntiles, run_base, run_tile, out, S);
            }
            fetch = true;
            cur = vt.inst;
            run_tile = vt.t_in_inst;
            run_C = I.C;
            run_Cp = I.Cp;
            run_W = I.Cp < 4 ? I.Cp : 4;
            run_ntiles = I.ntiles;
            run_base = I.part_base;
        } else if ((int)threadIdx.x < I.C) {
            out[I.part_base + (int64_t)threadIdx.x * I.ntiles + vt.t_in_inst] =
                make_float2(0.0f, 0.0f);
        }
        if (PHASE == 2 && !COMP && !(WMAX == 4 && I.Cp > 4) && tile + 1 < t1 &&
            A.vt[tile + 1].inst == vt.inst) {
            // two tiles of the same image at once (the second is never a run start)
            const VTile vb = A.vt[tile + 1];
            if ((int)threadIdx.x < I.C)
                out[I.part_base + (int64_t)threadIdx.x * I.ntiles + vb.t_in_inst] =
                    make_float2(0.0f, 0.0f);
            if (WMAX == 1 || I.Cp == 1)
                update_pair<1, CO>(A, I, vt, vb, dsrc, S, run, fetch, in, it);
            else if (WMAX == 2 || I.Cp == 2)
                update_pair<2, CO>(A, I, vt, vb, dsrc, S, run, fetch, in, it);
            else
                update_pair<4, CO>(A, I, vt, vb, dsrc, S, run, fetch, in, it);
            fetch = false;
            ++tile;
            continue;
        }
        if (WMAX == 4 && I.Cp > 4) {
            if (fetch) phase_scalars<PHASE, CO, 4>(A, I, in, it, S);
            if (PHASE == 1) apply_wide<COMP, CO, HIER, Z>(A, I, vt, dsrc, ddst, first, S, run);
            else update_wide<COMP, CO>(A, I, vt, dsrc, S, run);
        } else if (PHASE == 1) {
            if (WMAX == 1 || I.Cp == 1)
                apply_tile<1, COMP, CO, HIER, Z>(A, I, vt, dsrc, ddst, first, S, run, fetch, in, it);
            else if (WMAX == 2 || I.Cp == 2)
                apply_tile<2, COMP, CO, HIER, Z>(A, I, vt, dsrc, ddst, first, S, run, fetch, in, it);
            else
                apply_tile<4, COMP, CO, HIER, Z>(A, I, vt, dsrc, ddst, first, S, run, fetch, in, it);
        } else {
            if (WMAX == 1 || I.Cp == 1)
                update_tile<1, COMP, CO>(A, I, vt, dsrc, S, run, fetch, in, it);
            else if (WMAX == 2 || I.Cp == 2)
                update_tile<2, COMP, CO>(A, I, vt, dsrc, S, run, fetch, in, it);
            else
                update_tile<4, COMP, CO>(A, I, vt, dsrc, S, run, fetch, in, it);
        }
        fetch = false;
    }
    if (cur >= 0) {
        if (WMAX == 4 && run_Cp > 4)
            flush_wide(run, run_Cp, run_C, run_ntiles, run_base, run_tile, out, Wd);
        else
            flush_run(run, run_W, run_C, run_ntiles, run_base, run_tile, out, S);
    }
}

// Phase kernels are instantiated per widest pass of the batch (WMAX = the
// largest Cp, capped at 4): a batch of one- and two-channel images gets the
// register budget of the narrow bodies and with it more resident warps.
// Resident blocks per SM asked of the compiler, per WMAX (measured best: the
// gathers are latency-bound, and more resident warps beat deeper per-thread
// load batches once those drop below ~64 registers for W <= 2).
template <int WMAX>
constexpr int phase_min_blocks() { return WMAX <= 2 ? 4 : 2; }

template <int WMAX, bool COMP, bool HIER = false, bool Z = false>
__global__ void __launch_bounds__(kVTile, phase_min_blocks<WMAX>())
pcg_apply_kernel(SolveArgs A, const float* __restrict__ dold, float* __restrict__ dnew, int it)
{
    __shared__ PhaseSmem S;
    __shared__ WideSmem Wd;
    int t0, t1;
    block_chunk(A.nvt, t0, t1);
    phase_run<1, COMP, false, WMAX, HIER, Z>(A, dold, dnew, it, t0, t1, S, Wd);
}

template <int WMAX, bool COMP>
__global__ void __launch_bounds__(kVTile, phase_min_blocks<WMAX>())
pcg_update_kernel(SolveArgs A, const float* __restrict__ d, int it)
{
    __shared__ PhaseSmem S;
    __shared__ WideSmem Wd;
    int t0, t1;
    block_chunk(A.nvt, t0, t1);
    phase_run<2, COMP, false, WMAX>(A, d, nullptr, it, t0, t1, S, Wd);
}

// ------------------------------------------ single-reduction PCG form ---
// The Chronopoulos-Gear form of Alg. 2 (same iterates in exact arithmetic):
// with u = M^-1 r, w = A u and s = A p carried along, iteration i is
//   beta = gamma_i / gamma_(i-1),  alpha = gamma_i / (mu_i - beta gamma_i / alpha_(i-1)),
//   s_i = w_i + beta s_(i-1),  p_i = u_i + beta p_(i-1),  y += alpha p_i,
//   r_(i+1) = r_i - alpha s_i,  u_(i+1) = M^-1 r_(i+1),  w_(i+1) = A u_(i+1),
//   gamma_(i+1) = r_(i+1)^T u_(i+1),  mu_(i+1) = w_(i+1)^T u_(i+1),
// one launch per iteration: each thread forms s_i, r_(i+1), u_(i+1) for its
// vertex and, from gathered (r_i, w_i, s_(i-1)), for each neighbour, so no
// second pass is needed; both inner products go to one set of partials.
// Buffers by iteration parity: r in r / r_lo, w in d[0] / d[1], s in aux[];
// p (in q) and y are updated in place.  Guards as Alg. 2's: beta = 0 when
// gamma_(i-1) = 0; the correction term is dropped when beta = 0 or
// alpha_(i-1) = 0; alpha = 0 when gamma = 0 or the denominator is not
// positive.  FP32 vectors, images with at most 4 channels.
__device__ __forceinline__ float* cg_r(const SolveArgs& A, int k) { return k ? A.rlo : A.r; }

// beta (S.sf) and alpha (S.sa) of iteration it for image I, from the
// partials of gamma_it and mu_it and the stored gamma, alpha of iteration
// it - 1; stores gamma_it and alpha_it.  Whole block; ends with a barrier.
template <int W>
__device__ void cg_scalars(const SolveArgs& A, const InstDev& I, int it, PhaseSmem& S)
{
    constexpr int H = W == 1 ? 8 : W == 2 ? 4 : 2;
    const int slot = it & 1;
    __syncthreads();
    reduce_partials_all<W, H>(A.part_rs[slot], I, S.sd, S.red);
    reduce_partials_all<W, H>(A.part_mu[slot], I, S.sd2, S.red);
    for (int ch = threadIdx.x; ch < I.Cp; ch += blockDim.x) {
        if (ch >= I.C) {
            S.sf[ch] = 0.0f;
            S.sa[ch] = 0.0;
            continue;
        }
        const double gamma = S.sd[ch], mu = S.sd2[ch];
        double beta = 0.0, den = mu;
        bool stalled = gamma == 0.0;
        if (it > 0) {
            const double gold = A.scal[I.pc + ch].gam[slot ^ 1];
            const double aold = A.scal[I.pc + ch].alp[slot ^ 1];
            stalled = cg_stalled(gamma, A.scal[I.pc + ch].delta0);
            beta = gold != 0.0 && !stalled ? gamma / gold : 0.0;
            if (beta != 0.0 && aold != 0.0) den = mu - beta * gamma / aold;
        } else {
            A.scal[I.pc + ch].delta0 = gamma;
        }
        const double alpha = (!stalled && den > 0.0) ? gamma / den : 0.0;
        S.sf[ch] = (float)beta;
        S.sa[ch] = alpha;
        A.scal[I.pc + ch].gam[slot] = gamma;   // same values from every block
        A.scal[I.pc + ch].alp[slot] = alpha;
    }
    __syncthreads();
}

// Iteration it on one tile (Cp = W).  last: only p and y are needed.
template <int W>
__device__ __forceinline__ void cg_tile(const SolveArgs& A, const InstDev& I, const VTile& vt,
                                        int it, bool last, PhaseSmem& S, DF (&rg)[4],
                                        DF (&rm)[4], bool fetch)
{
    const int v = (int)vt.v0 + (int)threadIdx.x;
    const bool valid = v < (int)vt.v1;
    const int vs = valid ? v : (int)vt.v0;
    const int cur = it & 1, nxt = cur ^ 1;
    const int64_t off = I.vec_base - I.voff * W;
    const float* __restrict__ rb = cg_r(A, cur) + off;      // r_i
    const float* __restrict__ wb = A.d[cur] + off;          // w_i
    const float* __restrict__ sb = A.aux[nxt] + off;        // s_(i-1)
    const bool first = it == 0;
    const float2 nmv = A.nm[vs];
    const float av = A.a[vs];
    float rv[W], wv[W], so[W], pv[W], yv[W];
    ldw<W, false>(rb + vs * W, rv);
    ldw<W, false>(wb + vs * W, wv);
    ldw<W, false>(A.y + off + vs * W, yv);
    if (!first) {
        ldw<W, false>(sb + vs * W, so);
        ldw<W, false>(A.q + off + vs * W, pv);
    }
    if (fetch) cg_scalars<W>(A, I, it, S);
    float beta[W], alpha[W], r1[W], u1[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
        beta[k] = S.sf[k];
        alpha[k] = (float)S.sa[k];
        const float si = first ? wv[k] : fmaf(beta[k], so[k], wv[k]);
        const float ui = nmv.y * rv[k];
        pv[k] = first ? ui : fmaf(beta[k], pv[k], ui);
        yv[k] = fmaf(alpha[k], pv[k], yv[k]);
        r1[k] = fmaf(-alpha[k], si, rv[k]);
        u1[k] = nmv.y * r1[k];
        so[k] = si;
    }
    if (valid) {
        stw<W>(A.y + off + v * W, yv);
        stw<W>(A.q + off + v * W, pv);
    }
    if (last) return;
    float lap[W];
#pragma unroll
    for (int k = 0; k < W; ++k) lap[k] = 0.0f;
#pragma unroll
    for (int j = 0; j < 10; ++j) {
        const int u0 = A.nbr[(int64_t)j * A.nbr_stride + vs];
        const int u = u0 >= 0 ? u0 : vs;        // absent: the vertex itself, term 0
        const float2 nm = A.nm[u];
        float ru[W], wu[W], su[W];
        ldw<W, false>(rb + u * W, ru);
        ldw<W, false>(wb + u * W, wu);
        if (!first) ldw<W, false>(sb + u * W, su);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const float s_u = first ? wu[k] : fmaf(beta[k], su[k], wu[k]);
            const float u_u = nm.y * fmaf(-alpha[k], s_u, ru[k]);
            lap[k] = fmaf(nm.x, u1[k] - u_u, lap[k]);
        }
    }
    const float lam_n = I.lam * nmv.x;
    float w1[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
        w1[k] = fmaf(av, u1[k], lam_n * lap[k]);
        if (valid && k < I.C) {
            rg[k] = df_add(rg[k], df_mul_exact(r1[k], u1[k]));
            rm[k] = df_add(rm[k], df_mul_exact(w1[k], u1[k]));
        }
    }
    if (valid) {
        stw<W>(A.aux[cur] + off + v * W, so);
        stw<W>(cg_r(A, nxt) + off + v * W, r1);
        stw<W>(A.d[nxt] + off + v * W, w1);
    }
}

// Set-up on one tile: w_0 = A M^-1 r_0 into d[0] and the products w_0^T u_0
// into rm (gamma_0 = r_0^T M^-1 r_0 comes from the initial residual).
template <int W>
__device__ __forceinline__ void cg_w0_tile(const SolveArgs& A, const InstDev& I, const VTile& vt,
                                           DF (&rm)[4])
{
    const int v = (int)vt.v0 + (int)threadIdx.x;
    const bool valid = v < (int)vt.v1;
    const int vs = valid ? v : (int)vt.v0;
    const int64_t off = I.vec_base - I.voff * W;
    const float* __restrict__ rb = A.r + off;
    const float2 nmv = A.nm[vs];
    const float av = A.a[vs];
    float rv[W], u0[W], lap[W];
    ldw<W, false>(rb + vs * W, rv);
#pragma unroll
    for (int k = 0; k < W; ++k) {
        u0[k] = nmv.y * rv[k];
        lap[k] = 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 10; ++j) {
        const int u0i = A.nbr[(int64_t)j * A.nbr_stride + vs];
        const int u = u0i >= 0 ? u0i : vs;
        const float2 nm = A.nm[u];
        float ru[W];
        ldw<W, false>(rb + u * W, ru);
#pragma unroll
        for (int k = 0; k < W; ++k) lap[k] = fmaf(nm.x, u0[k] - nm.y * ru[k], lap[k]);
    }
    const float lam_n = I.lam * nmv.x;
    float w0[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
        w0[k] = fmaf(av, u0[k], lam_n * lap[k]);
        if (valid && k < I.C) rm[k] = df_add(rm[k], df_mul_exact(w0[k], u0[k]));
    }
    if (valid) stw<W>(A.d[0] + off + v * W, w0);
}

// A block's chunk of tiles for one single-reduction iteration (it >= 0) or
// the set-up (it < 0): per image, the CG scalars at the start and the
// products accumulated over the block's run of the image's tiles.
template <int WMAX>
__device__ void cg_run(const SolveArgs& A, int it, bool last, int t0, int t1, PhaseSmem& S)
{
    const int nxt = (it + 1) & 1;              // set-up (it = -1) writes slot 0
    float2* const out_g = A.part_rs[nxt];
    float2* const out_m = A.part_mu[nxt];
    int cur = -1, run_tile = 0, run_C = 0, run_W = 1, run_ntiles = 0;
    int64_t run_base = 0;
    bool fetch = false;
    DF rg[4], rm[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) rg[k] = rm[k] = {0.0f, 0.0f};
    for (int tile = t0; tile < t1; ++tile) {
        const VTile vt = A.vt[tile];
        const InstDev I = A.inst[vt.inst];
        if (vt.inst != cur) {
            if (cur >= 0 && !last) {
                if (it >= 0) flush_run(rg, run_W, run_C, run_ntiles, run_base, run_tile, out_g, S);
                flush_run(rm, run_W, run_C, run_ntiles, run_base, run_tile, out_m, S);
            }
            fetch = it >= 0;
            cur = vt.inst;
            run_tile = vt.t_in_inst;
            run_C = I.C;
            run_W = I.Cp < 4 ? I.Cp : 4;
            run_ntiles = I.ntiles;
            run_base = I.part_base;
        } else if (!last && (int)threadIdx.x < I.C) {
            const int64_t o = I.part_base + (int64_t)threadIdx.x * I.ntiles + vt.t_in_inst;
            if (it >= 0) out_g[o] = make_float2(0.0f, 0.0f);
            out_m[o] = make_float2(0.0f, 0.0f);
        }
        if (it < 0) {
            if (WMAX == 1 || I.Cp == 1) cg_w0_tile<1>(A, I, vt, rm);
            else if (WMAX == 2 || I.Cp == 2) cg_w0_tile<2>(A, I, vt, rm);
            else cg_w0_tile<4>(A, I, vt, rm);
        } else {
            if (WMAX == 1 || I.Cp == 1) cg_tile<1>(A, I, vt, it, last, S, rg, rm, fetch);
            else if (WMAX == 2 || I.Cp == 2) cg_tile<2>(A, I, vt, it, last, S, rg, rm, fetch);
            else cg_tile<4>(A, I, vt, it, last, S, rg, rm, fetch);
        }
        fetch = false;
    }
    if (cur >= 0 && !last) {
        if (it >= 0) flush_run(rg, run_W, run_C, run_ntiles, run_base, run_tile, out_g, S);
        flush_run(rm, run_W, run_C, run_ntiles, run_base, run_tile, out_m, S);
    }
}

template <int WMAX>
constexpr int single_min_blocks() { return WMAX <= 2 ? 3 : 2; }

template <int WMAX>
__global__ void __launch_bounds__(kVTile, single_min_blocks<WMAX>())
pcg_single_kernel(SolveArgs A, int it, int last)
{
    __shared__ PhaseSmem S;
    int t0, t1;
    block_chunk(A.nvt, t0, t1);
    cg_run<WMAX>(A, it, last != 0, t0, t1, S);
}

// ------------------------------------- hierarchical preconditioner ---
// The bilateral-space pyramid passes of Sec. 4 (levels built by pyramid.cu;
// see PyrDev).  P sums children into parents level by level, in ascending
// child order and in double-float arithmetic: deterministic, and free of
// the cancellation error that FP32 sums of a converging, oscillating
// residual would feed back into CG as a changing preconditioner.  P^T
// broadcasts parents back down, adding each level's own scaled value:
//   M_hier^-1 r = P^T(coef o P(r)),  coef = w(k) P(1) / P(diag A),
//   y_hier = P^T(cinit o P(b)) / P^T(cinit o P(S c)),  cinit = w_init(k) / P(1).
// The weights are FP32 (a rounded weight leaves M_hier^-1 linear and
// symmetric).  Launches: level 1 from the grid (pyr_gather0), levels 2 and
// 3 (pyr_gather), levels >= 4 of each image up and back down in one block
// per image (pyr_tail), levels 3 .. 1 down (pyr_down_low), and level 0
// (pyr_precond0 / pyr_init0).  A level
// vector holds nc double-float values per vertex: W channels (the widest
// image's Cp; an image uses its first Cp), plus S c and diag(A) in the setup
// pass (nc = W + 2).

__device__ __forceinline__ DF pyr_ld(const float2* p) { const float2 v = *p; return {v.x, v.y}; }
__device__ __forceinline__ void pyr_st(float2* p, DF v) { *p = make_float2(v.hi, v.lo); }

// Level 1 parents sum their grid children: channels [0, cp) from the CG
// vector src (the child image's layout), and with scal, S c into channel W
// and diag(A) into channel W + 1.
__global__ void __launch_bounds__(256)
pyr_gather0_kernel(SolveArgs A, const float* __restrict__ src, int nc, int scal)
{
    const PyrDev& P = A.pyr;
    const int W = P.W;
    const int64_t np = P.off[2] - P.off[1];
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        // a parent's children are grid vertices of its own image
        const InstDev& I = A.inst[P.vimg[P.off[1] + p]];
        const int cp = I.Cp;
        const float* base = src + I.vec_base - I.voff * cp;
        const int32_t j0 = P.child_off[p], j1 = P.child_off[p + 1];
        float2* dst = P.lv + p * nc;
        for (int c0 = 0; c0 < W; c0 += 4) {          // 4 channels per walk of the children
            DF acc[4], asc = {0.0f, 0.0f}, adg = {0.0f, 0.0f};
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] = DF{0.0f, 0.0f};
            const bool sc_here = scal && c0 == 0;
#pragma unroll 4
            for (int32_t j = j0; j < j1; ++j) {
                const int64_t c = P.child_idx[j];
                const float* x = base + c * cp + c0;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (c0 + k < cp) acc[k] = df_add_f(acc[k], x[k]);
                if (sc_here) {
                    asc = df_add_f(asc, P.scv[c]);
                    adg = df_add_f(adg, P.dg[c]);
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (c0 + k < W) pyr_st(dst + c0 + k, acc[k]);
            if (sc_here) {
                pyr_st(dst + W, asc);
                pyr_st(dst + W + 1, adg);
            }
        }
    }
}

// one parent g (absolute, level k + 1 >= 2) sums its level-k children
__device__ __forceinline__ void pyr_sum_children(const PyrDev& P, int k, int64_t g, int nc)
{
    const int64_t gl = g - P.off[1];
    const int32_t j0 = P.child_off[gl], j1 = P.child_off[gl + 1];
    float2* dst = P.lv + gl * nc;
    for (int c0 = 0; c0 < nc; c0 += kPyrMaxNc) {     // kPyrMaxNc values per walk
        DF acc[kPyrMaxNc];
#pragma unroll
        for (int ch = 0; ch < kPyrMaxNc; ++ch) acc[ch] = DF{0.0f, 0.0f};
#pragma unroll 4
        for (int32_t j = j0; j < j1; ++j) {
            const float2* x = P.lv + (P.off[k] + P.child_idx[j] - P.off[1]) * nc + c0;
#pragma unroll
            for (int ch = 0; ch < kPyrMaxNc; ++ch)
                if (c0 + ch < nc) acc[ch] = df_add(acc[ch], pyr_ld(x + ch));
        }
#pragma unroll
        for (int ch = 0; ch < kPyrMaxNc; ++ch)
            if (c0 + ch < nc) pyr_st(dst + c0 + ch, acc[ch]);
    }
}

// Level k + 1 from level k, every image.
__global__ void __launch_bounds__(256)
pyr_gather_kernel(SolveArgs A, int k, int nc)
{
    const PyrDev& P = A.pyr;
    const int64_t n = P.off[k + 2] - P.off[k + 1];
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        pyr_sum_children(P, k, P.off[k + 1] + p, nc);
}

// Levels >= 4 of one image per block: with up, parents of levels 4 .. top
// sum their children; with wt, levels top .. 4 take x <- wt o x + (parent's
// x) (the image's top has no parent).  Images whose own pyramid has at most
// four levels have nothing here.
__global__ void __launch_bounds__(kPyrTailThreads)
pyr_tail_kernel(SolveArgs A, int nc, int up, const float* __restrict__ wt)
{
    const PyrDev& P = A.pyr;
    const int n = A.ninst;
    for (int im = blockIdx.x; im < n; im += gridDim.x) {
        const int Ki = P.kimg[im];
        if (up) {
            for (int k = 3; k + 1 < Ki; ++k) {
                const int64_t g0 = P.ioff[(k + 1) * (n + 1) + im];
                const int64_t g1 = P.ioff[(k + 1) * (n + 1) + im + 1];
                for (int64_t g = g0 + threadIdx.x; g < g1; g += blockDim.x)
                    pyr_sum_children(P, k, g, nc);
                __syncthreads();
            }
        }
        if (wt) {
            for (int k = Ki - 1; k >= 4; --k) {
                const int64_t g0 = P.ioff[k * (n + 1) + im];
                const int64_t g1 = P.ioff[k * (n + 1) + im + 1];
                const bool top = k == Ki - 1;
                for (int64_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
                    float2* x = P.lv + (g - P.off[1]) * nc;
                    const float2* u =
                        top ? nullptr : P.lv + (P.off[k + 1] + P.parent[g] - P.off[1]) * nc;
                    const float w = wt[g];
                    for (int ch = 0; ch < nc; ++ch) {
                        const DF xv = df_mul_f(pyr_ld(x + ch), w);
                        pyr_st(x + ch, top ? xv : df_add(xv, pyr_ld(u + ch)));
                    }
                }
                __syncthreads();
            }
        }
    }
}

// coef = w(k) P(1) / P(diag A) on every pyramid vertex (w(0) = 1,
// w(k) = 2^-(5 + k)); 0 where P(diag A) <= 0 and on the vertices an image
// keeps past its own top (P(1) = 0 there).  P(diag A) of levels >= 1 is the
// setup pass's channel W + 1.
__global__ void __launch_bounds__(256)
pyr_coef_kernel(SolveArgs A)
{
    const PyrDev& P = A.pyr;
    const int nc = P.W + 2;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < P.off[P.K];
         g += (int64_t)gridDim.x * blockDim.x) {
        int k = 0;
        while (g >= P.off[k + 1]) ++k;
        float D;
        if (k == 0) {
            D = P.dg[g];
        } else {
            const float2 d = P.lv[(g - P.off[1]) * nc + P.W + 1];
            D = d.x + d.y;
        }
        const float w = k == 0 ? 1.0f : exp2f(-(float)(5 + k));
        P.coef[g] = D > 0.0f ? w * P.cnt[g] / D : 0.0f;
    }
}

// The down-sweep of levels 3, 2 and 1, finished for each level-1 vertex in
// place (weights wt): x1 = wt o l1 + x2, x2 = wt o l2 + x3 and x3 = wt o l3
// + x4 along the vertex's ancestors, with x4 the level-4 ancestor's final
// value from pyr_tail, each while the image's own pyramid reaches that
// level (the image's top has no parent).  Levels 2 and 3 are read, not
// written, so every level-1 vertex sees them whole.
__global__ void __launch_bounds__(256)
pyr_down_low_kernel(SolveArgs A, int nc, const float* __restrict__ wt)
{
    const PyrDev& P = A.pyr;
    const int64_t n1 = P.off[2] - P.off[1];
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n1;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g1 = P.off[1] + p;
        const int Ki = P.kimg[P.vimg[g1]];
        float2* x1 = P.lv + p * nc;
        const float w1 = wt[g1];
        const float2 *l2 = nullptr, *l3 = nullptr, *l4 = nullptr;
        float w2 = 0.0f, w3 = 0.0f;
        if (Ki > 2) {
            const int64_t g2 = P.off[2] + P.parent[g1];
            w2 = wt[g2];
            l2 = P.lv + (g2 - P.off[1]) * nc;
            if (Ki > 3) {
                const int64_t g3 = P.off[3] + P.parent[g2];
                w3 = wt[g3];
                l3 = P.lv + (g3 - P.off[1]) * nc;
                if (Ki > 4) l4 = P.lv + (P.off[4] + P.parent[g3] - P.off[1]) * nc;
            }
        }
        for (int ch = 0; ch < nc; ++ch) {
            DF x = df_mul_f(pyr_ld(x1 + ch), w1);
            if (Ki > 2) {
                DF x2 = df_mul_f(pyr_ld(l2 + ch), w2);
                if (Ki > 3) {
                    DF x3 = df_mul_f(pyr_ld(l3 + ch), w3);
                    if (Ki > 4) x3 = df_add(x3, pyr_ld(l4 + ch));
                    x2 = df_add(x2, x3);
                }
                x = df_add(x, x2);
            }
            pyr_st(x1 + ch, x);
        }
    }
}

// Level 0 of the preconditioner, per vertex tile: z = coef r + x1(ancestors);
// partials of r^T z into `out` for every tile.
template <int W>
__device__ __forceinline__ void pyr_precond_tile(const SolveArgs& A, const InstDev& I,
                                                 const VTile& vt, float2* out, PhaseSmem& S)
{
    const PyrDev& P = A.pyr;
    const int v = (int)vt.v0 + (int)threadIdx.x;
    const bool valid = v < (int)vt.v1;
    const int vs = valid ? v : (int)vt.v0;
    const int64_t off = I.vec_base - I.voff * W;
    float rv[W], zv[W];
    ldw<W, false>(A.r + off + vs * W, rv);
    const float c0 = P.coef[vs];
    float x[W];
#pragma unroll
    for (int k = 0; k < W; ++k) x[k] = 0.0f;
    if (P.K > 1) {                      // level-1 ancestor's final value (pyr_down_low)
        const float2* x1 = P.lv + (int64_t)P.parent[vs] * P.W;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const float2 t = x1[k];
            x[k] = t.x + t.y;
        }
    }
    DF acc[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
        zv[k] = fmaf(c0, rv[k], x[k]);
        acc[k] = valid && k < I.C ? df_mul_exact(rv[k], zv[k]) : DF{0.0f, 0.0f};
    }
    if (valid) stw<W>(P.z + off + v * W, zv);
    store_partials<W>(acc, I.C, I.ntiles, I.part_base, 0, vt.t_in_inst, out, S.red);
}

// Level 0 on a tile of a wide image (Cp > 4), in the wide phases' lane
// layout (the Cp / 4 threads of a vertex take one float4 of its row each);
// products r z accumulate in run[] over the block's run of the image's
// tiles.
__device__ __forceinline__ void pyr_precond_wide(const SolveArgs& A, const InstDev& I,
                                                 const VTile& vt, DF (&run)[4])
{
    const PyrDev& P = A.pyr;
    int Pn, nvc, lv, p;
    wide_lane(I, Pn, nvc, lv, p);
    const int cb = 4 * p, Cp = I.Cp;
    const int64_t base = pass_base(I, cb);
    const int nverts = (int)(vt.v1 - vt.v0);
    for (int c0 = 0; c0 < nverts; c0 += nvc) {
        const int v = (int)vt.v0 + c0 + lv;
        const bool valid = lv < nvc && c0 + lv < nverts;
        const int vs = valid ? v : (int)vt.v0;
        float rv[4], zv[4], x[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        ldw<4, false>(A.r + base + (int64_t)vs * Cp, rv);
        const float c0f = P.coef[vs];
        if (P.K > 1) {
            const float2* x1 = P.lv + (int64_t)P.parent[vs] * P.W + cb;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 t = x1[k];
                x[k] = t.x + t.y;
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            zv[k] = fmaf(c0f, rv[k], x[k]);
            if (valid && cb + k < I.C) run[k] = df_add(run[k], df_mul_exact(rv[k], zv[k]));
        }
        if (valid) stw<4>(P.z + base + (int64_t)v * Cp, zv);
    }
}

__global__ void __launch_bounds__(kVTile)
pyr_precond0_kernel(SolveArgs A, float2* out)
{
    __shared__ PhaseSmem S;
    __shared__ WideSmem Wd;
    int t0, t1;
    block_chunk(A.nvt, t0, t1);
    // wide images: one partial per run of the block's tiles of an image,
    // stored in the run's first slot, the run's other slots zero (as in the
    // phase kernels)
    int cur = -1, run_tile = 0, run_C = 0, run_Cp = 8, run_ntiles = 0;
    int64_t run_base = 0;
    DF run[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) run[k] = {0.0f, 0.0f};
    for (int tile = t0; tile < t1; ++tile) {
        const VTile vt = A.vt[tile];
        const InstDev I = A.inst[vt.inst];
        if (I.Cp > 4) {
            if (vt.inst != cur) {
                if (cur >= 0) flush_wide(run, run_Cp, run_C, run_ntiles, run_base, run_tile, out, Wd);
                cur = vt.inst;
                run_tile = vt.t_in_inst;
                run_C = I.C;
                run_Cp = I.Cp;
                run_ntiles = I.ntiles;
                run_base = I.part_base;
            } else if ((int)threadIdx.x < I.C) {
                out[I.part_base + (int64_t)threadIdx.x * I.ntiles + vt.t_in_inst] =
                    make_float2(0.0f, 0.0f);
            }
            pyr_precond_wide(A, I, vt, run);
            continue;
        }
        if (cur >= 0) {
            flush_wide(run, run_Cp, run_C, run_ntiles, run_base, run_tile, out, Wd);
            cur = -1;
        }
        if (I.Cp == 1) pyr_precond_tile<1>(A, I, vt, out, S);
        else if (I.Cp == 2) pyr_precond_tile<2>(A, I, vt, out, S);
        else pyr_precond_tile<4>(A, I, vt, out, S);
    }
    if (cur >= 0) flush_wide(run, run_Cp, run_C, run_ntiles, run_base, run_tile, out, Wd);
}

// Level 0 of the initialisation: y = (cinit b + x1_b) / (cinit S c + x1_Sc),
// 0 where the denominator is not positive; b is in r after the splat.
__global__ void __launch_bounds__(256)
pyr_init0_kernel(SolveArgs A)
{
    const PyrDev& P = A.pyr;
    const int W = P.W, nc = W + 2;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < P.off[1];
         v += (int64_t)gridDim.x * blockDim.x) {
        const int im = P.vimg[v];
        const InstDev& I = A.inst[im];
        const int64_t o = I.vec_base + (v - I.voff) * I.Cp;
        // level-1 ancestor's final values (pyr_down_low): channels, then S c
        const float2* x1 = P.K > 1 ? P.lv + (int64_t)P.parent[v] * nc : nullptr;
        const float ci = P.cinit[v];
        const float den = fmaf(ci, P.scv[v], x1 ? x1[W].x + x1[W].y : 0.0f);
        for (int ch = 0; ch < I.Cp; ++ch) {
            const float num = fmaf(ci, A.r[o + ch], x1 ? x1[ch].x + x1[ch].y : 0.0f);
            A.y[o + ch] = den > 0.0f ? num / den : 0.0f;
        }
    }
}

int pyr_blocks(int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)device_info().sms * 8));
}

// P of a level-0 vector (levels 1 .. top of every image) into lv: level 1
// from src (with scal, S c and diag(A) too), levels 2 and 3, then each
// image's levels above; with wt, the down-sweep to level 1 as well (each
// image's levels top .. 4 in pyr_tail, levels 3 .. 1 in pyr_down_low).
cudaError_t pyr_sweep(const SolveArgs& A, const float* src, int nc, int scal, int up,
                      const float* wt, cudaStream_t s)
{
    const PyrDev& P = A.pyr;
    if (P.K < 2) return cudaSuccess;
    if (up) {
        pyr_gather0_kernel<<<pyr_blocks(P.off[2] - P.off[1]), 256, 0, s>>>(A, src, nc, scal);
        if (P.K > 2)
            pyr_gather_kernel<<<pyr_blocks(P.off[3] - P.off[2]), 256, 0, s>>>(A, 1, nc);
        if (P.K > 3)
            pyr_gather_kernel<<<pyr_blocks(P.off[4] - P.off[3]), 256, 0, s>>>(A, 2, nc);
    }
    if (P.K > 4 && (up || wt))
        pyr_tail_kernel<<<A.ninst, kPyrTailThreads, 0, s>>>(A, nc, up, wt);
    if (wt) pyr_down_low_kernel<<<pyr_blocks(P.off[2] - P.off[1]), 256, 0, s>>>(A, nc, wt);
    return cudaGetLastError();
}

// z = M_hier^-1 r and the partials of r^T z into out
cudaError_t pyr_precond(const SolveArgs& A, float2* out, cudaStream_t s)
{
    static int fam = prof_family("pyr_precond");
    static const int occ = [] {
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, pyr_precond0_kernel, kVTile, 0);
        return o > 0 ? o : 1;
    }();
    prof_begin(fam, s);
    cudaError_t e = pyr_sweep(A, A.r, A.pyr.W, 0, 1, A.pyr.coef, s);
    if (e == cudaSuccess) {
        const int nb = std::min(A.nvt, device_info().sms * occ);
        pyr_precond0_kernel<<<nb, kVTile, 0, s>>>(A, out);
        e = cudaGetLastError();
    }
    prof_end(fam, s);
    return e;
}

// the preconditioner's scale (after the splat) and the initial state y0:
// one up-sweep of (b, S c, diag A), coef, one down-sweep with cinit
cudaError_t pyr_setup(const SolveArgs& A, cudaStream_t s)
{
    static int fam = prof_family("pyr_setup");
    prof_begin(fam, s);
    const int nc = A.pyr.W + 2;
    cudaError_t e = pyr_sweep(A, A.r, nc, 1, 1, nullptr, s);
    if (e == cudaSuccess) {
        pyr_coef_kernel<<<pyr_blocks(A.pyr.off[A.pyr.K]), 256, 0, s>>>(A);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = pyr_sweep(A, nullptr, nc, 0, 0, A.pyr.cinit, s);
    if (e == cudaSuccess) {
        pyr_init0_kernel<<<pyr_blocks(A.pyr.off[1]), 256, 0, s>>>(A);
        e = cudaGetLastError();
    }
    prof_end(fam, s);
    return e;
}

// ------------------------------------------------- persistent PCG loop ---
// Grid barrier for a cooperative launch: one arrival counter that only
// grows.  Thread 0 of each block publishes the block's writes (fence), adds
// 1, and polls the counter with acquire loads until it reaches (epoch + 1) x
// gridDim.x, the arrivals of every block at this barrier; `epoch` counts
// the block's barriers (it starts at 0 with the counter).  The comparison is
// of the signed difference, so a counter preset to 2^31 (the failure-path
// test) is never reached.  Every wait is bounded: on time-out the block
// records kErrTimeout and false is returned.  Layout of `bar`: word 0.
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ bool grid_barrier(unsigned* bar, unsigned& epoch, uint32_t* err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = (epoch + 1u) * gridDim.x;
        __threadfence();
        atomicAdd(bar, 1u);
        unsigned spins = 0;
        while ((int)(ld_acquire_gpu(bar) - target) < 0) {
            if (++spins > kBarrierSpinLimit) {
                atomicOr(err, kErrTimeout);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        s_ok = ok;
    }
    ++epoch;
    __syncthreads();
    return s_ok != 0;
}

// Store the scalars that follow a reduced inner product of one (image,
// channel): kind 0, sum = r^T M^-1 r of iteration `it` -> delta_it, beta_it;
// kind 1, sum = d^T A d of iteration `it` -> alpha_it (as phase_scalars).
__device__ __forceinline__ void set_scalars(Scal* sc, int kind, int it, double sum)
{
    const double d0 = __ldcg(&sc->delta0);
    if (kind == 0) {
        double beta = 0.0;
        if (it > 0) {
            const double dprev = __ldcg(&sc->delta[(it & 1) ^ 1]);
            beta = dprev != 0.0 && !cg_stalled(sum, d0) ? sum / dprev : 0.0;
        } else {
            sc->delta0 = sum;
        }
        sc->delta[it & 1] = sum;
        sc->beta = (float)beta;
    } else {
        const double delta = __ldcg(&sc->delta[it & 1]);
        sc->alpha = (sum > 0.0 && !cg_stalled(delta, d0)) ? delta / sum : 0.0;
    }
}

// The scalars of every (image, channel) after a phase of the resident loop
// (kind and it as in set_scalars), by the block that completed the phase.
// Each sum is formed in the order of reduce_partials_all (thread t of the
// block takes slots t, t + kVTile, ...; warp trees; warps in order), so every
// launch style reaches the same scalar.  An image of at most 32 tiles is one
// warp tree (the other warps' sums are exact zeros), so such images are
// taken by the warps in turn; a larger image by the whole block.  `own` is
// the block's own image, used when the batch has one image.  Whole block.
__device__ void finalise_all(const SolveArgs& A, const InstDev& own, const float2* __restrict__ part,
                             int kind, int it, PhaseSmem& S)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < A.ninst; ++k) {
        const InstDev I = A.ninst == 1 ? own : A.inst[k];
        if (I.ntiles <= 32) continue;
        if (I.Cp == 1) reduce_partials_all<1, 8>(part, I, S.sd, S.red);
        else if (I.Cp == 2) reduce_partials_all<2, 4>(part, I, S.sd, S.red);
        else if (I.Cp == 4) reduce_partials_all<4, 2>(part, I, S.sd, S.red);
        else {
            reduce_instance_partials(part, I, S.sd);
            __syncthreads();
        }
        for (int ch = threadIdx.x; ch < I.C; ch += blockDim.x)
            set_scalars(&A.scal[I.pc + ch], kind, it, S.sd[ch]);
        __syncthreads();
    }
    int pair = 0;
    for (int k = 0; k < A.ninst; ++k) {
        const int ntiles = A.ninst == 1 ? own.ntiles : A.inst[k].ntiles;
        if (ntiles > 32) continue;
        const InstDev& I = A.ninst == 1 ? own : A.inst[k];
        for (int ch = 0; ch < I.C; ++ch, ++pair) {
            if (pair % nw != w) continue;
            const float2 v = lane < ntiles ? __ldcg(part + I.part_base + (int64_t)ch * ntiles + lane)
                                           : make_float2(0.0f, 0.0f);
            DF acc = {0.0f, 0.0f};
            acc = df_add(acc, DF{v.x, v.y});
            const DF t = df_warp_sum(acc);
            if (lane == 0) set_scalars(&A.scal[I.pc + ch], kind, it, df_to_double(t));
        }
    }
}

// The single-reduction form's scalars of iteration `it` from gamma_it and
// mu_it (cg_scalars' rules, with gamma and alpha of iteration it - 1 from
// sc), stored for the next pass: beta and alpha to be read, gamma_it and
// alpha_it by parity.
__device__ __forceinline__ void single_scalars(Scal* sc, int it, double gamma, double mu)
{
    const int slot = it & 1;
    double beta = 0.0, den = mu;
    bool stalled = gamma == 0.0;
    if (it > 0) {
        const double gold = __ldcg(&sc->gam[slot ^ 1]);
        const double aold = __ldcg(&sc->alp[slot ^ 1]);
        stalled = cg_stalled(gamma, __ldcg(&sc->delta0));
        beta = gold != 0.0 && !stalled ? gamma / gold : 0.0;
        if (beta != 0.0 && aold != 0.0) den = mu - beta * gamma / aold;
    } else {
        sc->delta0 = gamma;
    }
    const double alpha = (!stalled && den > 0.0) ? gamma / den : 0.0;
    sc->gam[slot] = gamma;
    sc->alp[slot] = alpha;
    sc->beta = (float)beta;
    sc->alpha = alpha;
}

// finalise_all for the single-reduction form: the partials of gamma_it
// (part_rs[it & 1]) and of mu_it (part_mu[it & 1]) of every (image, channel),
// in the order of reduce_partials_all, then single_scalars.  Whole block.
__device__ void finalise_single(const SolveArgs& A, const InstDev& own, int it, PhaseSmem& S)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float2* __restrict__ pg = A.part_rs[it & 1];
    const float2* __restrict__ pm = A.part_mu[it & 1];
    for (int k = 0; k < A.ninst; ++k) {
        const InstDev I = A.ninst == 1 ? own : A.inst[k];
        if (I.ntiles <= 32) continue;
        if (I.Cp == 1) {
            reduce_partials_all<1, 8>(pg, I, S.sd, S.red);
            reduce_partials_all<1, 8>(pm, I, S.sd2, S.red);
        } else if (I.Cp == 2) {
            reduce_partials_all<2, 4>(pg, I, S.sd, S.red);
            reduce_partials_all<2, 4>(pm, I, S.sd2, S.red);
        } else {
            reduce_partials_all<4, 2>(pg, I, S.sd, S.red);
            reduce_partials_all<4, 2>(pm, I, S.sd2, S.red);
        }
        for (int ch = threadIdx.x; ch < I.C; ch += blockDim.x)
            single_scalars(&A.scal[I.pc + ch], it, S.sd[ch], S.sd2[ch]);
        __syncthreads();
    }
    int pair = 0;
    for (int k = 0; k < A.ninst; ++k) {
        const int ntiles = A.ninst == 1 ? own.ntiles : A.inst[k].ntiles;
        if (ntiles > 32) continue;
        const InstDev& I = A.ninst == 1 ? own : A.inst[k];
        for (int ch = 0; ch < I.C; ++ch, ++pair) {
            if (pair % nw != w) continue;
            const int64_t o = I.part_base + (int64_t)ch * ntiles + lane;
            const float2 g = lane < ntiles ? __ldcg(pg + o) : make_float2(0.0f, 0.0f);
            const float2 m = lane < ntiles ? __ldcg(pm + o) : make_float2(0.0f, 0.0f);
            DF ag = {0.0f, 0.0f}, am = {0.0f, 0.0f};
            ag = df_add(ag, DF{g.x, g.y});
            am = df_add(am, DF{m.x, m.y});
            const DF tg = df_warp_sum(ag), tm = df_warp_sum(am);
            if (lane == 0)
                single_scalars(&A.scal[I.pc + ch], it, df_to_double(tg), df_to_double(tm));
        }
    }
}

__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier of the resident loop that also finalises the phase: every
// block has stored its tile partials; the block whose arrival completes the
// count reduces all (image, channel) partials, stores the next phase's
// scalars and then releases the others through the release word (bar[32],
// its own 128-byte line), which holds the number of barriers passed.  The
// arrival count only grows (as in grid_barrier); a counter preset to 2^31
// (the failure-path test) completes no barrier, and every wait is bounded:
// on time-out the block records kErrTimeout and false is returned.  kind 0
// and 1 as in finish_image; kind 2: the single-reduction form's gamma and
// mu of iteration `it` (part is not used).
__device__ bool reduce_barrier(const SolveArgs& A, const InstDev& own, unsigned* bar,
                               unsigned& epoch, const float2* __restrict__ part, int kind, int it,
                               PhaseSmem& S)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = (epoch + 1u) * gridDim.x;
        __threadfence();
        const unsigned old = atomicAdd(bar, 1u);
        S.last = old == target - 1u;
        if (S.last) __threadfence();
        s_ok = 1;
    }
    __syncthreads();
    if (S.last) {
        if (kind == 2) finalise_single(A, own, it, S);    // single-reduction form
        else finalise_all(A, own, part, kind, it, S);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_gpu(bar + 32, epoch + 1u);
        }
    } else if (threadIdx.x == 0) {
        unsigned spins = 0;
        while ((int)(ld_acquire_gpu(bar + 32) - (epoch + 1u)) < 0) {
            if (++spins > kBarrierSpinLimit) {
                atomicOr(A.err, kErrTimeout);
                s_ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    ++epoch;
    __syncthreads();
    return s_ok != 0;
}

// All `iters` PCG iterations in one cooperative launch: phase 1, barrier,
// phase 2, barrier.  Every block keeps the same chunk of tiles throughout.
template <int WMAX, bool COMP>
__global__ void __launch_bounds__(kVTile, phase_min_blocks<WMAX>())
pcg_loop_kernel(SolveArgs A, int iters, unsigned* bar)
{
    __shared__ PhaseSmem S;
    __shared__ WideSmem Wd;
    int t0, t1;
    block_chunk(A.nvt, t0, t1);
    unsigned epoch = 0;
    for (int it = 0; it < iters; ++it) {
        const float* dold = A.d[(it + 1) & 1];
        float* dnew = A.d[it & 1];
        if (!COMP && it > 0 && A.zq)
            phase_run<1, COMP, true, WMAX, false, !COMP>(A, dold, dnew, it, t0, t1, S, Wd);
        else
            phase_run<1, COMP, true, WMAX>(A, dold, dnew, it, t0, t1, S, Wd);
        if (!grid_barrier(bar, epoch, A.err)) return;
        phase_run<2, COMP, true, WMAX>(A, dnew, nullptr, it, t0, t1, S, Wd);
        if (!grid_barrier(bar, epoch, A.err)) return;
    }
}

// ------------------------------------------ resident persistent PCG loop ---
// The same iterations when every tile has its own co-resident block and each
// image's channels fit one pass (Cp <= 4): each block keeps its tile's
// neighbour ids and neighbours' {n, M^-1} in shared memory for the whole
// loop, and each thread keeps its vertex's r, y, d (and q) in registers,
// writing d and r for the neighbours and y once at the end.  Neighbour
// gathers use a safe index (the vertex itself when a neighbour is absent) so
// they issue together with the reduction of the previous phase's partials.

template <int W, bool COMP, int NG = (COMP && W == 4 ? 5 : 10)>
__device__ void resident_loop(const SolveArgs& A, const InstDev& I, const VTile& vt, int iters,
                              unsigned* bar, int32_t (*s_nb)[kVTile], float2 (*s_nmu)[kVTile],
                              PhaseSmem& S)
{
    const int tx = threadIdx.x;
    const int64_t v = vt.v0 + tx;
    const bool valid = v < vt.v1;
    // topology, once
    float av = 0.0f;
    float2 nmv = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        const int32_t u = valid ? A.nbr[(int64_t)k * A.nbr_stride + v] : -1;
        s_nb[k][tx] = u;
        s_nmu[k][tx] = u >= 0 ? A.nm[u] : make_float2(0.0f, 0.0f);
    }
    if (valid) {
        av = A.a[v];
        nmv = A.nm[v];
    }
    const float lam_n = I.lam * nmv.x;
    const int64_t vs = valid ? v : vt.v0;   // safe gather index for absent neighbours
    const int64_t base = pass_base(I, 0);
    // own state in registers (y's low part too when y is a double-float pair)
    const bool ydf = COMP && A.ylo != nullptr;
    const float alv = COMP && A.alo && valid ? A.alo[v] : 0.0f;
    float r[W], rlo[W], y[W], yl[W], d[W], q[W];
    ldw<W, false>(A.r + base + vs * I.Cp, r);
    ldw<W, false>(A.y + base + vs * I.Cp, y);
    if (COMP) ldw<W, false>(A.rlo + base + vs * I.Cp, rlo);
    if (ydf) ldw<W, false>(A.ylo + base + vs * I.Cp, yl);
#pragma unroll
    for (int k = 0; k < W; ++k) {
        d[k] = 0.0f;
        q[k] = 0.0f;
        if (!COMP) rlo[k] = 0.0f;
    }
    unsigned epoch = 0;
    for (int it = 0; it < iters; ++it) {
        const int slot = it & 1;
        const float* dold = A.d[(it + 1) & 1];
        float* dnew = A.d[it & 1];
        // ---- phase 1.  FP32: the z form, q = A z + beta q_old (A d, since
        // d = z + beta d_old is linear), so a neighbour contributes only its
        // z = M^-1 r -- stored by the previous phase 2, or, in iteration 0,
        // formed from the initial residual.  Compensated: a neighbour's d is
        // formed from its gathered r and d_old and q = A d, the arithmetic of
        // the per-phase kernels (whose results this loop reproduces
        // bitwise).  Gathers first (they do not depend on beta), then the
        // reduction of the previous phase's partials overlaps their latency;
        // groups of NG neighbours.
        {
            float zv[W], dv[W], beta[W];
#pragma unroll
            for (int k = 0; k < W; ++k) zv[k] = nmv.y * r[k];
            DF s[W];
#pragma unroll
            for (int k = 0; k < W; ++k) s[k] = {0.0f, 0.0f};
#pragma unroll
            for (int g0 = 0; g0 < 10; g0 += NG) {
                float zu[NG][W], du[NG][W];
#pragma unroll
                for (int j = 0; j < NG; ++j) {
                    const int32_t u0 = s_nb[g0 + j][tx];
                    const int64_t u = u0 >= 0 ? u0 : vs;
                    ldw<W, true>((!COMP && it > 0 ? A.zq : A.r) + base + u * I.Cp, zu[j]);
                    if (COMP && it > 0) {
                        ldw<W, true>(dold + base + u * I.Cp, du[j]);
                    } else {
#pragma unroll
                        for (int k = 0; k < W; ++k) du[j][k] = 0.0f;
                    }
                }
                if (g0 == 0) {
                    load_scalars<1>(A, I, S);
#pragma unroll
                    for (int k = 0; k < W; ++k) {
                        beta[k] = S.sf[k];
                        dv[k] = fmaf(beta[k], d[k], zv[k]);
                    }
                }
#pragma unroll
                for (int j = 0; j < NG; ++j) {
                    const float2 nm = s_nmu[g0 + j][tx];
                    float dz[W];
#pragma unroll
                    for (int k = 0; k < W; ++k)
                        dz[k] = COMP ? fmaf(beta[k], du[j][k], nm.y * zu[j][k])
                                     : (it == 0 ? nm.y * zu[j][k] : zu[j][k]);
                    lap_acc<W, false>(s, nm.x, COMP ? dv : zv, dz);
                }
            }
            DF acc[W];
#pragma unroll
            for (int k = 0; k < W; ++k) {
                if (COMP) {
                    q[k] = lap_finish<false>(av, lam_n, dv[k], s[k]).hi;
                } else {
                    const DF az = lap_finish<false>(av, lam_n, zv[k], s[k]);
                    q[k] = fmaf(beta[k], q[k], az.hi);      // q = 0 before iteration 0
                }
                d[k] = dv[k];
                const bool on = valid && k < I.C;
                acc[k] = !on ? DF{0.0f, 0.0f} : df_mul_exact(dv[k], q[k]);
            }
            if (COMP && valid) stw<W>(dnew + base + v * I.Cp, dv);
            store_partials<W>(acc, I.C, I.ntiles, I.part_base, 0, vt.t_in_inst, A.part_dq, S.red);
        }
        if (!reduce_barrier(A, I, bar, epoch, A.part_dq, 1, it, S)) return;
        // ---- phase 2
        {
            DF s[W];
#pragma unroll
            for (int k = 0; k < W; ++k) s[k] = {0.0f, 0.0f};
#pragma unroll
            for (int g0 = 0; g0 < 10; g0 += NG) {
                float dn[NG][W];
                if (COMP) {
#pragma unroll
                    for (int j = 0; j < NG; ++j) {
                        const int32_t u0 = s_nb[g0 + j][tx];
                        const int64_t u = u0 >= 0 ? u0 : vs;
                        ldw<W, true>(dnew + base + u * I.Cp, dn[j]);
                    }
                }
                if (g0 == 0) load_scalars<2>(A, I, S);
                if (COMP) {
#pragma unroll
                    for (int j = 0; j < NG; ++j) lap_acc<W, true>(s, s_nmu[g0 + j][tx].x, d, dn[j]);
                }
                if (!COMP) break;   // no gathers in the FP32 update
            }
            DF acc[W];
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const double alpha = S.sa[k];
                if (ydf) {
                    const DF yy = df_add(DF{y[k], yl[k]}, df_mul_f(df_from_double(alpha), d[k]));
                    y[k] = yy.hi;
                    yl[k] = yy.lo;
                } else {
                    y[k] = fmaf((float)alpha, d[k], y[k]);
                }
                if (COMP) {
                    const DF qq = lap_finish<true>(av, lam_n, d[k], s[k], alv);
                    const DF rr = df_add(DF{r[k], rlo[k]},
                                         df_neg(df_mul(df_from_double(alpha), qq)));
                    r[k] = rr.hi;
                    rlo[k] = rr.lo;
                } else {
                    r[k] = fmaf(-(float)alpha, q[k], r[k]);
                }
                const bool on = valid && k < I.C;
                acc[k] = on ? df_mul_exact(r[k], nmv.y * r[k]) : DF{0.0f, 0.0f};
            }
            if (valid && COMP) {
                stw<W>(A.r + base + v * I.Cp, r);
            } else if (valid) {          // z = M^-1 r for the neighbours' next phase 1
                float zv[W];
#pragma unroll
                for (int k = 0; k < W; ++k) zv[k] = nmv.y * r[k];
                stw<W>(A.zq + base + v * I.Cp, zv);
            }
            store_partials<W>(acc, I.C, I.ntiles, I.part_base, 0, vt.t_in_inst,
                              A.part_rs[slot ^ 1], S.red);
        }
        if (!reduce_barrier(A, I, bar, epoch, A.part_rs[slot ^ 1], 0, it + 1, S)) return;
    }
    if (valid) {
        stw<W>(A.y + base + v * I.Cp, y);
        if (!COMP) stw<W>(A.r + base + v * I.Cp, r);
        if (COMP) stw<W>(A.rlo + base + v * I.Cp, rlo);
        if (ydf) stw<W>(A.ylo + base + v * I.Cp, yl);
    }
}

// WMAX: the widest pass of the batch (the largest Cp), so that a batch of
// single-channel images gets the register budget of the W = 1 body alone.
template <int WMAX, bool COMP>
__global__ void __launch_bounds__(kVTile, 3)
pcg_resident_kernel(SolveArgs A, int iters, unsigned* bar)
{
    __shared__ int32_t s_nb[10][kVTile];
    __shared__ float2 s_nmu[10][kVTile];
    __shared__ PhaseSmem S;
    const VTile vt = A.vt[blockIdx.x];
    const InstDev I = A.inst[vt.inst];
    if (WMAX == 1 || I.Cp == 1) resident_loop<1, COMP>(A, I, vt, iters, bar, s_nb, s_nmu, S);
    else if (WMAX == 2 || I.Cp == 2) resident_loop<2, COMP>(A, I, vt, iters, bar, s_nb, s_nmu, S);
    else resident_loop<4, COMP>(A, I, vt, iters, bar, s_nb, s_nmu, S);
}

// ------------------------------- resident single-reduction PCG loop ---
// The single-reduction form (see cg_tile) with all iterations in one
// cooperative launch, one tile per block: one grid barrier per iteration
// instead of two, the last block to reach it forming beta and alpha of the
// next iteration from the partials of gamma and mu.  Each thread keeps its
// vertex's r, w and s in registers (p and y stay in memory: read and
// written once per iteration), gathers the neighbours' r_i, w_i and
// s_(i-1) from the previous iteration's buffers (by parity, as cg_tile), and
// writes its own for the next.  The set-up pass forms w_0 = A M^-1 r_0 and
// the partials of mu_0 (gamma_0's come from the initial residual).  FP32
// vectors, Cp <= 4; the same arithmetic per vertex as cg_tile.
template <int W, int NG = (W == 4 ? 2 : 5)>
__device__ void resident_single_loop(const SolveArgs& A, const InstDev& I, const VTile& vt,
                                     int iters, unsigned* bar, int32_t (*s_nb)[kVTile],
                                     float2 (*s_nmu)[kVTile], PhaseSmem& S)
{
    const int tx = threadIdx.x;
    const int v = (int)vt.v0 + tx;
    const bool valid = v < (int)vt.v1;
    const int vs = valid ? v : (int)vt.v0;
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        const int32_t u = valid ? A.nbr[(int64_t)k * A.nbr_stride + v] : -1;
        s_nb[k][tx] = u;
        s_nmu[k][tx] = u >= 0 ? A.nm[u] : make_float2(0.0f, 0.0f);
    }
    const float2 nmv = A.nm[vs];
    const float av = A.a[vs];
    const float lam_n = I.lam * nmv.x;
    const int64_t off = I.vec_base - I.voff * W;
    DF rg[W], rm[W];
    float r[W], w[W], so[W];
    unsigned epoch = 0;
    // set-up: w_0 = A M^-1 r_0 (into d[0]) and the partials of mu_0
    {
        const float* __restrict__ rb = A.r + off;
        float u0[W], lap[W];
        ldw<W, false>(rb + vs * W, r);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            u0[k] = nmv.y * r[k];
            lap[k] = 0.0f;
        }
        __syncthreads();                    // s_nb, s_nmu
#pragma unroll
        for (int j = 0; j < 10; ++j) {
            const int32_t u0i = s_nb[j][tx];
            const int u = u0i >= 0 ? u0i : vs;
            const float2 nm = s_nmu[j][tx];
            float ru[W];
            ldw<W, false>(rb + u * W, ru);
#pragma unroll
            for (int k = 0; k < W; ++k) lap[k] = fmaf(nm.x, u0[k] - nm.y * ru[k], lap[k]);
        }
#pragma unroll
        for (int k = 0; k < W; ++k) {
            w[k] = fmaf(av, u0[k], lam_n * lap[k]);
            so[k] = 0.0f;
            rm[k] = valid && k < I.C ? df_mul_exact(w[k], u0[k]) : DF{0.0f, 0.0f};
        }
        if (valid) stw<W>(A.d[0] + off + v * W, w);
        store_partials<W>(rm, I.C, I.ntiles, I.part_base, 0, vt.t_in_inst, A.part_mu[0], S.red);
    }
    if (!reduce_barrier(A, I, bar, epoch, nullptr, 2, 0, S)) return;
    for (int it = 0; it < iters; ++it) {
        const int cur = it & 1, nxt = cur ^ 1;
        const bool first = it == 0, last = it == iters - 1;
        __syncthreads();
        for (int ch = tx; ch < I.Cp; ch += blockDim.x) {
            const bool on = ch < I.C;
            S.sf[ch] = on ? __ldcg(&A.scal[I.pc + ch].beta) : 0.0f;
            S.sa[ch] = on ? __ldcg(&A.scal[I.pc + ch].alpha) : 0.0;
        }
        __syncthreads();
        float beta[W], alpha[W], pv[W], yv[W], r1[W], u1[W];
        if (!first) ldw<W, false>(A.q + off + vs * W, pv);
        ldw<W, false>(A.y + off + vs * W, yv);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            beta[k] = S.sf[k];
            alpha[k] = (float)S.sa[k];
            const float si = first ? w[k] : fmaf(beta[k], so[k], w[k]);
            const float ui = nmv.y * r[k];
            pv[k] = first ? ui : fmaf(beta[k], pv[k], ui);
            yv[k] = fmaf(alpha[k], pv[k], yv[k]);
            r1[k] = fmaf(-alpha[k], si, r[k]);
            u1[k] = nmv.y * r1[k];
            so[k] = si;
        }
        if (last) {
            if (valid) {
                stw<W>(A.y + off + v * W, yv);
                stw<W>(A.q + off + v * W, pv);
            }
            break;
        }
        const float* __restrict__ rb = (cur ? A.rlo : A.r) + off;   // r_i
        const float* __restrict__ wb = A.d[cur] + off;             // w_i
        const float* __restrict__ sb = A.aux[nxt] + off;           // s_(i-1)
        float lap[W];
#pragma unroll
        for (int k = 0; k < W; ++k) lap[k] = 0.0f;
#pragma unroll
        for (int g0 = 0; g0 < 10; g0 += NG) {
            float ru[NG][W], wu[NG][W], su[NG][W];
#pragma unroll
            for (int j = 0; j < NG; ++j) {
                const int32_t u0i = s_nb[g0 + j][tx];
                const int u = u0i >= 0 ? u0i : vs;
                ldw<W, false>(rb + u * W, ru[j]);
                ldw<W, false>(wb + u * W, wu[j]);
                if (!first) ldw<W, false>(sb + u * W, su[j]);
            }
#pragma unroll
            for (int j = 0; j < NG; ++j) {
                const float2 nm = s_nmu[g0 + j][tx];
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    const float s_u = first ? wu[j][k] : fmaf(beta[k], su[j][k], wu[j][k]);
                    const float u_u = nm.y * fmaf(-alpha[k], s_u, ru[j][k]);
                    lap[k] = fmaf(nm.x, u1[k] - u_u, lap[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < W; ++k) {
            w[k] = fmaf(av, u1[k], lam_n * lap[k]);
            r[k] = r1[k];
            const bool on = valid && k < I.C;
            rg[k] = on ? df_mul_exact(r1[k], u1[k]) : DF{0.0f, 0.0f};
            rm[k] = on ? df_mul_exact(w[k], u1[k]) : DF{0.0f, 0.0f};
        }
        if (valid) {                // every store after the last gather
            stw<W>(A.y + off + v * W, yv);
            stw<W>(A.q + off + v * W, pv);
            stw<W>(A.aux[cur] + off + v * W, so);
            stw<W>((nxt ? A.rlo : A.r) + off + v * W, r1);
            stw<W>(A.d[nxt] + off + v * W, w);
        }
        store_partials<W>(rg, I.C, I.ntiles, I.part_base, 0, vt.t_in_inst, A.part_rs[nxt], S.red);
        store_partials<W>(rm, I.C, I.ntiles, I.part_base, 0, vt.t_in_inst, A.part_mu[nxt], S.red);
        if (!reduce_barrier(A, I, bar, epoch, nullptr, 2, it + 1, S)) return;
    }
}

template <int WMAX>
__global__ void __launch_bounds__(kVTile, 3)
pcg_resident_single_kernel(SolveArgs A, int iters, unsigned* bar)
{
    __shared__ int32_t s_nb[10][kVTile];
    __shared__ float2 s_nmu[10][kVTile];
    __shared__ PhaseSmem S;
    const VTile vt = A.vt[blockIdx.x];
    const InstDev I = A.inst[vt.inst];
    if (WMAX == 1 || I.Cp == 1) resident_single_loop<1>(A, I, vt, iters, bar, s_nb, s_nmu, S);
    else if (WMAX == 2 || I.Cp == 2) resident_single_loop<2>(A, I, vt, iters, bar, s_nb, s_nmu, S);
    else resident_single_loop<4>(A, I, vt, iters, bar, s_nb, s_nmu, S);
}

// index of the widest pass: 0 (W = 1), 1 (W = 2), 2 (W = 4)
int width_index(int cmax) { return cmax <= 1 ? 0 : cmax <= 2 ? 1 : 2; }

// ---------------------------------------------------------------- slice ---
// x = S^T y for every pixel of image blockIdx.y.
__global__ void __launch_bounds__(256)
slice_kernel(SolveArgs A)
{
    const InstDev I = A.inst[blockIdx.y];
    if (I.x == nullptr) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < I.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = A.vid[I.pix_base + i];
        for (int ch = 0; ch < I.C; ++ch)
            I.x[(int64_t)ch * I.N + i] =
                A.y[vec_index(I, ch, v)] + (A.ylo ? A.ylo[vec_index(I, ch, v)] : 0.0f);
    }
}

// ------------------------------------------------------------- backward ---
// With z = A^-1 S dL/dx in y: dL/dt = c o S^T z,
// dL/dc = sum_ch (S^T z) o (t - S^T y-hat).
__global__ void __launch_bounds__(256)
backward_slice_kernel(SolveArgs A)
{
    const InstDev I = A.inst[blockIdx.y];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < I.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = A.vid[I.pix_base + i];
        const float ci = I.c[i];
        float dc = 0.0f;
        for (int ch = 0; ch < I.C; ++ch) {
            const float z = A.y[vec_index(I, ch, v)] + (A.ylo ? A.ylo[vec_index(I, ch, v)] : 0.0f);
            if (I.dt) I.dt[(int64_t)ch * I.N + i] = ci * z;
            const float yh = I.yhat[(int64_t)ch * I.V + (v - I.voff)];
            dc = fmaf(z, I.t[(int64_t)ch * I.N + i] - yh, dc);
        }
        if (I.dc) I.dc[i] = dc;
    }
}

// copy y to the caller's buffers (their layout: C x V per image)
__global__ void __launch_bounds__(256)
export_y_kernel(SolveArgs A)
{
    const InstDev I = A.inst[blockIdx.y];
    float* dst = I.yout;
    if (dst == nullptr) return;
    const int64_t n = (int64_t)I.C * I.V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ch = i / I.V, j = i - ch * I.V;
        dst[i] = A.y[I.vec_base + j * I.Cp + ch] + (A.ylo ? A.ylo[I.vec_base + j * I.Cp + ch] : 0.0f);
    }
}

int occupancy(const void* fn)
{
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, kVTile, 0);
    return o > 0 ? o : 1;
}

int persistent_blocks(int occ, int nvt)
{
    const int cap = device_info().sms * occ;
    return nvt < cap ? nvt : cap;
}

template <bool COMP>
cudaError_t launch_loop(const SolveArgs& A, const SolvePlan& P, cudaStream_t s)
{
    static int f_apply = prof_family("pcg_apply");
    static int f_update = prof_family("pcg_update");
    static int f_loop = prof_family("pcg_loop");
    static int f_res_loop = prof_family("pcg_resident");
    static const void* const fn_p[3] = {(const void*)pcg_apply_kernel<1, COMP>,
                                        (const void*)pcg_apply_kernel<2, COMP>,
                                        (const void*)pcg_apply_kernel<4, COMP>};
    static const void* const fn_u[3] = {(const void*)pcg_update_kernel<1, COMP>,
                                        (const void*)pcg_update_kernel<2, COMP>,
                                        (const void*)pcg_update_kernel<4, COMP>};
    static const void* const fn_l[3] = {(const void*)pcg_loop_kernel<1, COMP>,
                                        (const void*)pcg_loop_kernel<2, COMP>,
                                        (const void*)pcg_loop_kernel<4, COMP>};
    static const int occ_p[3] = {occupancy(fn_p[0]), occupancy(fn_p[1]), occupancy(fn_p[2])};
    static const int occ_u[3] = {occupancy(fn_u[0]), occupancy(fn_u[1]), occupancy(fn_u[2])};
    static const int occ_l[3] = {occupancy(fn_l[0]), occupancy(fn_l[1]), occupancy(fn_l[2])};
    const int wi = width_index(P.cmax);
    static const int occ_res[3] = {occupancy((const void*)pcg_resident_kernel<1, COMP>),
                                   occupancy((const void*)pcg_resident_kernel<2, COMP>),
                                   occupancy((const void*)pcg_resident_kernel<4, COMP>)};
    static const int occ_res_single[3] = {occupancy((const void*)pcg_resident_single_kernel<1>),
                                          occupancy((const void*)pcg_resident_single_kernel<2>),
                                          occupancy((const void*)pcg_resident_single_kernel<4>)};
    if (P.persistent && P.pcg_iters > 0 && P.single && !COMP && P.cmax <= 4 &&
        A.nvt <= device_info().sms * occ_res_single[wi]) {
        // the single-reduction form, resident: one barrier per iteration
        static int f_res_single = prof_family("pcg_resident_single");
        cudaError_t e = cudaMemsetAsync(P.barrier, 0, kBarrierWords * sizeof(unsigned), s);
        if (e == cudaSuccess && P.inject_timeout)   // counter = 2^31 (little-endian)
            e = cudaMemsetAsync(reinterpret_cast<unsigned char*>(P.barrier) + 3, 0x80, 1, s);
        if (e != cudaSuccess) return e;
        SolveArgs a = A;
        int iters = P.pcg_iters;
        unsigned* bar = P.barrier;
        void* args[] = {&a, &iters, &bar};
        const void* fn = wi == 0   ? (const void*)pcg_resident_single_kernel<1>
                         : wi == 1 ? (const void*)pcg_resident_single_kernel<2>
                                   : (const void*)pcg_resident_single_kernel<4>;
        prof_begin(f_res_single, s);
        e = cudaLaunchCooperativeKernel(fn, dim3(A.nvt), dim3(kVTile), args, 0, s);
        prof_end(f_res_single, s);
        if (e == cudaSuccess) return cudaGetLastError();
        cudaGetLastError();   // clear, and fall back to per-phase launches
    }
    if (P.persistent && P.pcg_iters > 0 && !P.single) {
        const bool resident = P.cmax <= 4 && A.nvt <= device_info().sms * occ_res[wi] &&
                              (COMP || A.zq);
        if (resident || P.force_persistent) {
            // barrier words zero (or, for the failure-path test, a top counter
            // that the last arrival can never match)
            cudaError_t e = cudaMemsetAsync(P.barrier, 0, kBarrierWords * sizeof(unsigned), s);
            if (e == cudaSuccess && P.inject_timeout)   // counter = 2^31 (little-endian)
                e = cudaMemsetAsync(reinterpret_cast<unsigned char*>(P.barrier) + 3, 0x80, 1, s);
            if (e != cudaSuccess) return e;
            SolveArgs a = A;
            int iters = P.pcg_iters;
            unsigned* bar = P.barrier;
            void* args[] = {&a, &iters, &bar};
            if (resident) {
                prof_begin(f_res_loop, s);
                const void* fn = wi == 0   ? (const void*)pcg_resident_kernel<1, COMP>
                                 : wi == 1 ? (const void*)pcg_resident_kernel<2, COMP>
                                           : (const void*)pcg_resident_kernel<4, COMP>;
                e = cudaLaunchCooperativeKernel(fn, dim3(A.nvt), dim3(kVTile), args, 0, s);
                prof_end(f_res_loop, s);
            } else {
                prof_begin(f_loop, s);
                e = cudaLaunchCooperativeKernel(fn_l[wi],
                                                dim3(persistent_blocks(occ_l[wi], A.nvt)),
                                                dim3(kVTile), args, 0, s);
                prof_end(f_loop, s);
            }
            if (e == cudaSuccess) return cudaGetLastError();
            cudaGetLastError();   // clear, and fall back to per-phase launches
        }
    }
    if (P.single) {
        static int f_single = prof_family("pcg_single");
        static const void* const fn_s[3] = {(const void*)pcg_single_kernel<1>,
                                            (const void*)pcg_single_kernel<2>,
                                            (const void*)pcg_single_kernel<4>};
        static const int occ_s[3] = {occupancy(fn_s[0]), occupancy(fn_s[1]), occupancy(fn_s[2])};
        const int nb = persistent_blocks(occ_s[wi] * (P.block_mult > 1 ? P.block_mult : 1), A.nvt);
        for (int it = -1; it < P.pcg_iters; ++it) {
            const int last = it == P.pcg_iters - 1 ? 1 : 0;
            prof_begin(f_single, s);
            if (wi == 0) pcg_single_kernel<1><<<nb, kVTile, 0, s>>>(A, it, last);
            else if (wi == 1) pcg_single_kernel<2><<<nb, kVTile, 0, s>>>(A, it, last);
            else pcg_single_kernel<4><<<nb, kVTile, 0, s>>>(A, it, last);
            prof_end(f_single, s);
        }
        return cudaGetLastError();
    }
    const int mult = P.block_mult > 1 ? P.block_mult : 1;
    const int nb_p = persistent_blocks(occ_p[wi] * mult, A.nvt);
    const int nb_u = persistent_blocks(occ_u[wi] * mult, A.nvt);
    for (int it = 0; it < P.pcg_iters; ++it) {
        const float* dold = A.d[(it + 1) & 1];
        float* dnew = A.d[it & 1];
        prof_begin(f_apply, s);
        if (P.hier) {
            if (wi == 0) pcg_apply_kernel<1, COMP, true><<<nb_p, kVTile, 0, s>>>(A, dold, dnew, it);
            else if (wi == 1) pcg_apply_kernel<2, COMP, true><<<nb_p, kVTile, 0, s>>>(A, dold, dnew, it);
            else pcg_apply_kernel<4, COMP, true><<<nb_p, kVTile, 0, s>>>(A, dold, dnew, it);
        } else if (!COMP && it > 0 && A.zq) {   // the z form
            constexpr bool Z = !COMP;
            if (wi == 0) pcg_apply_kernel<1, COMP, false, Z><<<nb_p, kVTile, 0, s>>>(A, dold, dnew, it);
            else if (wi == 1) pcg_apply_kernel<2, COMP, false, Z><<<nb_p, kVTile, 0, s>>>(A, dold, dnew, it);
            else pcg_apply_kernel<4, COMP, false, Z><<<nb_p, kVTile, 0, s>>>(A, dold, dnew, it);
        } else {
            if (wi == 0) pcg_apply_kernel<1, COMP><<<nb_p, kVTile, 0, s>>>(A, dold, dnew, it);
            else if (wi == 1) pcg_apply_kernel<2, COMP><<<nb_p, kVTile, 0, s>>>(A, dold, dnew, it);
            else pcg_apply_kernel<4, COMP><<<nb_p, kVTile, 0, s>>>(A, dold, dnew, it);
        }
        prof_end(f_apply, s);
        prof_begin(f_update, s);
        if (wi == 0) pcg_update_kernel<1, COMP><<<nb_u, kVTile, 0, s>>>(A, dnew, it);
        else if (wi == 1) pcg_update_kernel<2, COMP><<<nb_u, kVTile, 0, s>>>(A, dnew, it);
        else pcg_update_kernel<4, COMP><<<nb_u, kVTile, 0, s>>>(A, dnew, it);
        prof_end(f_update, s);
        if (P.hier) {                       // z = M_hier^-1 r and the next delta's partials
            cudaError_t e = pyr_precond(A, A.part_rs[(it + 1) & 1], s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

template <int CB>
cudaError_t launch_splat(const SolveArgs& A, const SolvePlan& P, int mode, cudaStream_t s)
{
    static const int occ_s = occupancy((const void*)splat_kernel<CB>);
    unsigned* work = P.barrier + kWorkCounterWord;
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    splat_kernel<CB><<<persistent_blocks(occ_s, A.nvt), kVTile, 0, s>>>(A, mode, P.sigma_gm,
                                                                     P.comp, work);
    return cudaGetLastError();
}

}  // namespace

bool resident_fits(const SolveArgs& A, const SolvePlan& P)
{
    static const int occ_single[3] = {occupancy((const void*)pcg_resident_single_kernel<1>),
                                      occupancy((const void*)pcg_resident_single_kernel<2>),
                                      occupancy((const void*)pcg_resident_single_kernel<4>)};
    if (P.single)
        return !P.comp && P.cmax <= 4 &&
               A.nvt <= device_info().sms * occ_single[width_index(P.cmax)];
    static const int occ[2][3] = {{occupancy((const void*)pcg_resident_kernel<1, false>),
                                   occupancy((const void*)pcg_resident_kernel<2, false>),
                                   occupancy((const void*)pcg_resident_kernel<4, false>)},
                                  {occupancy((const void*)pcg_resident_kernel<1, true>),
                                   occupancy((const void*)pcg_resident_kernel<2, true>),
                                   occupancy((const void*)pcg_resident_kernel<4, true>)}};
    if (P.cmax > 4 || (!P.comp && !A.zq)) return false;   // FP32: the loop keeps z in zq
    return A.nvt <= device_info().sms * occ[P.comp ? 1 : 0][width_index(P.cmax)];
}

bool resident_preferred(const SolveArgs& A, const SolvePlan& P)
{
    return resident_fits(A, P) && A.nvt <= device_info().sms;
}

cudaError_t launch_segment(const SolveArgs& A, const SolvePlan& P, int seg, int mode,
                           cudaStream_t s)
{
    static int f_splat = prof_family("splat");
    static int f_res = prof_family("residual");
    static int f_slice = prof_family("slice");
    static int f_bwd = prof_family("backward_slice");
    static int f_export = prof_family("export_y");
    static const int occ_rf = occupancy((const void*)residual_kernel<false>);
    static const int occ_rt = occupancy((const void*)residual_kernel<true>);
    cudaError_t e = cudaSuccess;
    if (seg == kSegSetup) {
        // CG scalars and the images' completion counters start at zero
        if ((e = cudaMemsetAsync(A.scal, 0, sizeof(Scal) * (size_t)A.nscal, s)) != cudaSuccess)
            return e;
        prof_begin(f_splat, s);
        switch (P.chan_block) {
            case 1: e = launch_splat<1>(A, P, mode, s); break;
            case 2: e = launch_splat<2>(A, P, mode, s); break;
            case 3: e = launch_splat<3>(A, P, mode, s); break;
            default: e = launch_splat<4>(A, P, mode, s); break;
        }
        prof_end(f_splat, s);
        if (e != cudaSuccess) return e;
        if (P.hier && (e = pyr_setup(A, s)) != cudaSuccess) return e;   // coef, y0
        prof_begin(f_res, s);
        if (P.comp)
            residual_kernel<true><<<persistent_blocks(occ_rt, A.nvt), kVTile, 0, s>>>(A);
        else
            residual_kernel<false><<<persistent_blocks(occ_rf, A.nvt), kVTile, 0, s>>>(A);
        prof_end(f_res, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (P.hier) return pyr_precond(A, A.part_rs[0], s);        // z0, delta_0
        return cudaSuccess;
    }
    if (seg == kSegLoop) return P.comp ? launch_loop<true>(A, P, s) : launch_loop<false>(A, P, s);
    const dim3 pix_grid((unsigned)std::min<int64_t>((P.max_pixels + 255) / 256,
                                                    (int64_t)device_info().sms * 8),
                        (unsigned)A.ninst);
    if (P.mode == kSplatBackward) {
        prof_begin(f_bwd, s);
        backward_slice_kernel<<<pix_grid, 256, 0, s>>>(A);
        prof_end(f_bwd, s);
    } else {
        prof_begin(f_slice, s);
        slice_kernel<<<pix_grid, 256, 0, s>>>(A);
        prof_end(f_slice, s);
        if (P.export_y) {
            const dim3 yg((unsigned)std::min<int64_t>((P.max_cv + 255) / 256,
                                                      (int64_t)device_info().sms * 4),
                          (unsigned)A.ninst);
            prof_begin(f_export, s);
            export_y_kernel<<<yg, 256, 0, s>>>(A);
            prof_end(f_export, s);
        }
    }
    return cudaGetLastError();
}

}  // namespace fbs
