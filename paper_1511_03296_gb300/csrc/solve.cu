// Solve kernels: splat (b = S(c o t), S c, diag(A), Jacobi M^-1 and the flat
// initialisation), the initial residual, the two phases of each PCG
// iteration, the slice, and the backward adjoints.
//
// Every vertex kernel walks a table of CTA-sized vertex tiles; each tile
// belongs to one image ("instance"), so one launch advances every (image,
// channel) problem of a batch.  Each block takes a contiguous chunk of tiles.
//
// CG inner products: every tile writes, per channel, the sum of its exact
// FP32 products as a double-float pair ("tile partial").  The next phase's
// blocks each reduce the partials of the instances they touch, in a fixed
// order, and form the CG scalar they need (alpha or beta) in FP64 -- every
// block obtains the same value, so there is no grid-wide serial step, no
// atomic and no fence, and results are bitwise reproducible.
#include "fbs_internal.cuh"
#include "solve.cuh"

namespace fbs {

namespace {

__device__ __forceinline__ int64_t vec_index(const InstDev& I, int ch, int64_t v)
{
    return I.vec_base + (int64_t)ch * I.V + (v - I.voff);
}

__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

// contiguous chunk of tiles for this block
__device__ __forceinline__ void block_chunk(int nvt, int& t0, int& t1)
{
    const int chunk = (nvt + gridDim.x - 1) / gridDim.x;
    t0 = blockIdx.x * chunk;
    t1 = min(t0 + chunk, nvt);
}

// Block-reduce the CB double-float partials per channel of this tile and
// store them (one float2 per (tile, channel)).
template <int CB>
__device__ void store_tile_partials(DF (&acc)[CB], const InstDev& I, const VTile& vt, int cb,
                                    float2* __restrict__ part, DF (*red)[kVTile / 32])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < CB; ++k) {
        DF s = df_warp_sum(acc[k]);
        if (lane == 0) red[k][w] = s;
    }
    __syncthreads();
    if (threadIdx.x < CB) {
        const int k = threadIdx.x, ch = cb + k;
        if (ch < I.C) {
            DF t = red[k][0];
            for (int j = 1; j < (int)(blockDim.x >> 5); ++j) t = df_add(t, red[k][j]);
            part[I.part_base + (int64_t)ch * I.ntiles + vt.t_in_inst] = make_float2(t.hi, t.lo);
        }
    }
    __syncthreads();
}

// Sum, per channel, the tile partials of one instance (fixed order: lane j
// takes tiles j, j+32, ... in groups of 8 loads issued together; then the
// warp tree) into out[ch] (FP64).  Warps take channels round-robin.  Must
// be called by the whole block.  Partials written earlier in the same kernel
// by other blocks are read through L2 (ld.cg).
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
__device__ __forceinline__ void vertex_epilogue_terms(const SolveArgs& A, const InstDev& I,
                                                      int64_t v, uint32_t cnt, DF sc, bool has_nbr,
                                                      double sum_n)
{
    const double nv = A.n64[v];
    const double scd = (double)sc.hi + (double)sc.lo;
    const double lam = (double)I.lam;
    const double rem = has_nbr ? lam * ((double)cnt - nv * (10.0 * nv + sum_n)) : 0.0;
    const double diag = has_nbr ? lam * ((double)cnt - 10.0 * nv * nv) + scd : scd;
    A.a[v] = (float)(rem + scd);
    A.nm[v] = make_float2((float)nv, diag > 0.0 ? (float)(1.0 / diag) : 0.0f);
}

__device__ __forceinline__ void vertex_epilogue(const SolveArgs& A, const InstDev& I, int64_t v,
                                                uint32_t cnt, DF sc)
{
    bool has_nbr = false;
    double sum_n = 0.0;
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        const int32_t u = A.nbr[(int64_t)k * A.Vtot + v];
        if (u >= 0) {
            has_nbr = true;
            sum_n += A.n64[u];
        }
    }
    vertex_epilogue_terms(A, I, v, cnt, sc, has_nbr, sum_n);
}


// One thread per vertex sums its pixels (in the sorted pixel order, so the
// result is deterministic) with exact products accumulated as double-float
// pairs.  Writes b into r, y0 = b / S c into y, diag(A) into a, and
// {n, M^-1} into nm.
template <int CB>
__global__ void __launch_bounds__(kVTile)
splat_kernel(SolveArgs A, int mode, float sigma_gm, int comp)
{
    const float s2 = sigma_gm * sigma_gm;
    int t0, t1;
    block_chunk(A.nvt, t0, t1);
    for (int tile = t0; tile < t1; ++tile) {
        const VTile vt = A.vt[tile];
        const InstDev I = A.inst[vt.inst];
        const int64_t v = vt.v0 + threadIdx.x;
        if (v >= vt.v1) continue;
        const uint32_t p0 = A.pstart[v], cnt = A.m[v];
        float yv = 0.0f;
        if (mode == kSplatRobust) yv = A.y[vec_index(I, 0, v)];
        DF sc = {0.0f, 0.0f};
        bool bad = false;
        for (int cb = 0; cb < I.C; cb += CB) {
            DF acc[CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) acc[k] = {0.0f, 0.0f};
            // software-pipelined: the pixel indices of 8 items, then their
            // values, then the accumulation in item order (same order, so the
            // sums are those of a plain sequential loop)
            for (uint32_t j0 = 0; j0 < cnt; j0 += 8) {
                int64_t ii[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    ii[u] = j0 + u < cnt ? (int64_t)A.perm[p0 + j0 + u] - I.pix_base : -1;
                float wv[8], val[CB][8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int64_t i = ii[u] >= 0 ? ii[u] : 0;
                    if (mode == kSplatRobust) {
                        const float e = yv - I.t[i];
                        const float den = s2 + e * e;
                        wv[u] = (2.0f * s2) / (den * den);
                    } else {
                        wv[u] = I.c[i];
                    }
#pragma unroll
                    for (int k = 0; k < CB; ++k) {
                        const int ch = min(cb + k, I.C - 1);
                        val[k][u] = mode == kSplatBackward ? I.dx[(int64_t)ch * I.N + i]
                                                           : I.t[(int64_t)ch * I.N + i];
                    }
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
                }
            }
        }
        if (bad) atomicOr(A.err, kErrNonFinite);
        vertex_epilogue(A, I, v, cnt, sc);
    }
}

// Laplacian-form apply at one vertex for one channel:
//   (A z)_v = a'_v z_v + lambda n_v sum_u n_u (z_v - z_u).
// COMP = false: FP32 arithmetic (result in .hi, .lo = 0).
// COMP = true: every product is exact (two-product) and the sums are carried
// as double-float pairs, so the result is accurate to ~2^-44 relative.
template <bool COMP, typename NbrVal>
__device__ __forceinline__ DF laplacian_apply(float av, float lam_n, const int32_t (&nb)[10],
                                              const float2 (&nmu)[10], float zv, NbrVal zu)
{
    if (COMP) {
        DF s = {0.0f, 0.0f};
#pragma unroll
        for (int j = 0; j < 10; ++j)
            if (nb[j] >= 0) s = df_add(s, df_mul_exact(nmu[j].x, zv - zu(j)));
        return df_add(df_mul_exact(av, zv), df_mul_f(s, lam_n));
    } else {
        float s = 0.0f;
#pragma unroll
        for (int j = 0; j < 10; ++j)
            if (nb[j] >= 0) s = fmaf(nmu[j].x, zv - zu(j), s);
        return DF{fmaf(av, zv, lam_n * s), 0.0f};
    }
}

// Branch-free form over register arrays: nu[j] = n of neighbour j (0 when
// absent, which makes its term an exact zero), zu[j] its (finite) value.
template <bool COMP>
__device__ __forceinline__ DF laplacian_apply_v(float av, float lam_n, float zv,
                                                const float (&nu)[10], const float (&zu)[10])
{
    if (COMP) {
        DF s = {0.0f, 0.0f};
#pragma unroll
        for (int j = 0; j < 10; ++j) s = df_add(s, df_mul_exact(nu[j], zv - zu[j]));
        return df_add(df_mul_exact(av, zv), df_mul_f(s, lam_n));
    } else {
        float s = 0.0f;
#pragma unroll
        for (int j = 0; j < 10; ++j) s = fmaf(nu[j], zv - zu[j], s);
        return DF{fmaf(av, zv, lam_n * s), 0.0f};
    }
}

// topology of one vertex: neighbour ids, {n, M^-1} of the neighbours, a', {n, M^-1}
struct VertexTopo {
    int32_t nb[10];
    float2 nmu[10];
    float av;
    float2 nmv;
};

__device__ __forceinline__ void load_topo(const SolveArgs& A, int64_t v, bool valid, VertexTopo& T)
{
    T.av = 0.0f;
    T.nmv = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        T.nb[k] = valid ? A.nbr[(int64_t)k * A.Vtot + v] : -1;
        T.nmu[k] = T.nb[k] >= 0 ? A.nm[T.nb[k]] : make_float2(0.0f, 0.0f);
    }
    if (valid) {
        T.av = A.a[v];
        T.nmv = A.nm[v];
    }
}

// ------------------------------------------------------- initial residual ---
// r = b - A y0 (b is in r, and in r_lo too when COMP); tile partials of
// r^T M^-1 r (delta_0) into rs slot 0.
template <int CB, bool COMP>
__global__ void __launch_bounds__(kVTile)
residual_kernel(SolveArgs A)
{
    __shared__ DF red[CB][kVTile / 32];
    int t0, t1;
    block_chunk(A.nvt, t0, t1);
    for (int tile = t0; tile < t1; ++tile) {
        const VTile vt = A.vt[tile];
        const InstDev I = A.inst[vt.inst];
        const int64_t v = vt.v0 + threadIdx.x;
        const bool valid = v < vt.v1;
        VertexTopo T;
        load_topo(A, v, valid, T);
        const float lam_n = I.lam * T.nmv.x;
        for (int cb = 0; cb < I.C; cb += CB) {
            DF acc[CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                acc[k] = {0.0f, 0.0f};
                const int ch = cb + k;
                if (valid && ch < I.C) {
                    const int64_t base = I.vec_base + (int64_t)ch * I.V - I.voff;
                    const float* y = A.y;
                    const DF Ay = laplacian_apply<COMP>(T.av, lam_n, T.nb, T.nmu, y[base + v],
                                                        [&](int j) { return y[base + T.nb[j]]; });
                    float rhi;
                    if (COMP) {
                        const DF r = df_add(DF{A.r[base + v], A.rlo[base + v]}, df_neg(Ay));
                        A.r[base + v] = r.hi;
                        A.rlo[base + v] = r.lo;
                        rhi = r.hi;
                    } else {
                        rhi = A.r[base + v] - Ay.hi;
                        A.r[base + v] = rhi;
                    }
                    acc[k] = df_mul_exact(rhi, T.nmv.y * rhi);
                }
            }
            store_tile_partials<CB>(acc, I, vt, cb, A.part_rs[0], red);
        }
    }
}

// Loads of CG vectors: plain in the per-phase kernels; through L2 (ld.cg)
// in the persistent loop, where other blocks rewrite them between grid
// barriers and an SM's L1 could otherwise hold a stale line.
template <bool CO>
__device__ __forceinline__ float ldv(const float* p)
{
    return CO ? __ldcg(p) : *p;
}

// shared scratch of the two PCG phases
template <int CB>
struct PhaseSmem {
    DF red[CB][kVTile / 32];
    double sd[kMaxChannels];     // reduced inner products
    float sf[kMaxChannels];      // beta (phase 1)
    double sa[kMaxChannels];     // alpha (phase 2)
};

// ------------------------------------------------------- PCG phase 1 ---
// Iteration `it`: delta_it = reduce(rs partials of slot it % 2);
// beta = delta_it / delta_{it-1} (0 at it = 0); d = M^-1 r + beta d_old (own
// vertex and, on the fly, its neighbours); q = A d; tile partials of d^T q.
// delta_it is also stored (slot it % 2) for phase 2 and the next phase 1.
// COMP: q is not stored (phase 2 recomputes it exactly from d).
template <int CB, bool COMP, bool CO>
__device__ void phase_apply(const SolveArgs& A, const float* __restrict__ dold,
                            float* __restrict__ dnew, int it, int t0, int t1, PhaseSmem<CB>& S)
{
    const int slot = it & 1;
    const bool first = it == 0;
    int cur = -1;
    for (int tile = t0; tile < t1; ++tile) {
        const VTile vt = A.vt[tile];
        const InstDev I = A.inst[vt.inst];
        if (vt.inst != cur) {
            __syncthreads();
            reduce_instance_partials(A.part_rs[slot], I, S.sd);
            __syncthreads();
            if (threadIdx.x < I.C) {
                const int ch = threadIdx.x;
                const double dnow = S.sd[ch];
                double beta = 0.0;
                if (!first) {
                    const double dprev = CO ? __ldcg(&A.scal[I.pc + ch].delta[slot ^ 1])
                                            : A.scal[I.pc + ch].delta[slot ^ 1];
                    beta = dprev != 0.0 ? dnow / dprev : 0.0;
                }
                S.sf[ch] = (float)beta;
                A.scal[I.pc + ch].delta[slot] = dnow;   // same value from every block
            }
            __syncthreads();
            cur = vt.inst;
        }
        const int64_t v = vt.v0 + threadIdx.x;
        const bool valid = v < vt.v1;
        VertexTopo T;
        load_topo(A, v, valid, T);
        const float lam_n = I.lam * T.nmv.x;
        for (int cb = 0; cb < I.C; cb += CB) {
            DF acc[CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                acc[k] = {0.0f, 0.0f};
                const int ch = cb + k;
                if (valid && ch < I.C) {
                    const int64_t base = I.vec_base + (int64_t)ch * I.V - I.voff;
                    const float beta = S.sf[ch];
                    const float* r = A.r;
                    float dv = T.nmv.y * ldv<CO>(r + base + v);
                    if (!first) dv = fmaf(beta, ldv<CO>(dold + base + v), dv);
                    const DF q = laplacian_apply<COMP>(T.av, lam_n, T.nb, T.nmu, dv, [&](int j) {
                        const int64_t u = base + T.nb[j];
                        float du = T.nmu[j].y * ldv<CO>(r + u);
                        if (!first) du = fmaf(beta, ldv<CO>(dold + u), du);
                        return du;
                    });
                    dnew[base + v] = dv;
                    if (COMP) {
                        acc[k] = df_add(df_mul_exact(dv, q.hi), DF{dv * q.lo, 0.0f});
                    } else {
                        A.q[base + v] = q.hi;
                        acc[k] = df_mul_exact(dv, q.hi);
                    }
                }
            }
            store_tile_partials<CB>(acc, I, vt, cb, A.part_dq, S.red);
        }
    }
}

// ------------------------------------------------------- PCG phase 2 ---
// alpha = delta_it / reduce(d^T q partials) (0 if d^T q <= 0 or delta = 0);
// y += alpha d; r -= alpha q; tile partials of r^T M^-1 r into rs slot
// (it + 1) % 2.
// COMP: q = A d is recomputed here with compensated arithmetic and the
// residual is kept as a double-float pair (r, r_lo), so the recurrence
// r <- r - alpha A d carries no rounding of q.
template <int CB, bool COMP, bool CO>
__device__ void phase_update(const SolveArgs& A, const float* __restrict__ d, int it, int t0,
                             int t1, PhaseSmem<CB>& S)
{
    const int slot = it & 1;
    int cur = -1;
    for (int tile = t0; tile < t1; ++tile) {
        const VTile vt = A.vt[tile];
        const InstDev I = A.inst[vt.inst];
        if (vt.inst != cur) {
            __syncthreads();
            reduce_instance_partials(A.part_dq, I, S.sd);
            __syncthreads();
            if (threadIdx.x < I.C) {
                const int ch = threadIdx.x;
                const double delta = CO ? __ldcg(&A.scal[I.pc + ch].delta[slot])
                                        : A.scal[I.pc + ch].delta[slot];
                const double dq = S.sd[ch];
                S.sa[ch] = (dq > 0.0 && delta != 0.0) ? delta / dq : 0.0;
            }
            __syncthreads();
            cur = vt.inst;
        }
        const int64_t v = vt.v0 + threadIdx.x;
        const bool valid = v < vt.v1;
        VertexTopo T;
        if (COMP) {
            load_topo(A, v, valid, T);
        } else {
            T.nmv = valid ? A.nm[v] : make_float2(0.0f, 0.0f);
        }
        const float lam_n = I.lam * T.nmv.x;
        for (int cb = 0; cb < I.C; cb += CB) {
            DF acc[CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                acc[k] = {0.0f, 0.0f};
                const int ch = cb + k;
                if (valid && ch < I.C) {
                    const int64_t base = I.vec_base + (int64_t)ch * I.V - I.voff;
                    const int64_t idx = base + v;
                    const double alpha = S.sa[ch];
                    const float dv = ldv<CO>(d + idx);
                    A.y[idx] = fmaf((float)alpha, dv, ldv<CO>(A.y + idx));
                    float rhi;
                    if (COMP) {
                        const DF q = laplacian_apply<true>(T.av, lam_n, T.nb, T.nmu, dv,
                                                           [&](int j) { return ldv<CO>(d + base + T.nb[j]); });
                        const DF r = df_add(DF{ldv<CO>(A.r + idx), ldv<CO>(A.rlo + idx)},
                                            df_neg(df_mul(df_from_double(alpha), q)));
                        A.r[idx] = r.hi;
                        A.rlo[idx] = r.lo;
                        rhi = r.hi;
                    } else {
                        rhi = fmaf(-(float)alpha, ldv<CO>(A.q + idx), ldv<CO>(A.r + idx));
                        A.r[idx] = rhi;
                    }
                    acc[k] = df_mul_exact(rhi, T.nmv.y * rhi);
                }
            }
            store_tile_partials<CB>(acc, I, vt, cb, A.part_rs[slot ^ 1], S.red);
        }
    }
}

template <int CB, bool COMP>
__global__ void __launch_bounds__(kVTile)
pcg_apply_kernel(SolveArgs A, const float* __restrict__ dold, float* __restrict__ dnew, int it)
{
    __shared__ PhaseSmem<CB> S;
    int t0, t1;
    block_chunk(A.nvt, t0, t1);
    phase_apply<CB, COMP, false>(A, dold, dnew, it, t0, t1, S);
}

template <int CB, bool COMP>
__global__ void __launch_bounds__(kVTile)
pcg_update_kernel(SolveArgs A, const float* __restrict__ d, int it)
{
    __shared__ PhaseSmem<CB> S;
    int t0, t1;
    block_chunk(A.nvt, t0, t1);
    phase_update<CB, COMP, false>(A, d, it, t0, t1, S);
}

// ------------------------------------------------- persistent PCG loop ---
// Grid barrier for a cooperative launch.  Thread 0 of each block arrives on
// its group's counter (groups of consecutive blocks, each counter on its own
// 128-byte line); the last arrival of a group arrives on the top counter;
// the last group to arrive resets the top counter and advances the
// generation word that every block polls.  Layout of `bar` (words): [0] top
// counter, [1] generation, [32 g] counter of group g.  Every wait is
// bounded: on time-out the block records kErrTimeout and false is returned.
__device__ bool grid_barrier(unsigned* bar, uint32_t* err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned* top = bar;
        unsigned* gen = bar + 1;
        const unsigned gsize = (gridDim.x + kBarrierGroups - 1) / kBarrierGroups;
        const unsigned ngroups = (gridDim.x + gsize - 1) / gsize;
        const unsigned grp = blockIdx.x / gsize;
        const unsigned members = min(gsize, gridDim.x - grp * gsize);
        unsigned* gcount = bar + 32 * (grp + 1);
        const unsigned g = *(volatile unsigned*)gen;
        __threadfence();
        bool released = false;
        if (atomicAdd(gcount, 1u) == members - 1) {
            *(volatile unsigned*)gcount = 0u;
            if (atomicAdd(top, 1u) == ngroups - 1) {
                *(volatile unsigned*)top = 0u;
                __threadfence();
                atomicAdd(gen, 1u);
                released = true;
            }
        }
        if (!released) {
            unsigned spins = 0;
            while (*(volatile unsigned*)gen == g) {
                if (++spins > kBarrierSpinLimit) {
                    atomicOr(err, kErrTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// All `iters` PCG iterations in one cooperative launch: phase 1, barrier,
// phase 2, barrier.  Every block keeps the same chunk of tiles throughout.
template <int CB, bool COMP>
__global__ void __launch_bounds__(kVTile)
pcg_loop_kernel(SolveArgs A, int iters, unsigned* bar)
{
    __shared__ PhaseSmem<CB> S;
    int t0, t1;
    block_chunk(A.nvt, t0, t1);
    for (int it = 0; it < iters; ++it) {
        const float* dold = A.d[(it + 1) & 1];
        float* dnew = A.d[it & 1];
        phase_apply<CB, COMP, true>(A, dold, dnew, it, t0, t1, S);
        if (!grid_barrier(bar, A.err)) return;
        phase_update<CB, COMP, true>(A, dnew, it, t0, t1, S);
        if (!grid_barrier(bar, A.err)) return;
    }
}

// ------------------------------------------ resident persistent PCG loop ---
// The same iterations when every tile has its own co-resident block and an
// image has at most CB channels: each block keeps its tile's neighbour ids
// and neighbours' {n, M^-1} in shared memory for the whole loop, and each
// thread keeps its vertex's r, y, d (and q) in registers, writing d and r for
// the neighbours and y once at the end.  Neighbour gathers use a safe index
// (the vertex itself when a neighbour is absent) so they issue together.

// All threads sum the tile partials of one instance for all its channels
// (thread t takes tiles t, t + blockDim, ...), then a block tree; out[ch].
template <int CB>
__device__ void reduce_partials_all(const float2* __restrict__ part, const InstDev& I,
                                    double* out, DF (*red)[kVTile / 32])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    DF acc[CB];
#pragma unroll
    for (int k = 0; k < CB; ++k) acc[k] = {0.0f, 0.0f};
    for (int j0 = threadIdx.x; j0 < I.ntiles; j0 += 2 * blockDim.x) {
        float2 v[CB][2];
#pragma unroll
        for (int k = 0; k < CB; ++k)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = j0 + h * blockDim.x;
                v[k][h] = (k < I.C && j < I.ntiles)
                              ? __ldcg(part + I.part_base + (int64_t)k * I.ntiles + j)
                              : make_float2(0.0f, 0.0f);
            }
#pragma unroll
        for (int k = 0; k < CB; ++k)
#pragma unroll
            for (int h = 0; h < 2; ++h) acc[k] = df_add(acc[k], DF{v[k][h].x, v[k][h].y});
    }
#pragma unroll
    for (int k = 0; k < CB; ++k) {
        const DF t = df_warp_sum(acc[k]);
        if (lane == 0) red[k][w] = t;
    }
    __syncthreads();
    if (threadIdx.x < CB && threadIdx.x < I.C) {
        const int k = threadIdx.x;
        DF t = red[k][0];
        for (int j = 1; j < nw; ++j) t = df_add(t, red[k][j]);
        out[k] = df_to_double(t);
    }
    __syncthreads();
}

template <int CB>
__device__ __forceinline__ void store_partials_resident(DF (&acc)[CB], const InstDev& I,
                                                        const VTile& vt, float2* __restrict__ part,
                                                        DF (*red)[kVTile / 32])
{
    store_tile_partials<CB>(acc, I, vt, 0, part, red);
}

template <int CB, bool COMP>
__global__ void __launch_bounds__(kVTile, 3)
pcg_resident_kernel(SolveArgs A, int iters, unsigned* bar)
{
    __shared__ int32_t s_nb[10][kVTile];
    __shared__ float2 s_nmu[10][kVTile];
    __shared__ PhaseSmem<CB> S;
    const VTile vt = A.vt[blockIdx.x];
    const InstDev I = A.inst[vt.inst];
    const int64_t v = vt.v0 + threadIdx.x;
    const bool valid = v < vt.v1;
    const int tx = threadIdx.x;
    // topology, once
    float av = 0.0f;
    float2 nmv = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        const int32_t u = valid ? A.nbr[(int64_t)k * A.Vtot + v] : -1;
        s_nb[k][tx] = u;
        s_nmu[k][tx] = u >= 0 ? A.nm[u] : make_float2(0.0f, 0.0f);
    }
    if (valid) {
        av = A.a[v];
        nmv = A.nm[v];
    }
    const float lam_n = I.lam * nmv.x;
    // own state in registers
    float r[CB], rlo[CB], y[CB], d[CB], q[CB];
    int64_t base[CB];
#pragma unroll
    for (int k = 0; k < CB; ++k) {
        base[k] = I.vec_base + (int64_t)min(k, I.C - 1) * I.V - I.voff;
        const bool on = valid && k < I.C;
        r[k] = on ? A.r[base[k] + v] : 0.0f;
        rlo[k] = on && COMP ? A.rlo[base[k] + v] : 0.0f;
        y[k] = on ? A.y[base[k] + v] : 0.0f;
        d[k] = 0.0f;
        q[k] = 0.0f;
    }
    const int64_t vs = valid ? v : vt.v0;   // safe gather index for absent neighbours
    for (int it = 0; it < iters; ++it) {
        const int slot = it & 1;
        const float* dold = A.d[(it + 1) & 1];
        float* dnew = A.d[it & 1];
        // ---- phase 1: gathers first (they do not depend on beta), then the
        // reduction of the previous phase's partials overlaps their latency
        {
            DF acc[CB];
            float ru[CB][10], du[CB][10], nu[10], mu[10];
#pragma unroll
            for (int j = 0; j < 10; ++j) {
                const int32_t u0 = s_nb[j][tx];
                const int64_t u = u0 >= 0 ? u0 : vs;
                const float2 nm = s_nmu[j][tx];
                nu[j] = nm.x;
                mu[j] = nm.y;
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    ru[k][j] = __ldcg(A.r + base[k] + u);
                    du[k][j] = it > 0 ? __ldcg(dold + base[k] + u) : 0.0f;
                }
            }
            reduce_partials_all<CB>(A.part_rs[slot], I, S.sd, S.red);
            if (threadIdx.x < I.C && threadIdx.x < CB) {
                const int ch = threadIdx.x;
                double beta = 0.0;
                if (it > 0) {
                    const double dprev = __ldcg(&A.scal[I.pc + ch].delta[slot ^ 1]);
                    beta = dprev != 0.0 ? S.sd[ch] / dprev : 0.0;
                }
                S.sf[ch] = (float)beta;
                A.scal[I.pc + ch].delta[slot] = S.sd[ch];
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                acc[k] = {0.0f, 0.0f};
                if (valid && k < I.C) {
                    const float beta = S.sf[k];
                    const float dv = fmaf(beta, d[k], nmv.y * r[k]);
                    float dz[10];
#pragma unroll
                    for (int j = 0; j < 10; ++j) dz[j] = fmaf(beta, du[k][j], mu[j] * ru[k][j]);
                    const DF qq = laplacian_apply_v<COMP>(av, lam_n, dv, nu, dz);
                    d[k] = dv;
                    q[k] = qq.hi;
                    dnew[base[k] + v] = dv;
                    acc[k] = COMP ? df_add(df_mul_exact(dv, qq.hi), DF{dv * qq.lo, 0.0f})
                                  : df_mul_exact(dv, qq.hi);
                }
            }
            store_partials_resident<CB>(acc, I, vt, A.part_dq, S.red);
        }
        if (!grid_barrier(bar, A.err)) return;
        // ---- phase 2
        reduce_partials_all<CB>(A.part_dq, I, S.sd, S.red);
        if (threadIdx.x < I.C && threadIdx.x < CB) {
            const int ch = threadIdx.x;
            const double delta = __ldcg(&A.scal[I.pc + ch].delta[slot]);
            const double dq = S.sd[ch];
            S.sa[ch] = (dq > 0.0 && delta != 0.0) ? delta / dq : 0.0;
        }
        __syncthreads();
        {
            DF acc[CB];
            float dn[CB][10], nu[10];
            if (COMP) {
#pragma unroll
                for (int j = 0; j < 10; ++j) {
                    const int32_t u0 = s_nb[j][tx];
                    const int64_t u = u0 >= 0 ? u0 : vs;
                    nu[j] = s_nmu[j][tx].x;
#pragma unroll
                    for (int k = 0; k < CB; ++k) dn[k][j] = __ldcg(dnew + base[k] + u);
                }
            }
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                acc[k] = {0.0f, 0.0f};
                if (valid && k < I.C) {
                    const double alpha = S.sa[k];
                    y[k] = fmaf((float)alpha, d[k], y[k]);
                    if (COMP) {
                        const DF qq = laplacian_apply_v<true>(av, lam_n, d[k], nu, dn[k]);
                        const DF rr = df_add(DF{r[k], rlo[k]},
                                             df_neg(df_mul(df_from_double(alpha), qq)));
                        r[k] = rr.hi;
                        rlo[k] = rr.lo;
                    } else {
                        r[k] = fmaf(-(float)alpha, q[k], r[k]);
                    }
                    A.r[base[k] + v] = r[k];
                    acc[k] = df_mul_exact(r[k], nmv.y * r[k]);
                }
            }
            store_partials_resident<CB>(acc, I, vt, A.part_rs[slot ^ 1], S.red);
        }
        if (!grid_barrier(bar, A.err)) return;
    }
#pragma unroll
    for (int k = 0; k < CB; ++k)
        if (valid && k < I.C) {
            A.y[base[k] + v] = y[k];
            if (COMP) A.rlo[base[k] + v] = rlo[k];
        }
}

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
        for (int ch = 0; ch < I.C; ++ch) I.x[(int64_t)ch * I.N + i] = A.y[vec_index(I, ch, v)];
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
            const float z = A.y[vec_index(I, ch, v)];
            if (I.dt) I.dt[(int64_t)ch * I.N + i] = ci * z;
            const float yh = I.yhat[(int64_t)ch * I.V + (v - I.voff)];
            dc = fmaf(z, I.t[(int64_t)ch * I.N + i] - yh, dc);
        }
        if (I.dc) I.dc[i] = dc;
    }
}

// copy y (C x V of each image) to the caller's buffers
__global__ void __launch_bounds__(256)
export_y_kernel(SolveArgs A)
{
    const InstDev I = A.inst[blockIdx.y];
    float* dst = I.yout;
    if (dst == nullptr) return;
    const int64_t n = (int64_t)I.C * I.V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = A.y[I.vec_base + i];
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

template <int CB, bool COMP>
cudaError_t launch_segment_t(const SolveArgs& A, const SolvePlan& P, int seg, int mode,
                             cudaStream_t s)
{
    static int f_splat = prof_family("splat");
    static int f_res = prof_family("residual");
    static int f_apply = prof_family("pcg_apply");
    static int f_update = prof_family("pcg_update");
    static int f_slice = prof_family("slice");
    static int f_bwd = prof_family("backward_slice");
    static int f_export = prof_family("export_y");
    static const int occ_s = occupancy((const void*)splat_kernel<CB>);
    static const int occ_r = occupancy((const void*)residual_kernel<CB, COMP>);
    static const int occ_p = occupancy((const void*)pcg_apply_kernel<CB, COMP>);
    static const int occ_u = occupancy((const void*)pcg_update_kernel<CB, COMP>);
    if (seg == kSegSetup) {
        prof_begin(f_splat, s);
        splat_kernel<CB><<<persistent_blocks(occ_s, A.nvt), kVTile, 0, s>>>(A, mode, P.sigma_gm,
                                                                         COMP ? 1 : 0);
        prof_end(f_splat, s);
        prof_begin(f_res, s);
        residual_kernel<CB, COMP><<<persistent_blocks(occ_r, A.nvt), kVTile, 0, s>>>(A);
        prof_end(f_res, s);
    } else if (seg == kSegLoop) {
        if (P.persistent && P.pcg_iters > 0) {
            static const int occ_l = occupancy((const void*)pcg_loop_kernel<CB, COMP>);
            static const int occ_res = occupancy((const void*)pcg_resident_kernel<CB, COMP>);
            static int f_loop = prof_family("pcg_loop");
            static int f_res_loop = prof_family("pcg_resident");
            const bool resident = P.cmax <= CB && A.nvt <= device_info().sms * occ_res;
            // barrier words zero (or, for the failure-path test, a top counter
            // that the last arrival can never match)
            cudaError_t e = cudaMemsetAsync(P.barrier, 0, kBarrierWords * sizeof(unsigned), s);
            if (e == cudaSuccess && P.inject_timeout)   // top counter = 0x40000000 (little-endian)
                e = cudaMemsetAsync(reinterpret_cast<unsigned char*>(P.barrier) + 3, 0x40, 1, s);
            if (e != cudaSuccess) return e;
            SolveArgs a = A;
            int iters = P.pcg_iters;
            unsigned* bar = P.barrier;
            void* args[] = {&a, &iters, &bar};
            if (resident) {
                prof_begin(f_res_loop, s);
                e = cudaLaunchCooperativeKernel((const void*)pcg_resident_kernel<CB, COMP>,
                                                dim3(A.nvt), dim3(kVTile), args, 0, s);
                prof_end(f_res_loop, s);
            } else {
                const int nb_l = persistent_blocks(occ_l, A.nvt);
                prof_begin(f_loop, s);
                e = cudaLaunchCooperativeKernel((const void*)pcg_loop_kernel<CB, COMP>, dim3(nb_l),
                                                dim3(kVTile), args, 0, s);
                prof_end(f_loop, s);
            }
            if (e == cudaSuccess) return cudaGetLastError();
            cudaGetLastError();   // clear, and fall back to per-phase launches
        }
        const int nb_p = persistent_blocks(occ_p, A.nvt);
        const int nb_u = persistent_blocks(occ_u, A.nvt);
        for (int it = 0; it < P.pcg_iters; ++it) {
            const float* dold = A.d[(it + 1) & 1];
            float* dnew = A.d[it & 1];
            prof_begin(f_apply, s);
            pcg_apply_kernel<CB, COMP><<<nb_p, kVTile, 0, s>>>(A, dold, dnew, it);
            prof_end(f_apply, s);
            prof_begin(f_update, s);
            pcg_update_kernel<CB, COMP><<<nb_u, kVTile, 0, s>>>(A, dnew, it);
            prof_end(f_update, s);
        }
    } else {
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
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_segment(const SolveArgs& A, const SolvePlan& P, int seg, int mode,
                           cudaStream_t s)
{
    if (P.comp) {
        switch (P.chan_block) {
            case 1: return launch_segment_t<1, true>(A, P, seg, mode, s);
            case 2: return launch_segment_t<2, true>(A, P, seg, mode, s);
            case 3: return launch_segment_t<3, true>(A, P, seg, mode, s);
            default: return launch_segment_t<4, true>(A, P, seg, mode, s);
        }
    }
    switch (P.chan_block) {
        case 1: return launch_segment_t<1, false>(A, P, seg, mode, s);
        case 2: return launch_segment_t<2, false>(A, P, seg, mode, s);
        case 3: return launch_segment_t<3, false>(A, P, seg, mode, s);
        default: return launch_segment_t<4, false>(A, P, seg, mode, s);
    }
}

}  // namespace fbs
