// Solve kernels: splat (b = S(c o t), S c, diag(A), Jacobi M^-1 and the flat
// initialisation), the initial residual, the two phases of each PCG
// iteration, the slice, and the backward adjoints.
//
// Every vertex kernel walks a table of CTA-sized vertex tiles; each tile
// belongs to one image ("instance"), so one launch advances every (image,
// channel) problem of a batch.  The two CG inner products of an iteration
// are reduced per tile (exact FP32 products summed as double-float pairs in
// registers, then FP64 across warps), stored as FP64 tile partials, and the
// last tile of an image to finish (counted with an atomic) sums that image's
// partials in a fixed order and updates its CG scalars -- so results are
// bitwise reproducible run to run and no host round trip is needed.
#include "fbs_internal.cuh"
#include "solve.cuh"

namespace fbs {

namespace {

__device__ __forceinline__ int64_t vec_index(const InstDev& I, int ch, int64_t v)
{
    return I.vec_base + (int64_t)ch * I.V + (v - I.voff);
}

__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

// Block-reduce CB double-float partials per channel and store each as the
// FP64 partial of this tile.
template <int CB>
__device__ void store_tile_partials(DF (&acc)[CB], const InstDev& I, const VTile& vt, int cb,
                                    double* __restrict__ part, double (*red)[kVTile / 32])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < CB; ++k) {
        DF s = df_warp_sum(acc[k]);
        if (lane == 0) red[k][w] = df_to_double(s);
    }
    __syncthreads();
    if (threadIdx.x < CB) {
        const int k = threadIdx.x, ch = cb + k;
        if (ch < I.C) {
            double t = 0.0;
            for (int j = 0; j < (int)(blockDim.x >> 5); ++j) t += red[k][j];
            part[I.part_base + (int64_t)ch * I.ntiles + vt.t_in_inst] = t;
        }
    }
    __syncthreads();
}

enum FinishKind { kFinishDelta0 = 0, kFinishAlpha = 1, kFinishBeta = 2 };

// Called by every block after it wrote all partials of a tile: the last
// tile of the image sums the image's partials (fixed order) and updates the
// CG scalars of its channels.
__device__ void finish_tile(const InstDev& I, int inst, double* __restrict__ part,
                            unsigned* __restrict__ cnt, Scal* __restrict__ scal, int kind)
{
    __shared__ int s_last;
    __shared__ double s_red[kVTile / 32];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(&cnt[inst], 1u);
        s_last = prev == (unsigned)(I.ntiles - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int ch = 0; ch < I.C; ++ch) {
        const double* p = part + I.part_base + (int64_t)ch * I.ntiles;
        double t = 0.0;
        for (int j = threadIdx.x; j < I.ntiles; j += blockDim.x) t += __ldcg(p + j);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
        if (lane == 0) s_red[w] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            double total = 0.0;
            for (int j = 0; j < (int)(blockDim.x >> 5); ++j) total += s_red[j];
            Scal& S = scal[I.pc + ch];
            if (kind == kFinishDelta0) {
                S.delta = total;
                S.beta = 0.0;
                S.alpha = 0.0;
            } else if (kind == kFinishAlpha) {
                S.dq = total;
                S.alpha = (total > 0.0 && S.delta != 0.0) ? S.delta / total : 0.0;
            } else {
                const double old = S.delta;
                S.delta = total;
                S.beta = old != 0.0 ? total / old : 0.0;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) cnt[inst] = 0u;
}

// ---------------------------------------------------------------- splat ---
// One thread per vertex sums its pixels (in the sorted pixel order, so the
// result is deterministic) with exact products accumulated as double-float
// pairs.  Writes b into r, y0 = b / S c into y, diag(A) into a, and
// {n, M^-1} into nm.
template <int CB>
__global__ void __launch_bounds__(kVTile)
splat_kernel(SolveArgs A, int mode, float sigma_gm, int comp)
{
    const float s2 = sigma_gm * sigma_gm;
    for (int tile = blockIdx.x; tile < A.nvt; tile += gridDim.x) {
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
            for (uint32_t j = 0; j < cnt; ++j) {
                const int64_t i = (int64_t)A.perm[p0 + j] - I.pix_base;
                float w;
                if (mode == kSplatRobust) {
                    const float e = yv - I.t[i];
                    const float den = s2 + e * e;
                    w = (2.0f * s2) / (den * den);
                } else {
                    w = I.c[i];
                }
                if (cb == 0) {
                    sc = df_add(sc, DF{w, 0.0f});
                    bad |= !isfinite(w);
                }
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    const int ch = cb + k;
                    if (ch < I.C) {
                        if (mode == kSplatBackward) {
                            const float g = I.dx[(int64_t)ch * I.N + i];
                            acc[k] = df_add(acc[k], DF{g, 0.0f});
                            bad |= !isfinite(g);
                        } else {
                            const float tv = I.t[(int64_t)ch * I.N + i];
                            acc[k] = df_add(acc[k], df_mul_exact(w, tv));
                            bad |= !isfinite(tv);
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
        // A is applied in Laplacian form,
        //   (A z)_v = a'_v z_v + lambda n_v sum_u n_u (z_v - z_u),
        //   a'_v    = lambda (m_v - n_v (Bbar n)_v) + (S c)_v,
        // which equals a_v z_v - lambda n_v sum_u n_u z_u with
        // a_v = diag(A)_v = lambda (m_v - 10 n_v^2) + (S c)_v.  a' is formed
        // in FP64 here; the off-diagonal part has zero row sums whatever the
        // rounding of n, so FP32 vectors keep the data term intact.  A vertex
        // without neighbours has smoothness part 0 (its row of
        // lambda (D_m - D_n Bbar D_n) vanishes once n^2 = m / 10).
        // M^-1 = 1 / diag(A), 0 where diag(A) <= 0.
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
        const double nv = A.n64[v];
        const double scd = (double)sc.hi + (double)sc.lo;
        const double lam = (double)I.lam;
        const double rem = has_nbr ? lam * ((double)cnt - nv * (10.0 * nv + sum_n)) : 0.0;
        const double diag = has_nbr ? lam * ((double)cnt - 10.0 * nv * nv) + scd : scd;
        A.a[v] = (float)(rem + scd);
        A.nm[v] = make_float2((float)nv, diag > 0.0 ? (float)(1.0 / diag) : 0.0f);
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
// r = b - A y0 (b is in r, and in r_lo too when COMP), then r^T M^-1 r ->
// delta, beta = 0.
template <int CB, bool COMP>
__global__ void __launch_bounds__(kVTile)
residual_kernel(SolveArgs A)
{
    __shared__ double red[CB][kVTile / 32];
    for (int tile = blockIdx.x; tile < A.nvt; tile += gridDim.x) {
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
            store_tile_partials<CB>(acc, I, vt, cb, A.part, red);
        }
        finish_tile(I, vt.inst, A.part, A.cnt + 0 * A.ninst, A.scal, kFinishDelta0);
    }
}

// ------------------------------------------------------- PCG phase 1 ---
// d = M^-1 r + beta d_old (own vertex and, on the fly, its neighbours),
// q = A d, partial d^T q; the last tile sets alpha = delta / d^T q.
// COMP: q is not stored (phase 2 recomputes it exactly from d).
template <int CB, bool COMP>
__global__ void __launch_bounds__(kVTile)
pcg_apply_kernel(SolveArgs A, const float* __restrict__ dold, float* __restrict__ dnew, int first)
{
    __shared__ double red[CB][kVTile / 32];
    for (int tile = blockIdx.x; tile < A.nvt; tile += gridDim.x) {
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
                    const float beta = first ? 0.0f : (float)A.scal[I.pc + ch].beta;
                    const float* r = A.r;
                    float dv = T.nmv.y * r[base + v];
                    if (!first) dv = fmaf(beta, dold[base + v], dv);
                    const DF q = laplacian_apply<COMP>(T.av, lam_n, T.nb, T.nmu, dv, [&](int j) {
                        const int64_t u = base + T.nb[j];
                        float du = T.nmu[j].y * r[u];
                        if (!first) du = fmaf(beta, dold[u], du);
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
            store_tile_partials<CB>(acc, I, vt, cb, A.part, red);
        }
        finish_tile(I, vt.inst, A.part, A.cnt + 1 * A.ninst, A.scal, kFinishAlpha);
    }
}

// ------------------------------------------------------- PCG phase 2 ---
// y += alpha d; r -= alpha q; partial r^T M^-1 r; the last tile sets
// beta = delta_new / delta_old.
// COMP: q = A d is recomputed here with compensated arithmetic and the
// residual is kept as a double-float pair (r, r_lo), so the recurrence
// r <- r - alpha A d carries no rounding of q.
template <int CB, bool COMP>
__global__ void __launch_bounds__(kVTile)
pcg_update_kernel(SolveArgs A, const float* __restrict__ d)
{
    __shared__ double red[CB][kVTile / 32];
    for (int tile = blockIdx.x; tile < A.nvt; tile += gridDim.x) {
        const VTile vt = A.vt[tile];
        const InstDev I = A.inst[vt.inst];
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
                    const double alpha = A.scal[I.pc + ch].alpha;
                    const float dv = d[idx];
                    A.y[idx] = fmaf((float)alpha, dv, A.y[idx]);
                    float rhi;
                    if (COMP) {
                        const DF q = laplacian_apply<true>(T.av, lam_n, T.nb, T.nmu, dv,
                                                           [&](int j) { return d[base + T.nb[j]]; });
                        const DF r = df_add(DF{A.r[idx], A.rlo[idx]},
                                            df_neg(df_mul(df_from_double(alpha), q)));
                        A.r[idx] = r.hi;
                        A.rlo[idx] = r.lo;
                        rhi = r.hi;
                    } else {
                        rhi = fmaf(-(float)alpha, A.q[idx], A.r[idx]);
                        A.r[idx] = rhi;
                    }
                    acc[k] = df_mul_exact(rhi, T.nmv.y * rhi);
                }
            }
            store_tile_partials<CB>(acc, I, vt, cb, A.part, red);
        }
        finish_tile(I, vt.inst, A.part, A.cnt + 2 * A.ninst, A.scal, kFinishBeta);
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
        const int nb_p = persistent_blocks(occ_p, A.nvt);
        const int nb_u = persistent_blocks(occ_u, A.nvt);
        for (int it = 0; it < P.pcg_iters; ++it) {
            const float* dold = A.d[(it + 1) & 1];
            float* dnew = A.d[it & 1];
            prof_begin(f_apply, s);
            pcg_apply_kernel<CB, COMP><<<nb_p, kVTile, 0, s>>>(A, dold, dnew, it == 0);
            prof_end(f_apply, s);
            prof_begin(f_update, s);
            pcg_update_kernel<CB, COMP><<<nb_u, kVTile, 0, s>>>(A, dnew);
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
