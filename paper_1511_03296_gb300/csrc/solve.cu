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
splat_kernel(SolveArgs A, int mode, float sigma_gm)
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
                    A.r[idx] = b;
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

// ------------------------------------------------------- initial residual ---
// r = b - A y0 (b is in r), then r^T M^-1 r -> delta, beta = 0.
template <int CB>
__global__ void __launch_bounds__(kVTile)
residual_kernel(SolveArgs A)
{
    __shared__ double red[CB][kVTile / 32];
    for (int tile = blockIdx.x; tile < A.nvt; tile += gridDim.x) {
        const VTile vt = A.vt[tile];
        const InstDev I = A.inst[vt.inst];
        const int64_t v = vt.v0 + threadIdx.x;
        const bool valid = v < vt.v1;
        int32_t nb[10];
        float2 nmu[10];
        float av = 0.0f;
        float2 nmv = make_float2(0.0f, 0.0f);
        if (valid) {
            av = A.a[v];
            nmv = A.nm[v];
#pragma unroll
            for (int k = 0; k < 10; ++k) {
                nb[k] = A.nbr[(int64_t)k * A.Vtot + v];
                nmu[k] = nb[k] >= 0 ? A.nm[nb[k]] : make_float2(0.0f, 0.0f);
            }
        }
        for (int cb = 0; cb < I.C; cb += CB) {
            DF acc[CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                acc[k] = {0.0f, 0.0f};
                const int ch = cb + k;
                if (valid && ch < I.C) {
                    const int64_t base = I.vec_base + (int64_t)ch * I.V - I.voff;
                    const float yv = A.y[base + v];
                    float s = 0.0f;
#pragma unroll
                    for (int j = 0; j < 10; ++j)
                        if (nb[j] >= 0) s = fmaf(nmu[j].x, yv - A.y[base + nb[j]], s);
                    const float Ay = fmaf(av, yv, I.lam * nmv.x * s);
                    const float rv = A.r[base + v] - Ay;
                    A.r[base + v] = rv;
                    acc[k] = df_mul_exact(rv, nmv.y * rv);
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
template <int CB>
__global__ void __launch_bounds__(kVTile)
pcg_apply_kernel(SolveArgs A, const float* __restrict__ dold, float* __restrict__ dnew, int first)
{
    __shared__ double red[CB][kVTile / 32];
    for (int tile = blockIdx.x; tile < A.nvt; tile += gridDim.x) {
        const VTile vt = A.vt[tile];
        const InstDev I = A.inst[vt.inst];
        const int64_t v = vt.v0 + threadIdx.x;
        const bool valid = v < vt.v1;
        int32_t nb[10];
        float2 nmu[10];
        float av = 0.0f;
        float2 nmv = make_float2(0.0f, 0.0f);
        if (valid) {
            av = A.a[v];
            nmv = A.nm[v];
#pragma unroll
            for (int k = 0; k < 10; ++k) {
                nb[k] = A.nbr[(int64_t)k * A.Vtot + v];
                nmu[k] = nb[k] >= 0 ? A.nm[nb[k]] : make_float2(0.0f, 0.0f);
            }
        }
        for (int cb = 0; cb < I.C; cb += CB) {
            DF acc[CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                acc[k] = {0.0f, 0.0f};
                const int ch = cb + k;
                if (valid && ch < I.C) {
                    const int64_t base = I.vec_base + (int64_t)ch * I.V - I.voff;
                    const float beta = first ? 0.0f : (float)A.scal[I.pc + ch].beta;
                    float dv = nmv.y * A.r[base + v];
                    if (!first) dv = fmaf(beta, dold[base + v], dv);
                    float s = 0.0f;
#pragma unroll
                    for (int j = 0; j < 10; ++j) {
                        if (nb[j] >= 0) {
                            float du = nmu[j].y * A.r[base + nb[j]];
                            if (!first) du = fmaf(beta, dold[base + nb[j]], du);
                            s = fmaf(nmu[j].x, dv - du, s);
                        }
                    }
                    const float qv = fmaf(av, dv, I.lam * nmv.x * s);
                    dnew[base + v] = dv;
                    A.q[base + v] = qv;
                    acc[k] = df_mul_exact(dv, qv);
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
template <int CB>
__global__ void __launch_bounds__(kVTile)
pcg_update_kernel(SolveArgs A, const float* __restrict__ d)
{
    __shared__ double red[CB][kVTile / 32];
    for (int tile = blockIdx.x; tile < A.nvt; tile += gridDim.x) {
        const VTile vt = A.vt[tile];
        const InstDev I = A.inst[vt.inst];
        const int64_t v = vt.v0 + threadIdx.x;
        const bool valid = v < vt.v1;
        const float minv = valid ? A.nm[v].y : 0.0f;
        for (int cb = 0; cb < I.C; cb += CB) {
            DF acc[CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                acc[k] = {0.0f, 0.0f};
                const int ch = cb + k;
                if (valid && ch < I.C) {
                    const int64_t idx = vec_index(I, ch, v);
                    const float alpha = (float)A.scal[I.pc + ch].alpha;
                    A.y[idx] = fmaf(alpha, d[idx], A.y[idx]);
                    const float rv = fmaf(-alpha, A.q[idx], A.r[idx]);
                    A.r[idx] = rv;
                    acc[k] = df_mul_exact(rv, minv * rv);
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

template <int CB>
cudaError_t launch_all(const SolveArgs& A, const SolvePlan& P, cudaStream_t s)
{
    static int f_splat = prof_family("splat");
    static int f_res = prof_family("residual");
    static int f_apply = prof_family("pcg_apply");
    static int f_update = prof_family("pcg_update");
    static int f_slice = prof_family("slice");
    static int f_bwd = prof_family("backward_slice");
    static int f_setup = prof_family("region:solve_setup", 2);
    static int f_loop = prof_family("region:pcg_loop", 2);
    static int f_out = prof_family("region:slice", 2);
    static const int occ_s = occupancy((const void*)splat_kernel<CB>);
    static const int occ_r = occupancy((const void*)residual_kernel<CB>);
    static const int occ_p = occupancy((const void*)pcg_apply_kernel<CB>);
    static const int occ_u = occupancy((const void*)pcg_update_kernel<CB>);
    const int nb_s = persistent_blocks(occ_s, A.nvt);
    const int nb_r = persistent_blocks(occ_r, A.nvt);
    const int nb_p = persistent_blocks(occ_p, A.nvt);
    const int nb_u = persistent_blocks(occ_u, A.nvt);
    const dim3 pix_grid((unsigned)std::min<int64_t>((P.max_pixels + 255) / 256,
                                                    (int64_t)device_info().sms * 8),
                        (unsigned)A.ninst);
    for (int outer = 0; outer < P.outer_iters; ++outer) {
        const int mode = P.mode == kSplatRobust && outer == 0 ? kSplatConfidence : P.mode;
        prof_begin(f_setup, s);
        prof_begin(f_splat, s);
        splat_kernel<CB><<<nb_s, kVTile, 0, s>>>(A, mode, P.sigma_gm);
        prof_end(f_splat, s);
        prof_begin(f_res, s);
        residual_kernel<CB><<<nb_r, kVTile, 0, s>>>(A);
        prof_end(f_res, s);
        prof_end(f_setup, s);
        prof_begin(f_loop, s);
        for (int it = 0; it < P.pcg_iters; ++it) {
            const float* dold = A.d[(it + 1) & 1];
            float* dnew = A.d[it & 1];
            prof_begin(f_apply, s);
            pcg_apply_kernel<CB><<<nb_p, kVTile, 0, s>>>(A, dold, dnew, it == 0);
            prof_end(f_apply, s);
            prof_begin(f_update, s);
            pcg_update_kernel<CB><<<nb_u, kVTile, 0, s>>>(A, dnew);
            prof_end(f_update, s);
        }
        prof_end(f_loop, s);
    }
    prof_begin(f_out, s);
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
            export_y_kernel<<<yg, 256, 0, s>>>(A);
        }
    }
    prof_end(f_out, s);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_solve(const SolveArgs& A, const SolvePlan& P, cudaStream_t s)
{
    switch (P.chan_block) {
        case 1: return launch_all<1>(A, P, s);
        case 2: return launch_all<2>(A, P, s);
        case 3: return launch_all<3>(A, P, s);
        default: return launch_all<4>(A, P, s);
    }
}

}  // namespace fbs
