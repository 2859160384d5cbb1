// Device passes of the low-rank reduction of a wide target (supplement,
// multiple output channels; the rank-revealing QR reduction of B): the
// splat B = S(c o t), the Gram matrix B^T B and per-pixel channel maps.
#include <algorithm>

#include "fbs_internal.cuh"
#include "lowrank.cuh"

namespace fbs {
namespace {

// image of grid vertex v (voff ascending, n + 1 entries)
__device__ __forceinline__ int lr_image_of(const int64_t* voff, int n, int64_t v)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (voff[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One thread per vertex: B[v][ch] = sum over the vertex's pixels of c t_ch,
// channels in blocks of 8, double-float sums in the sorted pixel order.
__global__ void __launch_bounds__(256)
lr_splat_kernel(const LrImg* __restrict__ imgs, int n, int64_t Vtot, const int64_t* __restrict__ voff,
                const uint32_t* __restrict__ pstart, const uint32_t* __restrict__ m,
                const uint32_t* __restrict__ perm, float* __restrict__ B)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < Vtot;
         v += (int64_t)gridDim.x * blockDim.x) {
        const LrImg& I = imgs[lr_image_of(voff, n, v)];
        const uint32_t p0 = pstart[v], cnt = m[v];
        float* row = B + I.boff + (v - I.v0) * I.C;
        for (int cb = 0; cb < I.C; cb += 8) {
            DF acc[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = DF{0.0f, 0.0f};
            // 4 pixels' loads in flight, then their sums in pixel order
            for (uint32_t j0 = 0; j0 < cnt; j0 += 4) {
                int64_t ii[4];
                float w[4], val[8][4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    ii[u] = j0 + u < cnt ? (int64_t)perm[p0 + j0 + u] - I.pix_base : 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    w[u] = j0 + u < cnt ? I.c[ii[u]] : 0.0f;
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        val[k][u] = cb + k < I.C ? I.t[(cb + k) * I.N + ii[u]] : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (j0 + u < cnt) {
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            if (cb + k < I.C) acc[k] = df_add(acc[k], df_mul_exact(w[u], val[k][u]));
                    }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (cb + k < I.C) row[cb + k] = acc[k].hi + acc[k].lo;
        }
    }
}

constexpr int kLrThreads = 256;
constexpr int kLrRows = 32;                                   // rows of B staged per round
constexpr int kLrPerThread = (kLrMaxEntries + kLrThreads - 1) / kLrThreads;

// Block (x, image): the Gram entries (i <= j, row-major upper triangle) over
// the block's share of the image's vertices; thread e takes entries e,
// e + 256, ...  Exact products, double-float sums in vertex order.
__global__ void __launch_bounds__(kLrThreads)
lr_gram_kernel(const LrImg* __restrict__ imgs, const float* __restrict__ B, float2* __restrict__ part,
               int pstride)
{
    __shared__ float rows[kLrRows * 64];
    const LrImg I = imgs[blockIdx.y];
    const int C = I.C;
    const int nent = C * (C + 1) / 2;
    int ei[kLrPerThread], ej[kLrPerThread];
    DF acc[kLrPerThread];
#pragma unroll
    for (int q = 0; q < kLrPerThread; ++q) {
        acc[q] = DF{0.0f, 0.0f};
        int e = threadIdx.x + q * kLrThreads, i = 0;
        ej[q] = -1;
        ei[q] = 0;
        if (e < nent) {
            while (e >= C - i) { e -= C - i; ++i; }
            ei[q] = i;
            ej[q] = i + e;
        }
    }
    const int64_t per = (I.nv + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * per, r1 = r0 + per < I.nv ? r0 + per : I.nv;
    const float* Bi = B + I.boff;
    for (int64_t rb = r0; rb < r1; rb += kLrRows) {
        const int nr = (int)(r1 - rb < kLrRows ? r1 - rb : kLrRows);
        __syncthreads();
        for (int k = threadIdx.x; k < nr * C; k += kLrThreads) rows[k] = Bi[rb * C + k];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kLrPerThread; ++q) {
            if (ej[q] < 0) continue;
            for (int r = 0; r < nr; ++r)
                acc[q] = df_add(acc[q], df_mul_exact(rows[r * C + ei[q]], rows[r * C + ej[q]]));
        }
    }
    float2* out = part + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * pstride;
#pragma unroll
    for (int q = 0; q < kLrPerThread; ++q) {
        const int e = threadIdx.x + q * kLrThreads;
        if (e < nent) out[e] = make_float2(acc[q].hi, acc[q].lo);
    }
}

// G (C x C, symmetric, FP64) of each image from its blocks' partials, in
// block order.
__global__ void __launch_bounds__(kLrThreads)
lr_gram_reduce_kernel(const LrImg* __restrict__ imgs, const float2* __restrict__ part, int nblk,
                      int pstride, double* __restrict__ G, int cmax)
{
    const LrImg I = imgs[blockIdx.x];
    const int C = I.C;
    const int nent = C * (C + 1) / 2;
    for (int e = threadIdx.x; e < nent; e += blockDim.x) {
        DF s = {0.0f, 0.0f};
        for (int b = 0; b < nblk; ++b) {
            const float2 p = part[((int64_t)blockIdx.x * nblk + b) * pstride + e];
            s = df_add(s, DF{p.x, p.y});
        }
        int i = 0, r = e;
        while (r >= C - i) { r -= C - i; ++i; }
        const int j = i + r;
        const double v = (double)s.hi + (double)s.lo;
        double* Gi = G + (int64_t)blockIdx.x * cmax * cmax;
        Gi[i * cmax + j] = v;
        Gi[j * cmax + i] = v;
    }
}

// Block (x, image): out[q][i] = sum_c M[c][q] in[c][i] for the image's
// pixels, outputs in blocks of 8 (M staged in shared memory).
__global__ void __launch_bounds__(256)
lr_map_kernel(const LrImg* __restrict__ imgs)
{
    __shared__ float sM[64 * 64];
    const LrImg I = imgs[blockIdx.y];
    for (int k = threadIdx.x; k < I.C * I.Cout; k += blockDim.x) sM[k] = I.M[k];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < I.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int q0 = 0; q0 < I.Cout; q0 += 8) {
            float acc[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = 0.0f;
            for (int c = 0; c < I.C; ++c) {
                const float v = I.t[c * I.N + i];
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (q0 + k < I.Cout) acc[k] = fmaf(sM[c * I.Cout + q0 + k], v, acc[k]);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (q0 + k < I.Cout) I.out[(q0 + k) * I.N + i] = acc[k];
        }
    }
}

}  // namespace

cudaError_t lr_splat(const LrImg* imgs_dev, int n_images, int64_t Vtot, const int64_t* voff_dev,
                     const uint32_t* pstart, const uint32_t* m, const uint32_t* perm, float* B,
                     cudaStream_t s)
{
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((Vtot + 255) / 256,
                                                               (int64_t)device_info().sms * 8));
    static int fam = prof_family("lr_splat");
    prof_begin(fam, s);
    lr_splat_kernel<<<nb, 256, 0, s>>>(imgs_dev, n_images, Vtot, voff_dev, pstart, m, perm, B);
    prof_end(fam, s);
    return cudaGetLastError();
}

cudaError_t lr_gram(const LrImg* imgs_dev, int n_images, const float* B, float2* part, double* G,
                    int cmax, cudaStream_t s)
{
    const int pstride = cmax * (cmax + 1) / 2;
    static int fam = prof_family("lr_gram");
    prof_begin(fam, s);
    lr_gram_kernel<<<dim3(kLrGramBlocks, n_images), kLrThreads, 0, s>>>(imgs_dev, B, part, pstride);
    lr_gram_reduce_kernel<<<n_images, kLrThreads, 0, s>>>(imgs_dev, part, kLrGramBlocks, pstride, G,
                                                         cmax);
    prof_end(fam, s);
    return cudaGetLastError();
}

cudaError_t lr_map(const LrImg* imgs_dev, int n_images, int64_t max_pixels, cudaStream_t s)
{
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((max_pixels + 255) / 256,
                                                               (int64_t)device_info().sms * 4));
    static int fam = prof_family("lr_map");
    prof_begin(fam, s);
    lr_map_kernel<<<dim3(nb, n_images), 256, 0, s>>>(imgs_dev);
    prof_end(fam, s);
    return cudaGetLastError();
}

}  // namespace fbs
