// Domain transform post-filter (the solver's output is smoothed by it in
// Sec. 5; Gastal and Oliveira 2011, recursive formulation).  For a
// 3-channel guide I the step from a pixel to its left (upper) neighbour has
// length d = 1 + (sigma_s / sigma_r) sum_c |I_c(p) - I_c(p')| in the
// transformed domain; iteration i of N filters every row, then every column,
// with the first-order recursive filter of feedback a_i = exp(-sqrt(2) /
// sigma_i), sigma_i = sigma_s sqrt(3) 2^(N-i) / sqrt(4^N - 1), forward then
// backward:
//     J[k] <- (1 - a^d[k]) J[k] + a^d[k] J[k-1]       (k ascending)
//     J[k] <- (1 - a^d[k+1]) J[k] + a^d[k+1] J[k+1]   (k descending).
// Rows: one block per (row, channel) stages the row in shared memory and
// runs each direction as a parallel scan of the affine maps J -> A J + B
// (each thread composes a contiguous chunk, the block scans the chunk maps,
// each thread replays its chunk from its prefix).  Columns: one block per 32
// columns and channel, 8 row segments per column, the same composition
// across the segments (a warp's loads are 32 consecutive floats of a row).
#include <algorithm>
#include <cmath>

#include "fbs_internal.cuh"

namespace fbs {
namespace {

constexpr int kDtThreads = 256;

// x -> a x + b
struct Aff {
    float a, b;
};

// apply `earlier`, then `later`
__device__ __forceinline__ Aff aff_then(Aff later, Aff earlier)
{
    return {later.a * earlier.a, fmaf(later.a, earlier.b, later.b)};
}

// exclusive scan of the threads' maps in thread order (thread 0 first)
__device__ Aff aff_block_exclusive(Aff m, Aff* s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Aff inc = m;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        Aff o;
        o.a = __shfl_up_sync(0xffffffffu, inc.a, off);
        o.b = __shfl_up_sync(0xffffffffu, inc.b, off);
        if (lane >= off) inc = aff_then(inc, o);
    }
    __syncthreads();                       // s_warp may still be read by a previous scan
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    Aff pre = {1.0f, 0.0f};
    for (int w = 0; w < warp; ++w) pre = aff_then(s_warp[w], pre);
    Aff ex;
    ex.a = __shfl_up_sync(0xffffffffu, inc.a, 1);
    ex.b = __shfl_up_sync(0xffffffffu, inc.b, 1);
    if (lane == 0) ex = {1.0f, 0.0f};
    return aff_then(ex, pre);
}

// One direction along a staged line of L values sx with step weights sw
// (sw[k] = a^d between k-1 and k).  Logical position r runs along the
// direction: forward r = k, backward r = L-1-k; element r's map is
// J -> A_r J + (1 - A_r) x with A_0 = 0 and A_r the weight of the step
// from the previous position.
// shared-memory slot of line element k: one pad word per 32, so that the
// threads' contiguous chunks fall in different banks
__device__ __forceinline__ int dt_pad(int k) { return k + (k >> 5); }

template <bool BACK>
__device__ void dt_scan(float* sx, const float* sw, int L, Aff* s_warp)
{
    const int per = (L + kDtThreads - 1) / kDtThreads;
    const int r0 = threadIdx.x * per, r1 = min(L, r0 + per);
    auto pos = [&](int r) { return dt_pad(BACK ? L - 1 - r : r); };
    auto wgt = [&](int r) { return r == 0 ? 0.0f : sw[dt_pad(BACK ? L - r : r)]; };
    Aff m = {1.0f, 0.0f};
    for (int r = r0; r < r1; ++r) {
        const float A = wgt(r);
        m = aff_then(Aff{A, (1.0f - A) * sx[pos(r)]}, m);
    }
    const Aff pre = aff_block_exclusive(m, s_warp);
    float J = pre.b;                       // the value before the chunk (A_0 = 0: start irrelevant)
    for (int r = r0; r < r1; ++r) {
        const float A = wgt(r);
        J = fmaf(A, J, (1.0f - A) * sx[pos(r)]);
        sx[pos(r)] = J;
    }
    __syncthreads();
}

// step lengths from the guide, pre-scaled: the weight of iteration i is
// exp2(k_i * d) with k_i = -sqrt(2) log2(e) / sigma_i
__global__ void __launch_bounds__(256)
dt_steps_kernel(const float* __restrict__ guide, int H, int W, float ratio, float* __restrict__ dh,
                float* __restrict__ dv)
{
    const int64_t N = (int64_t)H * W;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(p % W), y = (int)(p / W);
        float sh = 0.0f, sv = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = guide[c * N + p];
            if (x > 0) sh += fabsf(v - guide[c * N + p - 1]);
            if (y > 0) sv += fabsf(v - guide[c * N + p - W]);
        }
        dh[p] = fmaf(ratio, sh, 1.0f);
        dv[p] = fmaf(ratio, sv, 1.0f);
    }
}

// block (row, channel): both directions of one row
__global__ void __launch_bounds__(kDtThreads)
dt_rows_kernel(float* __restrict__ x, const float* __restrict__ dh, int H, int W, float kexp)
{
    extern __shared__ float s_line[];
    __shared__ Aff s_warp[kDtThreads / 32];
    const int Wp = dt_pad(W - 1) + 1;
    float* sx = s_line;
    float* sw = s_line + Wp;
    const int y = blockIdx.x;
    float* row = x + ((int64_t)blockIdx.y * H + y) * W;
    const float* d = dh + (int64_t)y * W;
    for (int k = threadIdx.x; k < W; k += kDtThreads) {
        sx[dt_pad(k)] = row[k];
        sw[dt_pad(k)] = exp2f(kexp * d[k]);
    }
    __syncthreads();
    dt_scan<false>(sx, sw, W, s_warp);
    dt_scan<true>(sx, sw, W, s_warp);
    for (int k = threadIdx.x; k < W; k += kDtThreads) row[k] = sx[dt_pad(k)];
}

// block (32 columns, channel), 8 row segments per column: each direction
// composes every segment's affine map, scans the 8 maps of each column in
// shared memory and replays the segments (a warp reads 32 consecutive
// floats of a row)
constexpr int kDtCols = 32, kDtSegs = 8;

__global__ void __launch_bounds__(kDtCols * kDtSegs)
dt_cols_kernel(float* __restrict__ x, const float* __restrict__ dv, int H, int W, float kexp)
{
    __shared__ Aff s_map[kDtSegs][kDtCols];
    const int lane = threadIdx.x % kDtCols, seg = threadIdx.x / kDtCols;
    const int col = blockIdx.x * kDtCols + lane;
    const bool valid = col < W;
    const int per = (H + kDtSegs - 1) / kDtSegs;
    const int y0 = min(H, seg * per), y1 = min(H, y0 + per);
    float* X = x + (int64_t)blockIdx.y * H * W + (valid ? col : 0);
    const float* d = dv + (valid ? col : 0);
    auto wdown = [&](int y) { return y == 0 ? 0.0f : exp2f(kexp * d[(int64_t)y * W]); };
    auto wup = [&](int y) { return y == H - 1 ? 0.0f : exp2f(kexp * d[(int64_t)(y + 1) * W]); };
    // down
    Aff m = {1.0f, 0.0f};
    if (valid)
        for (int y = y0; y < y1; ++y) {
            const float A = wdown(y);
            m = aff_then(Aff{A, (1.0f - A) * X[(int64_t)y * W]}, m);
        }
    s_map[seg][lane] = m;
    __syncthreads();
    Aff P = {1.0f, 0.0f};
    for (int q = 0; q < seg; ++q) P = aff_then(s_map[q][lane], P);
    if (valid) {
        float J = P.b;
        float xn = y0 < y1 ? X[(int64_t)y0 * W] : 0.0f;
        for (int y = y0; y < y1; ++y) {
            const float xv = xn;
            if (y + 1 < y1) xn = X[(int64_t)(y + 1) * W];     // the next row's load goes first
            const float A = wdown(y);
            J = fmaf(A, J, (1.0f - A) * xv);
            X[(int64_t)y * W] = J;
        }
    }
    __syncthreads();
    // up: segments in the order 7 .. 0, rows descending
    m = {1.0f, 0.0f};
    if (valid)
        for (int y = y1 - 1; y >= y0; --y) {
            const float A = wup(y);
            m = aff_then(Aff{A, (1.0f - A) * X[(int64_t)y * W]}, m);
        }
    s_map[seg][lane] = m;
    __syncthreads();
    P = {1.0f, 0.0f};
    for (int q = kDtSegs - 1; q > seg; --q) P = aff_then(s_map[q][lane], P);
    if (valid) {
        float J = P.b;
        float xn = y0 < y1 ? X[(int64_t)(y1 - 1) * W] : 0.0f;
        for (int y = y1 - 1; y >= y0; --y) {
            const float xv = xn;
            if (y - 1 >= y0) xn = X[(int64_t)(y - 1) * W];
            const float A = wup(y);
            J = fmaf(A, J, (1.0f - A) * xv);
            X[(int64_t)y * W] = J;
        }
    }
}

}  // namespace

// Rows longer than this do not fit the row kernel's shared memory.
constexpr int kDtMaxWidth = 28000;   // 2 x 4 B x 33/32 per pixel of a row: 231008 B of shared memory

cudaError_t domain_transform(const float* guide, int H, int W, float* x, int C, float sigma_s,
                             float sigma_r, int iters, float* dh, float* dv, cudaStream_t s)
{
    const int64_t N = (int64_t)H * W;
    const int sms = device_info().sms;
    dt_steps_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, sms * 8)), 256, 0,
                      s>>>(guide, H, W, sigma_s / sigma_r, dh, dv);
    const size_t smem = (size_t)2 * (W + W / 32 + 1) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(dt_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)std::max<size_t>(smem, 1));
    if (e != cudaSuccess) return e;
    const double log2e = 1.4426950408889634;
    for (int i = 1; i <= iters; ++i) {
        const double sig = sigma_s * sqrt(3.0) * pow(2.0, (double)(iters - i)) /
                           sqrt(pow(4.0, (double)iters) - 1.0);
        const float kexp = (float)(-sqrt(2.0) * log2e / sig);
        dt_rows_kernel<<<dim3((unsigned)H, (unsigned)C), kDtThreads, smem, s>>>(x, dh, H, W, kexp);
        dt_cols_kernel<<<dim3((unsigned)((W + kDtCols - 1) / kDtCols), (unsigned)C),
                         kDtCols * kDtSegs, 0, s>>>(x, dv, H, W, kexp);
    }
    return cudaGetLastError();
}

int domain_transform_max_width() { return kDtMaxWidth; }

}  // namespace fbs
