// Internal declarations of libfbs: device-side descriptors, helpers and the
// launch functions shared between translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/fbs.h"

namespace fbs {

// ---------------------------------------------------------------- limits ---
constexpr int kFieldMax = 4095;          // 12-bit key fields
constexpr int kMaxTilePixels = 16384;    // pixels sorted by one CTA of the grid build
constexpr int kGridThreads = 512;        // CTA size of the grid-build kernels
constexpr int kVTile = 256;              // vertices per PCG tile (= CTA size)
constexpr int kChanBlock = 4;            // channels processed per pass of a PCG tile
constexpr int kMaxChannels = 64;         // channels per image
// grid-barrier block (words): 0 the arrival counter, kWorkCounterWord the
// splat's work counter, 32 (a 128-byte line of its own) the release word of
// the resident loop's barrier; 33 lines in all
constexpr unsigned kBarrierWords = 32 * 33;
constexpr int kNbrOffMax = 32767;          // packed 16-bit neighbour offsets (y): |offset| <= this
constexpr int kNbrEscape = -32768;         // ... else this, and the 32-bit table holds the id
constexpr int kNbrOffMax8 = 127;           // packed 8-bit offsets (x, l, u, v): |offset| <= this
constexpr int kNbrEscape8 = -128;          // ... else this (the 32-bit table holds the id)
constexpr int kNbrWords = 3;               // packed words per vertex
constexpr unsigned kWorkCounterWord = 2;   // in the barrier block, unused by the barrier:
                                           // the splat's work counter
constexpr unsigned kBarrierSpinLimit = 1u << 20;   // polls of >= 64 ns (an L2 round trip and a
                                                    // 32 ns sleep): >= 67 ms before a time-out

// device error bits (latched in fbs_grid::err)
enum : uint32_t {
    kErrRange = 1u,       // key field outside [0, 4095] or NaN colour
    kErrNonFinite = 2u,   // NaN / Inf in t or c
    kErrGeometry = 4u,    // host / device disagree on a pixel's cell (internal)
    kErrTimeout = 8u,     // bounded wait ran out
};

// bit position of dimension d = (x, y, l, u, v) in the packed key
__host__ __device__ constexpr int key_shift(int d)
{
    return d == 0 ? 36 : d == 1 ? 48 : d == 2 ? 24 : d == 3 ? 12 : 0;
}

// --------------------------------------------------------- descriptors ---
struct ImgDev {
    const float* yuv;       // 3 x H x W
    int H, W;
    float sxy, sl, suv;
    float isxy, isl, isuv;  // 1 / sigma (FP32), for the quantiser's first estimate
    int ncx, ncy;           // number of cell columns / rows
    int64_t pix_base;       // first pixel in the concatenated pixel order
    int64_t cell_base;      // first cell in the concatenated cell order
};

// one CTA of the grid build: cells kx0 .. kx0+nkx-1 of cell row ky
struct GTile {
    int img, ky, kx0, nkx;
    int y0, y1, x0, x1;     // pixel rectangle [y0, y1) x [x0, x1)
    int64_t sort_off;       // offset of this tile's pixels in the sorted pixel order
};

// one CTA-sized run of vertices of one image, for the vertex kernels
struct VTile {
    int inst;
    int v0, v1;             // global vertex range [v0, v1)
    int t_in_inst;          // index of this tile among its image's tiles
};

// one problem (image) of a solve
struct InstDev {
    int64_t voff;           // first vertex (global)
    int V;
    int C;
    int Cp;                 // channels padded: 1, 2 or a multiple of 4 (vector row length)
    int64_t vec_base;       // offset (multiple of 4) of this image's V x Cp block
    int tile0, ntiles;      // its VTiles
    int pc;                 // first (image, channel) scalar slot
    int64_t part_base;      // first tile-partial slot (C x ntiles doubles)
    float lam;
    int64_t N;
    int64_t pix_base;
    const float* t;         // C x N
    const float* c;         // N
    float* x;               // C x N (slice output) or nullptr
    float* yout;            // C x V (caller's copy of y) or nullptr
    const float* yhat;      // C x V (backward: forward solution)
    const float* dx;        // C x N (backward: dL/dx)
    float* dt;              // C x N (backward out)
    float* dc;              // N     (backward out)
};

// padded channel count of a vector row
__host__ __device__ inline int padded_channels(int C) { return C <= 2 ? C : (C + 3) / 4 * 4; }

// CG scalar carried between phases of one (image, channel): delta =
// r^T M^-1 r of iteration `it` in slot it % 2
struct Scal {
    double delta[2];
    double delta0;          // r_0^T M^-1 r_0 (both forms): the stall test's scale
    double gam[2], alp[2];  // single-reduction form: gamma_i and alpha_i by iteration parity
    double alpha;           // finalised scalars (standard form, Jacobi): alpha of the
    float beta;             //   current iteration, beta of the next phase 1
    unsigned done;          // tiles of the image whose partials are stored (first
                            //   channel's entry only; 0 between phases)
};

// FP32-vector safeguard of the CG scalars: a channel whose r^T M^-1 r has
// fallen to 2^-96 of its first value (the preconditioned residual down by
// 2^-48, far below what FP32 vectors resolve) takes alpha = beta = 0 from
// then on.  Without it the recursive FP32 residual keeps shrinking, over
// thousands of iterations, into the subnormal range, where beta overflows
// and 0 * inf turns y into NaN.  Also true for now = 0 (or NaN).
__device__ __forceinline__ bool cg_stalled(double now, double first)
{
    return !(now > first * 0x1p-96);
}

// splat modes
enum SplatMode : int {
    kSplatConfidence = 0,   // weights c, b = S(c o t)
    kSplatRobust = 1,       // weights w(y_v - t) (Geman-McClure), b = S(w o t)
    kSplatBackward = 2,     // weights c for S c, b = S(dL/dx)
};

// ---------------------------------------------------- exact quantiser ---
// k = floor(p / sigma + 1/2) exactly (as rational numbers), computed with
// FP32 operations: an estimate, then one correction step decided by the
// sign of 2p - (2k +- 1) sigma, which one fused multiply-add evaluates with
// a single rounding (sign-exact).  Returns false when k is outside
// [0, kFieldMax] or p is NaN.
__device__ __forceinline__ bool quantise_exact(float p, float sigma, float inv_sigma, int& k)
{
    // estimate: within one of the exact result (|p / sigma| <= 4097, so the
    // two roundings of p * (1 / sigma) + 1/2 move it by far less than 1/2)
    float kf = floorf(__fmaf_rn(p, inv_sigma, 0.5f));
    if (!(kf >= -1.0f && kf <= (float)(kFieldMax + 2))) return false;
    float twop = __fmul_rn(2.0f, p);
    if (__fmaf_rn(-(2.0f * kf + 1.0f), sigma, twop) >= 0.0f) kf += 1.0f;
    else if (__fmaf_rn(-(2.0f * kf - 1.0f), sigma, twop) < 0.0f) kf -= 1.0f;
    if (!(kf >= 0.0f && kf <= (float)kFieldMax)) return false;
    k = (int)kf;
    return true;
}

// ------------------------------------------- double-float accumulation ---
// An unevaluated sum hi + lo of two floats (about 48 significant bits).
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    DF s = df_two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    float h = __fadd_rn(s.hi, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s.hi))};
}

// a + b for a double-float a and a float b
__device__ __forceinline__ DF df_add_f(DF a, float b)
{
    DF s = df_two_sum(a.hi, b);
    float e = __fadd_rn(s.lo, a.lo);
    float h = __fadd_rn(s.hi, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s.hi))};
}

// exact product a * b = hi + lo
__device__ __forceinline__ DF df_mul_exact(float a, float b)
{
    float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ DF df_shfl_down(DF v, int off)
{
    return {__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off)};
}

__device__ __forceinline__ DF df_warp_sum(DF v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = df_add(v, df_shfl_down(v, off));
    return v;
}

__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }

// (hi, lo) renormalised; requires |a| >= |b| or a == 0
__device__ __forceinline__ DF df_fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a * b for a double-float a and a float b (relative error ~2^-44)
__device__ __forceinline__ DF df_mul_f(DF a, float b)
{
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return df_fast_two_sum(p, e);
}

// a * b for double-float a and b
__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

// split an FP64 scalar into a double-float pair
__device__ __forceinline__ DF df_from_double(double x)
{
    float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

// ----------------------------------------------------- launch helpers ---
struct Profiler;

struct DeviceInfo {
    int dev = -1;
    int sms = 0;
    size_t l2 = 0;
};
const DeviceInfo& device_info();

// profiling: returns an id to pass to prof_begin / prof_end.  level 1 =
// one kernel family, level 2 = a region spanning several launches; only the
// level chosen by fbs_profile_enable records.
int prof_family(const char* name, int level = 1);
void prof_begin(int fam, cudaStream_t s);
void prof_end(int fam, cudaStream_t s);
int prof_level();

}  // namespace fbs
