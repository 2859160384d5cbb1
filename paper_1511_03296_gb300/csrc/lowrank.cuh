// Low-rank reduction of a wide target (supplement, multiple output
// channels): the device passes.  The rank choice itself runs on the host.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace fbs {

constexpr int kLrGramBlocks = 256;     // Gram partial sums per image
constexpr int kLrMaxEntries = 2080;    // C (C + 1) / 2 for C = 64

// one image of a low-rank pass
struct LrImg {
    const float* t;       // C x N targets (planar), or the map's input
    const float* c;       // N confidences (splat only)
    float* out;           // the map's output (Cout x N planar)
    const float* M;       // the map's Cin x Cout matrix (row-major, device)
    int C, Cout;
    int64_t N, pix_base;  // pixels; first pixel in the grid's concatenated order
    int64_t v0, nv;       // the image's grid vertices
    int64_t boff;         // first float of the image's rows of B
};

// B = S(c o t) for every image, vertex-major rows of C floats at boff
// (double-float sums over each vertex's pixels, rounded once).
cudaError_t lr_splat(const LrImg* imgs_dev, int n_images, int64_t Vtot, const int64_t* voff_dev,
                     const uint32_t* pstart, const uint32_t* m, const uint32_t* perm, float* B,
                     cudaStream_t s);
// G = B^T B per image (cmax x cmax blocks, FP64 from exact products and
// double-float sums in a fixed order): kLrGramBlocks partials per image
// (part: n_images x kLrGramBlocks x cmax (cmax + 1) / 2), then reduced.
cudaError_t lr_gram(const LrImg* imgs_dev, int n_images, const float* B, float2* part, double* G,
                    int cmax, cudaStream_t s);
// out = M^T applied per pixel: out[q][i] = sum_c M[c][q] in[c][i]
cudaError_t lr_map(const LrImg* imgs_dev, int n_images, int64_t max_pixels, cudaStream_t s);

}  // namespace fbs
