// Device passes that build the bilateral-space pyramid (supplement,
// bilateral-space pyramids) of a grid, level by level.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace fbs {

constexpr unsigned long long kPyrHashEmpty = ~0ull;   // packed keys use 60 bits

// level k -> k + 1 of every image at once.  The hash region of image im
// (a power of two >= 2 x its level-k vertex count) starts at htoff[im].
struct PyrLevelArgs {
    const uint64_t* key;      // [n] level-k keys
    const uint16_t* img;      // [n] image of each level-k vertex
    int64_t n;
    const int64_t* htoff;     // [n_images + 1] hash region offsets
    unsigned long long* hkey; // hash keys (kPyrHashEmpty when free)
    int32_t* hmin;            // smallest level-k index holding each key
    int32_t* slot;            // [n] the hash slot of each vertex's halved key
    uint32_t* flag;           // [n] 1 where the vertex is its key's representative
    uint32_t* id;             // [n] exclusive scan of flag: next-level ids
    int32_t* parent;          // [n] out: next-level id of each vertex's key
    uint64_t* key1;           // out: next-level keys
    uint16_t* img1;           // out: next-level images
    uint32_t* err;
};

cudaError_t pyr_level_insert(const PyrLevelArgs& L, cudaStream_t s);     // hash, flags
cudaError_t pyr_level_finish(const PyrLevelArgs& L, cudaStream_t s);     // parents, next keys
// exclusive scan of n uint32 (tmp: (n + 1023) / 1024 + 1 words); out[n] = total
cudaError_t scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s);
// out[i] = in[idx[i]] for i < m (64-bit indices)
cudaError_t gather_u32(const uint32_t* in, const int64_t* idx, int64_t* out, int m, cudaStream_t s);
// image of each grid vertex from the vertex offsets (n_images + 1)
cudaError_t fill_vimg(const int64_t* voff, int n_images, int64_t V, uint16_t* vimg, cudaStream_t s);
// children lists of the levels >= 1 vertices, ascending: counts, scan,
// scatter, sort (tmp_cnt: 3 (T - off1 + 1) words; tmp_scan: (T - off1) / 1024 + 2)
cudaError_t pyr_children(const int32_t* parent, const int64_t* off_dev, int K, int64_t T, int64_t off1,
                         int32_t* child_off, int32_t* child_idx, uint32_t* tmp_cnt,
                         uint32_t* tmp_scan, cudaStream_t s);
// P(1) level by level, initialisation weights 4^-k / P(1), zero on the
// vertices an image keeps past its own top
cudaError_t pyr_counts(const int32_t* child_off, const int32_t* child_idx, const int64_t* off_host,
                       const int64_t* off_dev, int K, const int64_t* ioffa_dev, const uint8_t* kimg_dev,
                       int n_images, float* cnt, float* cinit, cudaStream_t s);

}  // namespace fbs
