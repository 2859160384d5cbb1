// Read-only view of a grid handle's arrays for translation units other than
// api.cu (which owns struct fbs_grid).
#pragma once

#include "fbs_internal.cuh"

namespace fbs {

struct GridView {
    int n_images;
    int64_t Vtot;
    int64_t max_pixels;
    int nvt;
    int bistoch_iters;
    int precision;             // FBS_VECTORS_*
    int persistent;            // 1: persistent PCG loop allowed
    int force_persistent;      // 1: persistent loop even where per-phase launches are preferred
    int phase_blocks;          // per-phase launch size, x (SMs x resident blocks)
    const ImgDev* img;         // host, n_images
    const int64_t* voff;       // host, n_images + 1
    const int* vt0;            // host, n_images
    const int* nvt_img;        // host, n_images
    const VTile* vt;           // device
    const int32_t* nbr;        // device, 10 rows of nbr_stride entries
    int64_t nbr_stride;
    const uint32_t* nbrp;      // device, packed offsets
    const double* n64;
    const float* nf;           // n in FP32
    const uint32_t* m;
    const uint32_t* pstart;
    const uint32_t* perm;
    const uint32_t* vid;
    uint32_t* err;
};

// Fills *out from g; false if g is null.
bool grid_view(const fbs_grid* g, GridView* out);

}  // namespace fbs
