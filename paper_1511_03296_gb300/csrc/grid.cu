// Grid construction on the GPU: quantised keys, canonical vertex ids, the
// splat map S (pixel -> vertex, plus the pixels of each vertex in sorted
// order), counts m = S 1, the +-1 neighbour tables, and bistochastisation.
//
// Design.  Vertices are ordered by packed key (row cell, column cell, l, u,
// v).  All pixels of one spatial cell (ky, kx) -- the pixels whose rounded
// (row / sigma_xy, col / sigma_xy) equal (ky, kx) -- form a small rectangle,
// and their vertices are contiguous in the canonical order.  One CTA takes a
// run of consecutive cells of one cell row (a "grid tile"), quantises its
// pixels, radix-sorts them in shared memory by a dense (cell, colour) key
// (stable, so equal keys keep pixel order) and de-duplicates them.  A scan over tiles gives every tile its first vertex
// id.  No global hash table and no global sort are needed; every pixel is
// read once per pass with coalesced row segments.
#include "fbs_internal.cuh"

namespace fbs {

namespace {


// -------------------------------------------------------------- sorting ---
// Exclusive block scan of one int per thread; *total receives the block sum.
__device__ int block_exclusive_scan(int v, int* warp_buf, int* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_buf[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < nw ? warp_buf[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, off);
            if (lane >= off) t += y;
        }
        warp_buf[lane] = t;
    }
    __syncthreads();
    int prefix = (w > 0 ? warp_buf[w - 1] : 0) + x - v;
    *total = warp_buf[nw - 1];
    __syncthreads();
    return prefix;
}

// ---------------------------------------------------------- radix sort ---
// Stable LSD radix sort of a tile's pixels, 4 bits per pass, on a dense key
// made of only the bits that vary inside the tile: the cell index and each
// colour field minus its tile minimum, in the significance order of the
// packed vertex key (cell, l, u, v).  The pixels start in pixel order and
// the sort is stable, so equal keys keep their pixel order.  Pixel indices
// (16-bit) are moved, not the keys.
struct DenseKey {
    int wl, wu, wv;          // bit widths of the l, u, v offsets
    int minl, minu, minv;
};

__device__ __forceinline__ int bit_width(uint32_t x) { return x ? 32 - __clz(x) : 0; }

// 16 counters of 16 bits packed in four 64-bit words
__device__ __forceinline__ void packed_add(uint64_t (&c)[4], int d, uint64_t v)
{
    const uint64_t inc = v << (16 * (d & 3));
    const int q = d >> 2;
    c[0] += q == 0 ? inc : 0ull;
    c[1] += q == 1 ? inc : 0ull;
    c[2] += q == 2 ? inc : 0ull;
    c[3] += q == 3 ? inc : 0ull;
}

__device__ __forceinline__ uint32_t packed_get(const uint64_t (&c)[4], int d)
{
    const int q = d >> 2;
    const uint64_t w = q == 0 ? c[0] : q == 1 ? c[1] : q == 2 ? c[2] : c[3];
    return (uint32_t)(w >> (16 * (d & 3))) & 0xffffu;
}

// Exclusive block scan of four packed words per thread (fields never carry:
// every count stays below 2^16); tot receives the block totals.
__device__ void block_scan_packed(const uint64_t (&x)[4], uint64_t (*wbuf)[4],
                                  uint64_t (&ex)[4], uint64_t (&tot)[4])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t in[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        in[k] = x[k];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, in[k], off);
            if (lane >= off) in[k] += y;
        }
        if (lane == 31) wbuf[w][k] = in[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint64_t t = lane < nw ? wbuf[lane][k] : 0ull;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, t, off);
                if (lane >= off) t += y;
            }
            wbuf[lane][k] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        ex[k] = (w > 0 ? wbuf[w - 1][k] : 0ull) + in[k] - x[k];
        tot[k] = wbuf[nw - 1][k];
    }
    __syncthreads();
}

// Sorts ord[0..P) (pixel indices, initially 0..P-1) by key[ord[.]]; tmp is
// scratch of P entries.  Each thread takes a contiguous run of positions.
__device__ void radix_sort_tile(const uint64_t* key, uint16_t* ord, uint16_t* tmp, int P,
                                int nbits, uint64_t (*wbuf)[4], uint32_t* base)
{
    const int E = (P + (int)blockDim.x - 1) / (int)blockDim.x;
    const int p0 = (int)threadIdx.x * E, p1 = min(p0 + E, P);
    uint16_t* a = ord;
    uint16_t* b = tmp;
    for (int sh = 0; sh < nbits; sh += 4) {
        uint64_t c[4] = {0ull, 0ull, 0ull, 0ull};
        for (int p = p0; p < p1; ++p) packed_add(c, (int)(key[a[p]] >> sh) & 15, 1ull);
        uint64_t ex[4], tot[4];
        block_scan_packed(c, wbuf, ex, tot);
        if (threadIdx.x == 0) {
            uint32_t acc = 0;
            for (int d = 0; d < 16; ++d) {
                base[d] = acc;
                acc += packed_get(tot, d);
            }
        }
        __syncthreads();
        for (int p = p0; p < p1; ++p) {
            const uint16_t j = a[p];
            const int d = (int)(key[j] >> sh) & 15;
            b[base[d] + packed_get(ex, d)] = j;
            packed_add(ex, d, 1ull);
        }
        __syncthreads();
        uint16_t* t = a;
        a = b;
        b = t;
    }
    if (a != ord) {
        for (int p = threadIdx.x; p < P; p += blockDim.x) ord[p] = a[p];
        __syncthreads();
    }
}

// x / d for 0 <= x < 2^14 and 1 <= d <= 2^14, from m = floor(2^32 / d) + 1
// (exact in that range; m needs 33 bits for d = 1)
__device__ __forceinline__ int div_small(int x, uint64_t m) { return (int)(((uint64_t)x * m) >> 32); }

// Quantise the pixels of one tile: key[i] = cell index in tile << 36 |
// l << 24 | u << 12 | v for tile pixel i (row-major in the tile rectangle);
// also the block minima and maxima of l, u, v into mm[0..5].
__device__ void quantise_tile(const GTile& t, const ImgDev& im, uint64_t* key, int P,
                              uint32_t* err, int* mm)
{
    const int tw = t.x1 - t.x0;
    const int64_t plane = (int64_t)im.H * im.W;
    int lo[3] = {4096, 4096, 4096}, hi[3] = {-1, -1, -1};
    // pixel i = r tw + cl, advanced by blockDim.x without division
    const int step = (int)blockDim.x;
    const int dq = step / tw, dr = step - dq * tw;
    int r = (int)threadIdx.x / tw, cl = (int)threadIdx.x - r * tw;
    for (int i = threadIdx.x; i < P; i += step) {
        const int y = t.y0 + r, x = t.x0 + cl;
        const int64_t pix = (int64_t)y * im.W + x;
        const float L = __ldg(im.yuv + pix), U = __ldg(im.yuv + plane + pix),
                    Vv = __ldg(im.yuv + 2 * plane + pix);
        int kx = 0, ky = 0, kl = 0, ku = 0, kv = 0;
        const bool okg = quantise_exact((float)x, im.sxy, im.isxy, kx) &
                         quantise_exact((float)y, im.sxy, im.isxy, ky);
        const bool okc = quantise_exact(L, im.sl, im.isl, kl) &
                         quantise_exact(U, im.suv, im.isuv, ku) &
                         quantise_exact(Vv, im.suv, im.isuv, kv);
        if (!okc) {
            atomicOr(err, kErrRange);
            kl = ku = kv = 0;
        }
        if (!okg || ky != t.ky || kx < t.kx0 || kx >= t.kx0 + t.nkx) {
            atomicOr(err, kErrGeometry);
            kx = t.kx0;
        }
        lo[0] = min(lo[0], kl); hi[0] = max(hi[0], kl);
        lo[1] = min(lo[1], ku); hi[1] = max(hi[1], ku);
        lo[2] = min(lo[2], kv); hi[2] = max(hi[2], kv);
        key[i] = ((uint64_t)(kx - t.kx0) << 36) | ((uint64_t)kl << 24) | ((uint64_t)ku << 12) |
                 (uint64_t)kv;
        cl += dr;
        r += dq;
        if (cl >= tw) {
            cl -= tw;
            ++r;
        }
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            lo[f] = min(lo[f], __shfl_xor_sync(0xffffffffu, lo[f], off));
            hi[f] = max(hi[f], __shfl_xor_sync(0xffffffffu, hi[f], off));
        }
    }
    if (threadIdx.x == 0)
        for (int f = 0; f < 3; ++f) {
            mm[f] = 4096;
            mm[3 + f] = -1;
        }
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
        for (int f = 0; f < 3; ++f) {
            atomicMin(&mm[f], lo[f]);
            atomicMax(&mm[3 + f], hi[f]);
        }
    __syncthreads();
}

// ------------------------------------------------------------- kernels ---
// Pass 1: sort and de-duplicate each tile once.  Writes everything that does
// not depend on the tile's first vertex id:
//   perm[sort_off + i]   = global pixel of sorted item i
//   vid[pixel]           = tile-local vertex rank of the pixel
//   tkey/tm/tps[sort_off + r] = key, count and first sorted slot of local vertex r
//   cell_voff[cell]      = tile-local first vertex of the cell, cell_nv = its count
//   tile_nv[tile]        = number of distinct keys in the tile
// CTA size of the tile sort (measured: 256 beats 128 and 512 -- fewer warps
// per barrier than 512, enough threads per tile for the passes); 8 resident
// CTAs per SM (32 registers; measured 3.5 % faster than 6 on a 64-image batch)
constexpr int kSortThreads = 256;

__global__ void __launch_bounds__(kSortThreads, 8)
grid_sort_kernel(const GTile* __restrict__ tiles, const ImgDev* __restrict__ imgs,
                 int* __restrict__ tile_nv, uint32_t* err, int P2, int max_cells,
                 uint32_t* __restrict__ vid, uint32_t* __restrict__ perm,
                 uint64_t* __restrict__ tkey, uint32_t* __restrict__ tm,
                 uint32_t* __restrict__ tps, uint32_t* __restrict__ cell_voff,
                 uint32_t* __restrict__ cell_nv)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* key = reinterpret_cast<uint64_t*>(smem_raw);
    uint16_t* ord = reinterpret_cast<uint16_t*>(key + P2);     // sorted position -> pixel
    uint16_t* tmp = ord + P2;                                   // radix scratch, then head positions
    int* cellcnt = reinterpret_cast<int*>(tmp + P2);
    __shared__ int warp_buf[32];
    __shared__ uint64_t wbuf[32][4];
    __shared__ uint32_t base[16];
    __shared__ int mm[6];

    const GTile t = tiles[blockIdx.x];
    const ImgDev im = imgs[t.img];
    const int tw = t.x1 - t.x0;
    const int P = (t.y1 - t.y0) * tw;
    const uint64_t mtw = (1ull << 32) / (uint64_t)tw + 1;

    for (int c = threadIdx.x; c < t.nkx && c < max_cells; c += blockDim.x) cellcnt[c] = 0;
    for (int i = threadIdx.x; i < P; i += blockDim.x) ord[i] = (uint16_t)i;
    quantise_tile(t, im, key, P, err, mm);      // ends with a barrier

    // dense keys in place (each thread rewrites the keys it wrote)
    DenseKey dk;
    dk.minl = mm[0];
    dk.minu = mm[1];
    dk.minv = mm[2];
    dk.wl = bit_width((uint32_t)max(mm[3] - mm[0], 0));
    dk.wu = bit_width((uint32_t)max(mm[4] - mm[1], 0));
    dk.wv = bit_width((uint32_t)max(mm[5] - mm[2], 0));
    const int wuv = dk.wu + dk.wv, wluv = dk.wl + wuv;
    const int nbits = bit_width((uint32_t)max(t.nkx - 1, 0)) + wluv;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const uint64_t it = key[i];
        const uint64_t cell = it >> 36;
        const uint64_t l = ((it >> 24) & 0xfff) - dk.minl, u = ((it >> 12) & 0xfff) - dk.minu,
                       v = (it & 0xfff) - dk.minv;
        key[i] = (cell << wluv) | (l << wuv) | (u << dk.wv) | v;
    }
    __syncthreads();
    radix_sort_tile(key, ord, tmp, P, nbits, wbuf, base);
    uint16_t* headpos = tmp;

    // each thread owns a contiguous chunk of the sorted items
    const int E = (P + (int)blockDim.x - 1) / (int)blockDim.x;
    const int i0 = threadIdx.x * E, i1 = min(i0 + E, P);
    int cnt = 0;
    for (int i = i0; i < i1; ++i) cnt += (i == 0 || key[ord[i]] != key[ord[i - 1]]) ? 1 : 0;
    int nv;
    int run = block_exclusive_scan(cnt, warp_buf, &nv);
    const uint64_t mwl = (1ull << dk.wl) - 1, mwu = (1ull << dk.wu) - 1, mwv = (1ull << dk.wv) - 1;
    for (int i = i0; i < i1; ++i) {
        const int pl = ord[i];
        const uint64_t k = key[pl];
        const bool head = i == 0 || k != key[ord[i - 1]];
        if (head) ++run;
        const int rank = run - 1;
        const int r = div_small(pl, mtw);
        const int64_t gpix = im.pix_base + (int64_t)(t.y0 + r) * im.W + (t.x0 + pl - r * tw);
        vid[gpix] = (uint32_t)rank;
        perm[t.sort_off + i] = (uint32_t)gpix;
        if (head) {
            const int cell = (int)(k >> wluv);
            const uint64_t l = ((k >> wuv) & mwl) + dk.minl, u = ((k >> dk.wv) & mwu) + dk.minu,
                           v = (k & mwv) + dk.minv;
            tkey[t.sort_off + rank] = ((uint64_t)t.ky << 48) | ((uint64_t)(t.kx0 + cell) << 36) |
                                      (l << 24) | (u << 12) | v;
            tps[t.sort_off + rank] = (uint32_t)(t.sort_off + i);
            headpos[rank] = (uint16_t)i;
            atomicAdd(&cellcnt[cell], 1);
        }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nv; r += blockDim.x)
        tm[t.sort_off + r] = (uint32_t)((r + 1 < nv ? (int)headpos[r + 1] : P) - (int)headpos[r]);
    if (threadIdx.x == 0) tile_nv[blockIdx.x] = nv;
    // per-cell vertex ranges, tile-local (cells of a tile are consecutive in key order)
    const int64_t cell0 = im.cell_base + (int64_t)t.ky * im.ncx + t.kx0;
    int carry = 0;
    for (int base_c = 0; base_c < t.nkx; base_c += blockDim.x) {
        int c = base_c + threadIdx.x;
        int v = c < t.nkx ? cellcnt[c] : 0;
        int tot;
        int ex = block_exclusive_scan(v, warp_buf, &tot);
        if (c < t.nkx) {
            cell_voff[cell0 + c] = (uint32_t)(carry + ex);
            cell_nv[cell0 + c] = (uint32_t)v;
        }
        carry += tot;
    }
}

// Exclusive scan of the per-tile counts (one CTA; the tile count is small).
__global__ void __launch_bounds__(1024) scan_tiles_kernel(const int* __restrict__ tile_nv,
                                                          int64_t* __restrict__ tile_voff,
                                                          int ntiles)
{
    __shared__ int warp_buf[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < ntiles; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = i < ntiles ? tile_nv[i] : 0;
        int total;
        int ex = block_exclusive_scan(v, warp_buf, &total);
        if (i < ntiles) tile_voff[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) tile_voff[ntiles] = carry;
}

// Pass 2: add each tile's first vertex id and move its vertex records to
// their canonical places.
__global__ void __launch_bounds__(256)
grid_finalize_kernel(const GTile* __restrict__ tiles, const ImgDev* __restrict__ imgs,
                     const int64_t* __restrict__ tile_voff, uint32_t* __restrict__ vid,
                     const uint64_t* __restrict__ tkey, const uint32_t* __restrict__ tm,
                     const uint32_t* __restrict__ tps, uint64_t* __restrict__ vkey,
                     uint32_t* __restrict__ m, uint32_t* __restrict__ pstart,
                     uint32_t* __restrict__ cell_voff)
{
    const GTile t = tiles[blockIdx.x];
    const ImgDev im = imgs[t.img];
    const int64_t v0 = tile_voff[blockIdx.x];
    const int nv = (int)(tile_voff[blockIdx.x + 1] - v0);
    const int tw = t.x1 - t.x0;
    const int P = (t.y1 - t.y0) * tw;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int r = i / tw;
        const int64_t gpix = im.pix_base + (int64_t)(t.y0 + r) * im.W + (t.x0 + i - r * tw);
        vid[gpix] += (uint32_t)v0;
    }
    for (int r = threadIdx.x; r < nv; r += blockDim.x) {
        vkey[v0 + r] = tkey[t.sort_off + r];
        m[v0 + r] = tm[t.sort_off + r];
        pstart[v0 + r] = tps[t.sort_off + r];
    }
    const int64_t cell0 = im.cell_base + (int64_t)t.ky * im.ncx + t.kx0;
    for (int c = threadIdx.x; c < t.nkx; c += blockDim.x) cell_voff[cell0 + c] += (uint32_t)v0;
}

__device__ __forceinline__ int find_in_cell(const uint64_t* __restrict__ vkey, uint32_t lo,
                                            uint32_t n, uint64_t key)
{
    uint32_t a = lo, b = lo + n;   // search [a, b)
    while (a < b) {
        uint32_t mid = a + ((b - a) >> 1);
        uint64_t k = vkey[mid];
        if (k < key) a = mid + 1; else b = mid;
    }
    return (a < lo + n && vkey[a] == key) ? (int)a : -1;
}

// +-1 neighbours along x, y, l, u, v of every vertex of a grid tile.
__global__ void __launch_bounds__(256)
grid_neighbours_kernel(const GTile* __restrict__ tiles, const ImgDev* __restrict__ imgs,
                       const int64_t* __restrict__ tile_voff, const uint64_t* __restrict__ vkey,
                       const uint32_t* __restrict__ cell_voff, const uint32_t* __restrict__ cell_nv,
                       int32_t* __restrict__ nbr, int64_t nstride)
{
    const GTile t = tiles[blockIdx.x];
    const ImgDev im = imgs[t.img];
    const int64_t v0 = tile_voff[blockIdx.x], v1 = tile_voff[blockIdx.x + 1];
    for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        const uint64_t key = vkey[v];
        const int kx = (int)((key >> 36) & kFieldMax), ky = (int)((key >> 48) & kFieldMax);
        const int64_t cell = im.cell_base + (int64_t)ky * im.ncx + kx;
#pragma unroll
        for (int d = 0; d < 5; ++d) {
            const int f = (int)((key >> key_shift(d)) & kFieldMax);
            const uint64_t unit = 1ull << key_shift(d);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                int found = -1;
                const bool ok = s == 0 ? f > 0 : f < kFieldMax;
                int64_t c = cell;
                bool in_grid = true;
                if (d == 0) {
                    const int nx = kx + (s ? 1 : -1);
                    in_grid = nx >= 0 && nx < im.ncx;
                    c = cell + (s ? 1 : -1);
                } else if (d == 1) {
                    const int ny = ky + (s ? 1 : -1);
                    in_grid = ny >= 0 && ny < im.ncy;
                    c = cell + (s ? im.ncx : -im.ncx);
                }
                if (ok && in_grid) {
                    const uint64_t target = s ? key + unit : key - unit;
                    found = find_in_cell(vkey, cell_voff[c], cell_nv[c], target);
                }
                nbr[(int64_t)(2 * d + s) * nstride + v] = found;
            }
        }
    }
}

// One Jacobi sweep of supplement Alg. 1 in FP64, with the operations in a
// fixed order: Bbar n = 10 n_v + n_u (k = 0..9), then sqrt(n_v m_v / Bbar n).
__global__ void __launch_bounds__(256)
bistoch_kernel(const double* __restrict__ nold, double* __restrict__ nnew,
               float* __restrict__ nf, const uint32_t* __restrict__ m,
               const int32_t* __restrict__ nbr, int64_t nstride, int64_t V, int first, int last)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V;
         v += (int64_t)gridDim.x * blockDim.x) {
        const double nv = first ? 1.0 : nold[v];
        double bn = __dmul_rn(10.0, nv);
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            const int32_t u = nbr[(int64_t)k * nstride + v];
            if (u >= 0) bn = __dadd_rn(bn, first ? 1.0 : nold[u]);
        }
        const double r = __dsqrt_rn(__ddiv_rn(__dmul_rn(nv, (double)m[v]), bn));
        nnew[v] = r;
        if (last) nf[v] = (float)r;
    }
}

}  // namespace

// Packed neighbour table: three 32-bit words per vertex (rows of V words)
// holding the ten neighbours as signed offsets from the vertex.  Spatial
// order keeps them small: l, u, v neighbours share the cell and x neighbours
// are in the next cell (8-bit offsets), y neighbours one cell row away
// (16-bit).  Word 0: x-, x+, l-, l+ (bytes 0..3); word 1: u-, u+, v-, v+;
// word 2: y- (low half), y+ (high half).  An absent neighbour is offset 0
// (the vertex itself, whose Laplacian term is exactly 0); an offset out of
// range is the escape value (-128, or -32768 for y): read the 32-bit table.
__device__ __forceinline__ uint32_t pack8(int64_t off)
{
    const int32_t h = (off >= -kNbrOffMax8 && off <= kNbrOffMax8) ? (int32_t)off : kNbrEscape8;
    return (uint32_t)h & 0xffu;
}

__device__ __forceinline__ uint32_t pack16(int64_t off)
{
    const int32_t h = (off >= -kNbrOffMax && off <= kNbrOffMax) ? (int32_t)off : kNbrEscape;
    return (uint32_t)h & 0xffffu;
}

__global__ void __launch_bounds__(256)
pack_neighbours_kernel(const int32_t* __restrict__ nbr, int64_t nstride, uint32_t* __restrict__ nbrp,
                       int64_t V)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V;
         v += (int64_t)gridDim.x * blockDim.x) {
        int64_t off[10];
#pragma unroll
        for (int j = 0; j < 10; ++j) {
            const int32_t u = nbr[(int64_t)j * nstride + v];
            off[j] = u >= 0 ? (int64_t)u - v : 0;
        }
        // neighbour j = 2 d + s: d = 0 x, 1 y, 2 l, 3 u, 4 v; s = 0 (-1), 1 (+1)
        nbrp[v] = pack8(off[0]) | pack8(off[1]) << 8 | pack8(off[4]) << 16 | pack8(off[5]) << 24;
        nbrp[V + v] = pack8(off[6]) | pack8(off[7]) << 8 | pack8(off[8]) << 16 |
                      pack8(off[9]) << 24;
        nbrp[2 * V + v] = pack16(off[2]) | pack16(off[3]) << 16;
    }
}

// ------------------------------------------------------ host launchers ---
size_t grid_smem_sort(int P2, int max_cells)
{
    return (size_t)P2 * (sizeof(uint64_t) + 2 * sizeof(uint16_t)) + (size_t)max_cells * sizeof(int);
}

cudaError_t launch_grid_sort(const GTile* tiles, int ntiles, const ImgDev* imgs, int* tile_nv,
                             uint32_t* err, int P2, int max_cells, uint32_t* vid, uint32_t* perm,
                             uint64_t* tkey, uint32_t* tm, uint32_t* tps, uint32_t* cell_voff,
                             uint32_t* cell_nv, cudaStream_t s)
{
    size_t smem = grid_smem_sort(P2, max_cells);
    cudaError_t e = cudaFuncSetAttribute(grid_sort_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    static int fam = prof_family("grid_sort");
    prof_begin(fam, s);
    grid_sort_kernel<<<ntiles, kSortThreads, smem, s>>>(tiles, imgs, tile_nv, err, P2, max_cells,
                                                        vid, perm, tkey, tm, tps, cell_voff,
                                                        cell_nv);
    prof_end(fam, s);
    return cudaGetLastError();
}

cudaError_t launch_scan_tiles(const int* tile_nv, int64_t* tile_voff, int ntiles, cudaStream_t s)
{
    static int fam = prof_family("scan_tiles");
    prof_begin(fam, s);
    scan_tiles_kernel<<<1, 1024, 0, s>>>(tile_nv, tile_voff, ntiles);
    prof_end(fam, s);
    return cudaGetLastError();
}

cudaError_t launch_grid_finalize(const GTile* tiles, int ntiles, const ImgDev* imgs,
                                 const int64_t* tile_voff, uint32_t* vid, const uint64_t* tkey,
                                 const uint32_t* tm, const uint32_t* tps, uint64_t* vkey,
                                 uint32_t* m, uint32_t* pstart, uint32_t* cell_voff,
                                 cudaStream_t s)
{
    static int fam = prof_family("grid_finalize");
    prof_begin(fam, s);
    grid_finalize_kernel<<<ntiles, 256, 0, s>>>(tiles, imgs, tile_voff, vid, tkey, tm, tps, vkey,
                                                m, pstart, cell_voff);
    prof_end(fam, s);
    return cudaGetLastError();
}

cudaError_t launch_grid_neighbours(const GTile* tiles, int ntiles, const ImgDev* imgs,
                                   const int64_t* tile_voff, const uint64_t* vkey,
                                   const uint32_t* cell_voff, const uint32_t* cell_nv,
                                   int32_t* nbr, int64_t nstride, cudaStream_t s)
{
    static int fam = prof_family("grid_neighbours");
    prof_begin(fam, s);
    grid_neighbours_kernel<<<ntiles, 256, 0, s>>>(tiles, imgs, tile_voff, vkey, cell_voff, cell_nv,
                                                  nbr, nstride);
    prof_end(fam, s);
    return cudaGetLastError();
}

cudaError_t launch_bistoch(const double* nold, double* nnew, float* nf, const uint32_t* m,
                           const int32_t* nbr, int64_t nstride, int64_t V, int first, int last,
                           cudaStream_t s)
{
    if (V == 0) return cudaSuccess;
    static int fam = prof_family("bistochastize");
    int blocks = (int)std::min<int64_t>((V + 255) / 256, (int64_t)device_info().sms * 8);
    prof_begin(fam, s);
    bistoch_kernel<<<blocks, 256, 0, s>>>(nold, nnew, nf, m, nbr, nstride, V, first, last);
    prof_end(fam, s);
    return cudaGetLastError();
}

cudaError_t launch_pack_neighbours(const int32_t* nbr, int64_t nstride, uint32_t* nbrp, int64_t V,
                                   cudaStream_t s)
{
    if (V == 0) return cudaSuccess;
    static int fam = prof_family("pack_neighbours");
    const int blocks = (int)std::min<int64_t>((V + 255) / 256, (int64_t)device_info().sms * 8);
    prof_begin(fam, s);
    pack_neighbours_kernel<<<blocks, 256, 0, s>>>(nbr, nstride, nbrp, V);
    prof_end(fam, s);
    return cudaGetLastError();
}

}  // namespace fbs
