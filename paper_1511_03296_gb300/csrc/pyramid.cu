// Building the bilateral-space pyramid on the GPU (supplement, bilateral-space
// pyramids): level k + 1 holds the distinct floor-halved keys of level k,
// per image.  Distinct keys are found with a hash table per image region;
// each key's representative is the smallest level-k index that holds it
// (atomicMin: the same whatever the order of the inserts), and a prefix scan
// over the representatives numbers the next level in first-occurrence order
// -- deterministic, with the images' vertices kept contiguous.  Children
// lists are sorted ascending so that every pyramid sum runs in a fixed order.
#include <algorithm>

#include "fbs_internal.cuh"
#include "pyramid.cuh"

namespace fbs {
namespace {

__device__ __forceinline__ uint64_t halve_packed(uint64_t k)
{
    uint64_t out = 0;
#pragma unroll
    for (int d = 0; d < 5; ++d) {
        const int sh = 48 - 12 * d;
        out |= (((k >> sh) & 0xFFFull) >> 1) << sh;
    }
    return out;
}

// Fibonacci hashing (multiply by 2^64 / golden ratio, keep the high bits)
__device__ __forceinline__ uint64_t hash_key(uint64_t k)
{
    k ^= k >> 29;
    return (k * 0x9E3779B97F4A7C15ull) >> 20;
}

__global__ void __launch_bounds__(256)
pyr_insert_kernel(PyrLevelArgs L)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int im = L.img[i];
        const int64_t base = L.htoff[im];
        const uint64_t size = (uint64_t)(L.htoff[im + 1] - base);   // a power of two
        const unsigned long long key = halve_packed(L.key[i]);
        uint64_t h = hash_key(key) & (size - 1);
        int32_t where = -1;
        for (uint64_t probe = 0; probe < size; ++probe) {
            const unsigned long long prev = atomicCAS(L.hkey + base + h, kPyrHashEmpty, key);
            if (prev == kPyrHashEmpty || prev == key) {
                where = (int32_t)(base + h);
                break;
            }
            h = (h + 1) & (size - 1);
        }
        if (where < 0) {                 // cannot happen with size >= 2 n; recorded, not faulted
            atomicOr(L.err, kErrRange);
            L.slot[i] = (int32_t)base;
            continue;
        }
        L.slot[i] = where;
        atomicMin(L.hmin + where, (int32_t)i);
    }
}

__global__ void __launch_bounds__(256)
pyr_flag_kernel(PyrLevelArgs L)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L.n;
         i += (int64_t)gridDim.x * blockDim.x)
        L.flag[i] = L.hmin[L.slot[i]] == (int32_t)i ? 1u : 0u;
}

__global__ void __launch_bounds__(256)
pyr_finish_kernel(PyrLevelArgs L)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t rep = L.hmin[L.slot[i]];
        const uint32_t nid = L.id[rep];
        L.parent[i] = (int32_t)nid;
        if (rep == (int32_t)i) {
            L.key1[nid] = halve_packed(L.key[i]);
            L.img1[nid] = L.img[i];
        }
    }
}

// ---- exclusive scan of uint32, 1024 elements per block ----
constexpr int kScanBlock = 1024;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp, uint32_t& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += o;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += o;
        }
        if (lane < (int)(blockDim.x >> 5)) s_warp[lane] = wi - w;   // exclusive per warp
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    total = s_warp[32];
    const uint32_t r = inc - v + s_warp[warp];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanBlock)
scan_sums_kernel(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ sums)
{
    __shared__ uint32_t s_warp[33];
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    uint32_t total;
    block_excl_scan(i < n ? in[i] : 0u, s_warp, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// one block: exclusive scan of the nb block sums in place, total in sums[nb]
__global__ void __launch_bounds__(kScanBlock)
scan_top_kernel(uint32_t* __restrict__ sums, int64_t nb)
{
    __shared__ uint32_t s_warp[33];
    uint32_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += kScanBlock) {
        const int64_t b = b0 + threadIdx.x;
        const uint32_t v = b < nb ? sums[b] : 0u;
        uint32_t total;
        const uint32_t ex = block_excl_scan(v, s_warp, total);
        if (b < nb) sums[b] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void __launch_bounds__(kScanBlock)
scan_apply_kernel(const uint32_t* __restrict__ in, int64_t n, const uint32_t* __restrict__ sums,
                  uint32_t* __restrict__ out)
{
    __shared__ uint32_t s_warp[33];
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    uint32_t total;
    const uint32_t ex = block_excl_scan(i < n ? in[i] : 0u, s_warp, total);
    if (i < n) out[i] = sums[blockIdx.x] + ex;
    if (i == n) out[n] = sums[blockIdx.x] + ex;    // the total (in[n] read as 0)
}

__global__ void gather_u32_kernel(const uint32_t* __restrict__ in, const int64_t* __restrict__ idx,
                                  int64_t* __restrict__ out, int m)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        out[i] = in[idx[i]];
}

__global__ void __launch_bounds__(256)
fill_vimg_kernel(const int64_t* __restrict__ voff, int n, int64_t V, uint16_t* __restrict__ vimg)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V;
         v += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (voff[mid] <= v) lo = mid;
            else hi = mid - 1;
        }
        vimg[v] = (uint16_t)lo;
    }
}

// level of pyramid vertex g (off: K + 1 offsets)
__device__ __forceinline__ int level_of(const int64_t* off, int K, int64_t g)
{
    int k = 0;
    while (k + 1 < K && g >= off[k + 1]) ++k;
    return k;
}

// children counts of every level >= 1 vertex (vertices of levels 0 .. K-2)
__global__ void __launch_bounds__(256)
child_count_kernel(const int32_t* __restrict__ parent, const int64_t* __restrict__ off, int K,
                   int64_t off1, uint32_t* __restrict__ cnt)
{
    const int64_t n = off[K - 1];
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int k = level_of(off, K, g);
        atomicAdd(cnt + (off[k + 1] + parent[g] - off1), 1u);
    }
}

__global__ void __launch_bounds__(256)
child_scatter_kernel(const int32_t* __restrict__ parent, const int64_t* __restrict__ off, int K,
                     int64_t off1, const uint32_t* __restrict__ start, uint32_t* __restrict__ cursor,
                     int32_t* __restrict__ child_idx)
{
    const int64_t n = off[K - 1];
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int k = level_of(off, K, g);
        const int64_t p = off[k + 1] + parent[g] - off1;
        const uint32_t pos = start[p] + atomicAdd(cursor + p, 1u);
        child_idx[pos] = (int32_t)(g - off[k]);
    }
}

// each children list ascending (at most 32 entries: 2 pre-images per field)
__global__ void __launch_bounds__(256)
child_sort_kernel(const uint32_t* __restrict__ start, int64_t np, int32_t* __restrict__ child_off,
                  int32_t* __restrict__ child_idx)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= np;
         p += (int64_t)gridDim.x * blockDim.x) {
        child_off[p] = (int32_t)start[p];
        if (p == np) continue;
        const uint32_t a = start[p], b = start[p + 1];
        for (uint32_t i = a + 1; i < b; ++i) {
            const int32_t v = child_idx[i];
            uint32_t j = i;
            while (j > a && child_idx[j - 1] > v) {
                child_idx[j] = child_idx[j - 1];
                --j;
            }
            child_idx[j] = v;
        }
    }
}

// P(1) of level k (k >= 1) from level k - 1
__global__ void __launch_bounds__(256)
count_level_kernel(const int32_t* __restrict__ child_off, const int32_t* __restrict__ child_idx,
                   int64_t o_prev, int64_t o_k, int64_t o_next, int64_t off1, float* __restrict__ cnt)
{
    for (int64_t g = o_k + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < o_next;
         g += (int64_t)gridDim.x * blockDim.x) {
        float c = 0.0f;
        for (int32_t j = child_off[g - off1]; j < child_off[g - off1 + 1]; ++j)
            c += cnt[o_prev + child_idx[j]];          // integers below 2^24: exact
        cnt[g] = c;
    }
}

__global__ void __launch_bounds__(256)
cinit_kernel(const int64_t* __restrict__ off, int K, const float* __restrict__ cnt,
             float* __restrict__ cinit)
{
    const int64_t T = off[K];
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < T;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int k = level_of(off, K, g);
        const float w = exp2f(-2.0f * (float)k);       // 4^-k, exact
        cinit[g] = cnt[g] > 0.0f ? __fdiv_rn(w, cnt[g]) : 0.0f;
    }
}

// the single vertex an image keeps past its own top: P(1) = 0, weight 0
__global__ void pad_zero_kernel(const int64_t* __restrict__ ioffa, const uint8_t* __restrict__ kimg,
                                int n, int K, float* __restrict__ cnt, float* __restrict__ cinit)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n * K; q += gridDim.x * blockDim.x) {
        const int im = q % n, k = q / n;
        if (k >= kimg[im]) {
            const int64_t g = ioffa[(int64_t)k * (n + 1) + im];
            cnt[g] = 0.0f;
            cinit[g] = 0.0f;
        }
    }
}

__global__ void __launch_bounds__(256)
fill_one_kernel(float* __restrict__ x, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = 1.0f;
}

int blocks_for(int64_t n, int per_sm)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)device_info().sms * per_sm));
}

}  // namespace

cudaError_t pyr_level_insert(const PyrLevelArgs& L, cudaStream_t s)
{
    pyr_insert_kernel<<<blocks_for(L.n, 8), 256, 0, s>>>(L);
    pyr_flag_kernel<<<blocks_for(L.n, 8), 256, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t pyr_level_finish(const PyrLevelArgs& L, cudaStream_t s)
{
    pyr_finish_kernel<<<blocks_for(L.n, 8), 256, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s)
{
    const int64_t nb = n / kScanBlock + 1;             // the extra block carries out[n]
    scan_sums_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(in, n, tmp);
    scan_top_kernel<<<1, kScanBlock, 0, s>>>(tmp, nb);
    scan_apply_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(in, n, tmp, out);
    return cudaGetLastError();
}

cudaError_t gather_u32(const uint32_t* in, const int64_t* idx, int64_t* out, int m, cudaStream_t s)
{
    gather_u32_kernel<<<std::max(1, std::min((m + 255) / 256, 64)), 256, 0, s>>>(in, idx, out, m);
    return cudaGetLastError();
}

cudaError_t fill_vimg(const int64_t* voff, int n_images, int64_t V, uint16_t* vimg, cudaStream_t s)
{
    fill_vimg_kernel<<<blocks_for(V, 8), 256, 0, s>>>(voff, n_images, V, vimg);
    return cudaGetLastError();
}

cudaError_t pyr_children(const int32_t* parent, const int64_t* off_dev, int K, int64_t T, int64_t off1,
                         int32_t* child_off, int32_t* child_idx, uint32_t* tmp_cnt,
                         uint32_t* tmp_scan, cudaStream_t s)
{
    const int64_t np = T - off1;                       // level >= 1 vertices
    cudaError_t e = cudaMemsetAsync(tmp_cnt, 0, (size_t)(np + 1) * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    child_count_kernel<<<blocks_for(off1 + np, 8), 256, 0, s>>>(parent, off_dev, K, off1, tmp_cnt);
    // start = exclusive scan of the counts (start[np] = total)
    uint32_t* start = tmp_cnt + (np + 1);
    uint32_t* cursor = start + (np + 1);
    if ((e = scan_u32(tmp_cnt, start, np, tmp_scan, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cursor, 0, (size_t)np * sizeof(uint32_t), s)) != cudaSuccess) return e;
    child_scatter_kernel<<<blocks_for(off1 + np, 8), 256, 0, s>>>(parent, off_dev, K, off1, start, cursor,
                                                                 child_idx);
    child_sort_kernel<<<blocks_for(np + 1, 8), 256, 0, s>>>(start, np, child_off, child_idx);
    return cudaGetLastError();
}

cudaError_t pyr_counts(const int32_t* child_off, const int32_t* child_idx, const int64_t* off_host,
                       const int64_t* off_dev, int K, const int64_t* ioffa_dev, const uint8_t* kimg_dev,
                       int n_images, float* cnt, float* cinit, cudaStream_t s)
{
    fill_one_kernel<<<blocks_for(off_host[1], 8), 256, 0, s>>>(cnt, off_host[1]);
    for (int k = 1; k < K; ++k)
        count_level_kernel<<<blocks_for(off_host[k + 1] - off_host[k], 8), 256, 0, s>>>(
            child_off, child_idx, off_host[k - 1], off_host[k], off_host[k + 1], off_host[1], cnt);
    cinit_kernel<<<blocks_for(off_host[K], 8), 256, 0, s>>>(off_dev, K, cnt, cinit);
    pad_zero_kernel<<<std::max(1, std::min((n_images * K + 255) / 256, 64)), 256, 0, s>>>(
        ioffa_dev, kimg_dev, n_images, K, cnt, cinit);
    return cudaGetLastError();
}

}  // namespace fbs
