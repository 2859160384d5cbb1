// C ABI of libfbs (declared in include/fbs.h): grid handles, device memory,
// argument checking, scheduling of the kernels on the caller's stream, and
// per-kernel-family event timing.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fbs_internal.cuh"
#include "lowrank.cuh"
#include "pyramid.cuh"
#include "solve.cuh"

namespace fbs {
// launchers defined in grid.cu
cudaError_t launch_grid_sort(const GTile*, int, const ImgDev*, int*, uint32_t*, int, int,
                             uint32_t*, uint32_t*, uint64_t*, uint32_t*, uint32_t*, uint32_t*,
                             uint32_t*, cudaStream_t);
cudaError_t launch_scan_tiles(const int*, int64_t*, int, cudaStream_t);
cudaError_t launch_grid_finalize(const GTile*, int, const ImgDev*, const int64_t*, uint32_t*,
                                 const uint64_t*, const uint32_t*, const uint32_t*, uint64_t*,
                                 uint32_t*, uint32_t*, uint32_t*, cudaStream_t);
cudaError_t launch_pack_neighbours(const int32_t*, int64_t, uint32_t*, int64_t, cudaStream_t);
cudaError_t launch_grid_neighbours(const GTile*, int, const ImgDev*, const int64_t*,
                                   const uint64_t*, const uint32_t*, const uint32_t*, int32_t*,
                                   int64_t, cudaStream_t);
cudaError_t launch_bistoch(const double*, double*, float*, const uint32_t*, const int32_t*,
                           int64_t, int64_t, int, int, cudaStream_t);

// ----------------------------------------------------------- device info ---
const DeviceInfo& device_info()
{
    static std::mutex mu;
    static std::map<int, DeviceInfo> infos;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = infos.find(dev);
    if (it == infos.end()) {
        DeviceInfo d;
        d.dev = dev;
        cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        int l2 = 0;
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
        d.l2 = (size_t)l2;
        it = infos.emplace(dev, d).first;
    }
    return it->second;
}

// -------------------------------------------------------------- profiler ---
namespace {
struct Family {
    std::string name;
    int level = 1;
    int64_t launches = 0;
    double ms = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    cudaEvent_t open = nullptr;
};
std::mutex g_prof_mu;
std::vector<Family>& families()
{
    static std::vector<Family> f;
    return f;
}
std::vector<cudaEvent_t>& event_pool()
{
    static std::vector<cudaEvent_t> p;
    return p;
}
int g_prof_level = 0;
}  // namespace
int prof_level() { return g_prof_level; }
namespace {

cudaEvent_t take_event()
{
    auto& pool = event_pool();
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

bool capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &st);
    return st != cudaStreamCaptureStatusNone;
}
}  // namespace

int prof_family(const char* name, int level)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    auto& f = families();
    for (size_t i = 0; i < f.size(); ++i)
        if (f[i].name == name) return (int)i;
    Family fam;
    fam.name = name;
    fam.level = level;
    f.push_back(fam);
    return (int)f.size() - 1;
}

void prof_begin(int fam, cudaStream_t s)
{
    if (!g_prof_level) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    Family& f = families()[fam];
    if (f.level != g_prof_level || capturing(s)) return;
    f.open = take_event();
    cudaEventRecord(f.open, s);
}

void prof_end(int fam, cudaStream_t s)
{
    if (!g_prof_level) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    Family& f = families()[fam];
    if (!f.open) return;
    cudaEvent_t e = take_event();
    cudaEventRecord(e, s);
    f.pending.emplace_back(f.open, e);
    f.open = nullptr;
}

// ---------------------------------------------------------- memory pool ---
namespace {
cudaMemPool_t pool_for_current_device()
{
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = pools.find(dev);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    pools[dev] = pool;
    return pool;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count, cudaStream_t s)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaMemPool_t pool = pool_for_current_device();
    if (!pool) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync((void**)p, count * sizeof(T), pool, s);
}

template <typename T>
void dfree(T*& p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
}

// Small host -> device copies through kernel parameters: asynchronous with
// respect to the host buffer and valid inside stream capture.
struct Chunk {
    unsigned char b[3968];
};
__global__ void upload_kernel(unsigned char* dst, Chunk c, int n)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = c.b[i];
}
// Host-to-device copies of host-built tables (image descriptors, sort
// tiles, vertex tiles) through a pinned staging ring: a copy from pageable
// memory first waits for all earlier work on the stream, which would leave
// the GPU idle between a caller's steps while the host prepares the next
// grid.  A region of the ring is reused only after the copy that last read
// it has completed (one event per copy).  Falls back to a plain copy inside
// a stream capture (the ring's contents would be read at replay time) and
// for copies larger than half the ring.
cudaError_t pinned_upload(void* dst, const void* src, size_t bytes, cudaStream_t s)
{
    struct Use {
        size_t lo, hi;
        cudaEvent_t ev;
    };
    static std::mutex mu;
    static unsigned char* ring = nullptr;
    static size_t cap = 0, head = 0;
    static std::deque<Use> inflight;
    if (bytes == 0) return cudaSuccess;
    std::lock_guard<std::mutex> lk(mu);
    if (!ring && cap == 0) {
        cap = (size_t)16 << 20;
        if (cudaMallocHost(&ring, cap) != cudaSuccess) {
            cudaGetLastError();
            ring = nullptr;
            cap = 1;                                // do not try again
        }
    }
    if (!ring || bytes > cap / 2 || capturing(s))
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    size_t lo = (head + 255) & ~(size_t)255;
    if (lo + bytes > cap) lo = 0;
    const size_t hi = lo + bytes;
    cudaError_t e = cudaSuccess;
    for (auto it = inflight.begin(); it != inflight.end();) {
        const bool overlaps = it->lo < hi && lo < it->hi;
        if (overlaps) {
            e = cudaEventSynchronize(it->ev);
            if (e != cudaSuccess) return e;
        }
        if (overlaps || cudaEventQuery(it->ev) == cudaSuccess) {
            cudaEventDestroy(it->ev);
            it = inflight.erase(it);
        } else {
            ++it;
        }
    }
    cudaGetLastError();                             // cudaEventQuery's cudaErrorNotReady
    memcpy(ring + lo, src, bytes);
    if ((e = cudaMemcpyAsync(dst, ring + lo, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    cudaEvent_t ev = nullptr;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ev, s)) != cudaSuccess) {
        cudaEventSynchronize(ev);
        cudaEventDestroy(ev);
        return e;
    }
    inflight.push_back(Use{lo, hi, ev});
    head = hi;
    return cudaSuccess;
}

// A pinned host buffer of this thread for device-to-host reads that the
// host waits for before the call returns (copies into pageable memory are
// synchronous: they would stop the host before the following launches).
// Grows as needed; an earlier read has completed by the time a call asks
// for it again.
unsigned char* pinned_readback(size_t bytes)
{
    thread_local unsigned char* buf = nullptr;
    thread_local size_t cap = 0;
    if (bytes > cap) {
        if (buf) cudaFreeHost(buf);
        buf = nullptr;
        cap = 0;
        const size_t want = std::max<size_t>(bytes, (size_t)1 << 20);
        if (cudaMallocHost(&buf, want) != cudaSuccess) {
            cudaGetLastError();
            buf = nullptr;
            return nullptr;
        }
        cap = want;
    }
    return buf;
}

cudaError_t upload(void* dst, const void* src, size_t bytes, cudaStream_t s)
{
    static int fam = prof_family("upload");
    const unsigned char* p = (const unsigned char*)src;
    for (size_t off = 0; off < bytes; off += sizeof(Chunk)) {
        Chunk c;
        size_t n = std::min(bytes - off, sizeof(Chunk));
        memcpy(c.b, p + off, n);
        prof_begin(fam, s);
        upload_kernel<<<1, 256, 0, s>>>((unsigned char*)dst + off, c, (int)n);
        prof_end(fam, s);
    }
    return cudaGetLastError();
}

fbs_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return FBS_OK;
    if (e == cudaErrorMemoryAllocation) return FBS_ERR_OOM;
    return FBS_ERR_CUDA;
}

// floor(p / sigma + 1/2) in FP64 (exact for these operands; see the device
// quantiser)
int round_half_up(double p, double sigma) { return (int)floor(p / sigma + 0.5); }

int64_t next_pow2(int64_t x)
{
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}
}  // namespace
}  // namespace fbs

namespace fbs {
cudaError_t domain_transform(const float* guide, int H, int W, float* x, int C, float sigma_s,
                             float sigma_r, int iters, float* dh, float* dv, cudaStream_t s);
int domain_transform_max_width();
}  // namespace fbs

using namespace fbs;

// -------------------------------------------------------------- handle ----
struct fbs_grid {
    int dev = 0;
    int n_images = 0;
    std::vector<ImgDev> img;            // host copy (yuv pointer not kept)
    std::vector<int64_t> voff;          // n_images + 1
    std::vector<int> vt0, nvt_img;      // VTiles per image
    int64_t Ntot = 0, Vtot = 0, ncells = 0;
    int64_t max_pixels = 0;
    // device arrays
    uint64_t* vkey = nullptr;
    uint32_t* vid = nullptr;
    uint32_t* perm = nullptr;
    uint32_t* pstart = nullptr;
    uint32_t* m = nullptr;
    int32_t* nbr = nullptr;
    int64_t nbr_stride = 0;    // entries between the 10 rows of nbr (its vertex capacity)
    cudaEvent_t ev_counts = nullptr;   // the grid build's vertex counts have reached the host
    uint32_t* nbrp = nullptr;           // kNbrWords x Vtot packed neighbour offsets
    double* n64 = nullptr;
    double* n64b = nullptr;
    float* nf = nullptr;
    uint32_t* cell_voff = nullptr;
    uint32_t* cell_nv = nullptr;
    uint32_t* err = nullptr;
    VTile* vt = nullptr;
    int nvt = 0;
    GTile* gt = nullptr;                // grid tiles, kept for the splat
    int64_t* gt_voff = nullptr;
    int ngt = 0;
    int gt_p2 = 0;
    int bistoch_iters = 0;
    // solve workspace
    size_t cap_vec = 0;                 // floats per vector
    float* vec = nullptr;               // 8 x cap_vec: y, r, r_lo, d0, d1, q, s0, s1
    int precision = FBS_VECTORS_AUTO;
    int persistent = 1;
    int force_persistent = 0;
    int pcg_form = FBS_PCG_FORM_STANDARD;
    int phase_blocks = 1;
    int tune_single = 0;       // fbs_autotune times first solves (graphs dropped)
    int precond = FBS_PRECOND_JACOBI;
    // bilateral-space pyramid (built on the first hierarchical solve)
    int pyr_K = 0;
    int64_t pyr_off[kMaxLevels + 1] = {0};
    int32_t* pyr_parent = nullptr;
    int32_t* pyr_child_off = nullptr;
    int32_t* pyr_child_idx = nullptr;
    uint16_t* pyr_vimg = nullptr;
    int64_t* pyr_ioff = nullptr;
    uint8_t* pyr_kimg = nullptr;
    uint64_t* pyr_key = nullptr;        // packed keys of every pyramid vertex (for export)
    std::vector<int64_t> pyr_ioff_host; // K x (n_images + 1), absolute
    float* pyr_cnt = nullptr;
    float* pyr_cinit = nullptr;
    float* pyr_coef = nullptr;
    float* pyr_dg = nullptr;
    float* pyr_scv = nullptr;
    float2* pyr_lv = nullptr;
    int pyr_lv_nc = 0;                  // level-vector values per vertex pyr_lv holds
    int inject_timeout = 0;
    float* a = nullptr;
    float* alo = nullptr;      // low part of a' (robust solver, compensated precision)
    float2* nm = nullptr;
    size_t cap_scal = 0, cap_part = 0;
    Scal* scal = nullptr;
    float2* part = nullptr;             // 3 x cap_part: rs slot 0, rs slot 1, dq
    unsigned* barrier = nullptr;        // grid-barrier words of the persistent PCG loop
    InstDev* inst = nullptr;
    std::vector<InstDev> inst_cached;
    // CUDA graphs of the solve segments, keyed by the exact launch arguments
    struct GraphEntry {
        SolveArgs A;
        SolvePlan P;
        int seg, mode;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;
    cudaStream_t cap_stream = nullptr;
};

namespace {

void free_graphs(fbs_grid* g)
{
    for (auto& e : g->graphs)
        if (e.exec) cudaGraphExecDestroy(e.exec);
    g->graphs.clear();
}

void free_grid_memory(fbs_grid* g, cudaStream_t s)
{
    free_graphs(g);
    if (g->cap_stream) {
        cudaStreamDestroy(g->cap_stream);
        g->cap_stream = nullptr;
    }
    if (g->ev_counts) {
        cudaEventDestroy(g->ev_counts);
        g->ev_counts = nullptr;
    }
    dfree(g->vkey, s); dfree(g->vid, s); dfree(g->perm, s); dfree(g->pstart, s);
    dfree(g->m, s); dfree(g->nbr, s); dfree(g->nbrp, s); dfree(g->n64, s); dfree(g->n64b, s); dfree(g->nf, s);
    dfree(g->cell_voff, s); dfree(g->cell_nv, s); dfree(g->err, s); dfree(g->vt, s);
    dfree(g->gt, s); dfree(g->gt_voff, s);
    dfree(g->vec, s); dfree(g->a, s); dfree(g->alo, s); dfree(g->nm, s); dfree(g->scal, s);
    dfree(g->part, s);
    dfree(g->inst, s); dfree(g->barrier, s);
    dfree(g->pyr_parent, s); dfree(g->pyr_child_off, s); dfree(g->pyr_child_idx, s);
    dfree(g->pyr_vimg, s); dfree(g->pyr_ioff, s); dfree(g->pyr_kimg, s); dfree(g->pyr_key, s);
    dfree(g->pyr_cnt, s);
    dfree(g->pyr_cinit, s); dfree(g->pyr_coef, s); dfree(g->pyr_dg, s); dfree(g->pyr_scv, s);
    dfree(g->pyr_lv, s);
}

fbs_status latched(uint32_t bits)
{
    if (bits & kErrRange) return FBS_ERR_RANGE;
    if (bits & kErrNonFinite) return FBS_ERR_NONFINITE;
    if (bits & kErrTimeout) return FBS_ERR_TIMEOUT;
    if (bits & kErrGeometry) return FBS_ERR_STATE;
    return FBS_OK;
}

}  // namespace

extern "C" {

const char* fbs_status_string(fbs_status s)
{
    switch (s) {
        case FBS_OK: return "ok";
        case FBS_ERR_ARG: return "invalid argument";
        case FBS_ERR_RANGE: return "quantised key field out of range [0, 4095]";
        case FBS_ERR_OOM: return "device out of memory";
        case FBS_ERR_CUDA: return "CUDA runtime error";
        case FBS_ERR_TIMEOUT: return "bounded device wait timed out";
        case FBS_ERR_NONFINITE: return "non-finite target or confidence";
        case FBS_ERR_STATE: return "call out of order or internal inconsistency";
    }
    return "unknown status";
}

fbs_status fbs_grid_build(const fbs_image_desc* imgs, int n_images, void* stream, fbs_grid** out)
{
    if (!out) return FBS_ERR_ARG;
    *out = nullptr;
    // image ids are 16-bit in the pyramid and index grid.y of per-image launches
    if (!imgs || n_images < 1 || n_images > 65535) return FBS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;

    // ---- host geometry: cells, cell-row / cell-column pixel ranges, tiles
    std::vector<ImgDev> img(n_images);
    std::vector<GTile> tiles;
    int64_t pix = 0, cells = 0, sorted = 0;
    int max_P = 0, max_cells = 1;
    const int target = 2048;
    for (int k = 0; k < n_images; ++k) {
        const fbs_image_desc& d = imgs[k];
        if (!d.yuv || d.height <= 0 || d.width <= 0) return FBS_ERR_ARG;
        if (!(d.sigma_xy > 0.f) || !(d.sigma_l > 0.f) || !(d.sigma_uv > 0.f) ||
            !isfinite(d.sigma_xy) || !isfinite(d.sigma_l) || !isfinite(d.sigma_uv))
            return FBS_ERR_ARG;
        const int kx_max = round_half_up(d.width - 1, d.sigma_xy);
        const int ky_max = round_half_up(d.height - 1, d.sigma_xy);
        if (kx_max > kFieldMax || ky_max > kFieldMax) return FBS_ERR_RANGE;
        ImgDev& im = img[k];
        im.yuv = d.yuv;
        im.H = d.height;
        im.W = d.width;
        im.sxy = d.sigma_xy;
        im.sl = d.sigma_l;
        im.suv = d.sigma_uv;
        im.isxy = 1.0f / d.sigma_xy;
        im.isl = 1.0f / d.sigma_l;
        im.isuv = 1.0f / d.sigma_uv;
        im.ncx = kx_max + 1;
        im.ncy = ky_max + 1;
        im.pix_base = pix;
        im.cell_base = cells;
        // first pixel column / row of each cell (monotone rounding)
        std::vector<int> xlo(im.ncx + 1, im.W), ylo(im.ncy + 1, im.H);
        for (int x = im.W - 1; x >= 0; --x) xlo[round_half_up(x, d.sigma_xy)] = x;
        for (int k2 = im.ncx - 1; k2 >= 0; --k2) xlo[k2] = std::min(xlo[k2], xlo[k2 + 1]);
        for (int y = im.H - 1; y >= 0; --y) ylo[round_half_up(y, d.sigma_xy)] = y;
        for (int k2 = im.ncy - 1; k2 >= 0; --k2) ylo[k2] = std::min(ylo[k2], ylo[k2 + 1]);
        for (int ky = 0; ky < im.ncy; ++ky) {
            const int rows = ylo[ky + 1] - ylo[ky];
            int kx = 0;
            while (kx < im.ncx) {
                const int kx0 = kx;
                int cols = 0;
                while (kx < im.ncx) {
                    const int c = xlo[kx + 1] - xlo[kx];
                    if (kx > kx0 && ((int64_t)(cols + c) * rows > target || kx - kx0 >= 4096))
                        break;
                    cols += c;
                    ++kx;
                }
                const int P = rows * cols;
                if (P > kMaxTilePixels) return FBS_ERR_ARG;   // one cell too large
                GTile t;
                t.img = k;
                t.ky = ky;
                t.kx0 = kx0;
                t.nkx = kx - kx0;
                t.y0 = ylo[ky];
                t.y1 = ylo[ky + 1];
                t.x0 = xlo[kx0];
                t.x1 = xlo[kx];
                t.sort_off = sorted;
                sorted += P;
                max_P = std::max(max_P, P);
                max_cells = std::max(max_cells, t.nkx);
                tiles.push_back(t);
            }
        }
        pix += (int64_t)im.H * im.W;
        cells += (int64_t)im.ncx * im.ncy;
    }
    if (pix >= (int64_t)0xFFFFFFFFll || pix > INT32_MAX) return FBS_ERR_ARG;
    const int ntiles = (int)tiles.size();
    const int P2 = (int)std::max<int64_t>(1024, next_pow2(max_P));

    static int f_region = prof_family("region:grid_build", 2);
    prof_begin(f_region, s);
    fbs_grid* g = new fbs_grid();
    cudaGetDevice(&g->dev);
    g->n_images = n_images;
    g->img = img;
    g->Ntot = pix;
    g->ncells = cells;
    for (auto& im : img) g->max_pixels = std::max<int64_t>(g->max_pixels, (int64_t)im.H * im.W);

    ImgDev* d_img = nullptr;
    GTile* d_tiles = nullptr;
    int* d_tile_nv = nullptr;
    int64_t* d_tile_voff = nullptr;
    uint64_t* d_tkey = nullptr;
    uint32_t* d_tm = nullptr;
    uint32_t* d_tps = nullptr;
    cudaError_t e = cudaSuccess;
    fbs_status st = FBS_OK;
    std::vector<int64_t> tile_voff(ntiles + 1);
    uint32_t err_bits = 0;
#define FBS_TRY(x)                       \
    do {                                 \
        e = (x);                         \
        if (e != cudaSuccess) goto fail; \
    } while (0)
    FBS_TRY(dalloc(&d_img, img.size(), s));
    FBS_TRY(dalloc(&d_tiles, tiles.size(), s));
    FBS_TRY(dalloc(&d_tile_nv, (size_t)ntiles, s));
    FBS_TRY(dalloc(&d_tile_voff, (size_t)ntiles + 1, s));
    FBS_TRY(dalloc(&d_tkey, (size_t)pix, s));
    FBS_TRY(dalloc(&d_tm, (size_t)pix, s));
    FBS_TRY(dalloc(&d_tps, (size_t)pix, s));
    FBS_TRY(dalloc(&g->err, 1, s));
    FBS_TRY(dalloc(&g->vid, g->Ntot, s));
    FBS_TRY(dalloc(&g->perm, g->Ntot, s));
    FBS_TRY(dalloc(&g->cell_voff, cells, s));
    FBS_TRY(dalloc(&g->cell_nv, cells, s));
    FBS_TRY(cudaMemsetAsync(g->err, 0, sizeof(uint32_t), s));
    FBS_TRY(pinned_upload(d_img, img.data(), img.size() * sizeof(ImgDev), s));
    FBS_TRY(pinned_upload(d_tiles, tiles.data(), tiles.size() * sizeof(GTile), s));
    FBS_TRY(launch_grid_sort(d_tiles, ntiles, d_img, d_tile_nv, g->err, P2, max_cells, g->vid,
                             g->perm, d_tkey, d_tm, d_tps, g->cell_voff, g->cell_nv, s));
    FBS_TRY(launch_scan_tiles(d_tile_nv, d_tile_voff, ntiles, s));
    {
        // The vertex counts come back to the host while the finalize and
        // neighbour passes run: those write arrays sized by the pixel count
        // (V <= N; the sort keeps its counts in range even when it latches an
        // error), and the neighbour table's row stride is that capacity.
        const size_t rb_bytes = (size_t)(ntiles + 1) * sizeof(int64_t) + sizeof(uint32_t);
        unsigned char* rb = pinned_readback(rb_bytes);
        uint32_t* rb_err = nullptr;
        int64_t* rb_voff = nullptr;
        if (rb) {
            rb_voff = reinterpret_cast<int64_t*>(rb);
            rb_err = reinterpret_cast<uint32_t*>(rb + (size_t)(ntiles + 1) * sizeof(int64_t));
            FBS_TRY(cudaMemcpyAsync(rb_voff, d_tile_voff, (ntiles + 1) * sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, s));
            FBS_TRY(cudaMemcpyAsync(rb_err, g->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            if (!g->ev_counts) FBS_TRY(cudaEventCreateWithFlags(&g->ev_counts, cudaEventDisableTiming));
            FBS_TRY(cudaEventRecord(g->ev_counts, s));
        }
        const int64_t Vcap = std::max<int64_t>(pix, 1);
        g->nbr_stride = Vcap;
        FBS_TRY(dalloc(&g->vkey, Vcap, s));
        FBS_TRY(dalloc(&g->pstart, Vcap, s));
        FBS_TRY(dalloc(&g->m, Vcap, s));
        FBS_TRY(launch_grid_finalize(d_tiles, ntiles, d_img, d_tile_voff, g->vid, d_tkey, d_tm,
                                     d_tps, g->vkey, g->m, g->pstart, g->cell_voff, s));
        FBS_TRY(dalloc(&g->nbr, (size_t)Vcap * 10, s));
        FBS_TRY(launch_grid_neighbours(d_tiles, ntiles, d_img, d_tile_voff, g->vkey, g->cell_voff,
                                       g->cell_nv, g->nbr, Vcap, s));
        if (rb) {
            FBS_TRY(cudaEventSynchronize(g->ev_counts));
            std::copy(rb_voff, rb_voff + ntiles + 1, tile_voff.begin());
            err_bits = *rb_err;
        } else {                            // no pinned memory: read synchronously
            FBS_TRY(cudaMemcpyAsync(tile_voff.data(), d_tile_voff, (ntiles + 1) * sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, s));
            FBS_TRY(cudaMemcpyAsync(&err_bits, g->err, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                    s));
            FBS_TRY(cudaStreamSynchronize(s));
        }
    }
    if (err_bits) {
        st = latched(err_bits);
        goto fail_status;
    }
    {
        g->Vtot = tile_voff[ntiles];
        g->voff.assign(n_images + 1, g->Vtot);
        int ti = 0;
        for (int k = 0; k < n_images; ++k) {
            while (ti < ntiles && tiles[ti].img < k) ++ti;
            g->voff[k] = tile_voff[ti];
        }
        const int64_t V = g->Vtot;
        FBS_TRY(dalloc(&g->nbrp, (size_t)V * kNbrWords, s));
        FBS_TRY(launch_pack_neighbours(g->nbr, g->nbr_stride, g->nbrp, V, s));
        FBS_TRY(dalloc(&g->n64, V, s));
        FBS_TRY(dalloc(&g->n64b, V, s));
        FBS_TRY(dalloc(&g->nf, V, s));
        // vertex tiles for the vertex kernels
        std::vector<VTile> vt;
        g->vt0.resize(n_images);
        g->nvt_img.resize(n_images);
        for (int k = 0; k < n_images; ++k) {
            g->vt0[k] = (int)vt.size();
            const int64_t a0 = g->voff[k], a1 = g->voff[k + 1];
            int j = 0;
            for (int64_t v = a0; v < a1; v += kVTile, ++j) {
                VTile t;
                t.inst = k;
                t.v0 = (int)v;
                t.v1 = (int)std::min<int64_t>(v + kVTile, a1);
                t.t_in_inst = j;
                vt.push_back(t);
            }
            g->nvt_img[k] = j;
        }
        g->nvt = (int)vt.size();
        FBS_TRY(dalloc(&g->vt, vt.size(), s));
        FBS_TRY(pinned_upload(g->vt, vt.data(), vt.size() * sizeof(VTile), s));
    }
    dfree(d_img, s);
    dfree(d_tile_nv, s);
    dfree(d_tkey, s);
    dfree(d_tm, s);
    dfree(d_tps, s);
    g->gt = d_tiles;          // kept for the splat
    g->gt_voff = d_tile_voff;
    g->ngt = ntiles;
    g->gt_p2 = P2;
    prof_end(f_region, s);
    *out = g;
    return FBS_OK;
fail:
    st = cuda_status(e);
fail_status:
    dfree(d_img, s);
    dfree(d_tiles, s);
    dfree(d_tile_nv, s);
    dfree(d_tile_voff, s);
    dfree(d_tkey, s);
    dfree(d_tm, s);
    dfree(d_tps, s);
    free_grid_memory(g, s);
    delete g;
    return st;
#undef FBS_TRY
}

fbs_status fbs_bistochastize(fbs_grid* g, int iters, void* stream)
{
    if (!g || iters < 1) return FBS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    static int f_region = prof_family("region:bistochastize", 2);
    prof_begin(f_region, s);
    for (int it = 0; it < iters; ++it) {
        const double* nold = g->n64;
        double* nnew = g->n64b;
        cudaError_t e = launch_bistoch(nold, nnew, g->nf, g->m, g->nbr, g->nbr_stride, g->Vtot,
                                       it == 0,
                                       it == iters - 1, s);
        if (e != cudaSuccess) return cuda_status(e);
        std::swap(g->n64, g->n64b);
    }
    prof_end(f_region, s);
    g->bistoch_iters = iters;
    return FBS_OK;
}

}  // extern "C"

namespace {

fbs_status check_problems(const fbs_grid* g, const fbs_problem_desc* probs, int pcg_iters)
{
    if (!g || !probs || pcg_iters < 0) return FBS_ERR_ARG;
    for (int k = 0; k < g->n_images; ++k) {
        const fbs_problem_desc& p = probs[k];
        if (!p.t || !p.c || p.channels < 1 || p.channels > kMaxChannels || !(p.lambda >= 0.f) ||
            !isfinite(p.lambda))
            return FBS_ERR_ARG;
    }
    if (g->bistoch_iters < 1) return FBS_ERR_STATE;
    return FBS_OK;
}

// One segment, replayed from a CUDA graph captured on first use (per exact
// launch arguments), or launched directly while the caller's stream is being
// captured or per-kernel timing is on.
cudaError_t run_segment(fbs_grid* g, const SolveArgs& A, const SolvePlan& P, int seg, int mode,
                        cudaStream_t s)
{
    if (capturing(s) || prof_level() == 1 || (seg == kSegLoop && P.persistent))
        return launch_segment(A, P, seg, mode, s);
    fbs_grid::GraphEntry* seen = nullptr;
    for (auto& e : g->graphs)
        if (e.seg == seg && e.mode == mode && memcmp(&e.A, &A, sizeof(A)) == 0 &&
            memcmp(&e.P, &P, sizeof(P)) == 0)
            seen = &e;
    if (seen && seen->exec) return cudaGraphLaunch(seen->exec, s);
    if (!seen) {
        // first sighting: launch directly and remember the arguments; a graph
        // is captured only when the same launch comes back
        if (g->graphs.size() >= 16) {
            if (g->graphs.front().exec) cudaGraphExecDestroy(g->graphs.front().exec);
            g->graphs.erase(g->graphs.begin());
        }
        fbs_grid::GraphEntry entry;
        memcpy(&entry.A, &A, sizeof(A));
        memcpy(&entry.P, &P, sizeof(P));
        entry.seg = seg;
        entry.mode = mode;
        entry.exec = nullptr;
        g->graphs.push_back(entry);
        return launch_segment(A, P, seg, mode, s);
    }
    cudaError_t err = cudaSuccess;
    if (!g->cap_stream) {
        err = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
        if (err != cudaSuccess) return err;
    }
    err = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return err;
    cudaError_t lerr = launch_segment(A, P, seg, mode, g->cap_stream);
    cudaGraph_t graph = nullptr;
    err = cudaStreamEndCapture(g->cap_stream, &graph);
    if (lerr != cudaSuccess) err = lerr;
    if (err != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return err;
    }
    cudaGraphExec_t exec = nullptr;
    err = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) return err;
    seen->exec = exec;
    return cudaGraphLaunch(exec, s);
}

fbs_status run_segments(fbs_grid* g, const SolveArgs& A, const SolvePlan& P, cudaStream_t s)
{
    static int f_setup = prof_family("region:solve_setup", 2);
    static int f_loop = prof_family("region:pcg_loop", 2);
    static int f_out = prof_family("region:slice", 2);
    cudaError_t e = cudaSuccess;
    for (int outer = 0; outer < P.outer_iters && e == cudaSuccess; ++outer) {
        const int mode = P.mode == kSplatRobust && outer == 0 ? kSplatConfidence : P.mode;
        prof_begin(f_setup, s);
        e = run_segment(g, A, P, kSegSetup, mode, s);
        prof_end(f_setup, s);
        if (e != cudaSuccess) break;
        prof_begin(f_loop, s);
        e = run_segment(g, A, P, kSegLoop, mode, s);
        prof_end(f_loop, s);
    }
    if (e == cudaSuccess) {
        prof_begin(f_out, s);
        e = run_segment(g, A, P, kSegOut, P.mode, s);
        prof_end(f_out, s);
    }
    return cuda_status(e);
}

// halves every 12-bit key field (floor): the parent key one pyramid level up
// The bilateral-space pyramid of the grid (supplement, bilateral-space
// pyramids), built on the GPU once per grid: per image, level k+1 is the
// distinct floor-halved keys of level k (floor halving reaches a single
// vertex), numbered in first-occurrence order (see pyramid.cu); the images'
// levels are concatenated level by level (an image that reached its top
// keeps one vertex, with count and weights 0, so each image's result is that
// of its own pyramid), with each vertex's parent, each vertex's children in
// ascending order (so the device sums are deterministic), the counts P(1)
// and the initialisation weights 4^-k / P(1).  The host reads back only the
// per-image level sizes (one synchronisation per level).
fbs_status build_pyramid(fbs_grid* g, cudaStream_t s)
{
    const int n = g->n_images;
    const int64_t V = g->Vtot;
    std::vector<std::vector<int64_t>> lstart(1, g->voff);          // level-local image starts
    std::vector<uint64_t*> keyL(1, g->vkey);
    std::vector<uint16_t*> imgL(1, nullptr);
    std::vector<int32_t*> parL;
    int64_t* d_idx = nullptr;
    int64_t* d_out = nullptr;
    int64_t* d_htoff = nullptr;
    unsigned long long* hkey = nullptr;
    int32_t *hmin = nullptr, *slot = nullptr;
    uint32_t *flag = nullptr, *idv = nullptr, *tmp = nullptr;
    int64_t* d_off = nullptr;
    uint32_t *tcnt = nullptr, *tscan = nullptr;
    cudaError_t e = cudaSuccess;
    auto level_tmp_free = [&]() {
        dfree(d_htoff, s); dfree(hkey, s); dfree(hmin, s); dfree(slot, s); dfree(flag, s);
        dfree(idv, s); dfree(tmp, s);
    };
    auto cleanup = [&]() {
        level_tmp_free();
        dfree(d_idx, s); dfree(d_out, s); dfree(d_off, s); dfree(tcnt, s); dfree(tscan, s);
        for (size_t k = 1; k < keyL.size(); ++k) dfree(keyL[k], s);
        for (auto*& p : imgL) dfree(p, s);
        for (auto*& p : parL) dfree(p, s);
    };
#define PYR_TRY(x)                        \
    do {                                  \
        if ((e = (x)) != cudaSuccess) {   \
            cleanup();                    \
            return cuda_status(e);        \
        }                                 \
    } while (0)
    PYR_TRY(dalloc(&imgL[0], (size_t)V, s));
    PYR_TRY(dalloc(&d_idx, (size_t)n + 1, s));
    PYR_TRY(dalloc(&d_out, (size_t)n + 1, s));
    PYR_TRY(cudaMemcpyAsync(d_idx, g->voff.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    PYR_TRY(fill_vimg(d_idx, n, V, imgL[0], s));
    std::vector<int64_t> hout(n + 1);
    for (int k = 0;; ++k) {
        const std::vector<int64_t>& ls = lstart[k];
        bool all_top = true;
        for (int im = 0; im < n; ++im) all_top &= ls[im + 1] - ls[im] == 1;
        if (all_top) break;
        if (k + 1 >= kMaxLevels) {
            cleanup();
            return FBS_ERR_ARG;
        }
        const int64_t nk = ls[n];
        std::vector<int64_t> htoff(n + 1, 0);
        for (int im = 0; im < n; ++im) {
            int64_t sz = 2;
            while (sz < 2 * (ls[im + 1] - ls[im])) sz <<= 1;
            htoff[im + 1] = htoff[im] + sz;
        }
        if (htoff[n] > INT32_MAX) {           // hash slots are 32-bit
            cleanup();
            return FBS_ERR_ARG;
        }
        PYR_TRY(dalloc(&d_htoff, (size_t)n + 1, s));
        PYR_TRY(dalloc(&hkey, (size_t)htoff[n], s));
        PYR_TRY(dalloc(&hmin, (size_t)htoff[n], s));
        PYR_TRY(dalloc(&slot, (size_t)nk, s));
        PYR_TRY(dalloc(&flag, (size_t)nk, s));
        PYR_TRY(dalloc(&idv, (size_t)nk + 1, s));
        PYR_TRY(dalloc(&tmp, (size_t)(nk / 1024 + 2), s));
        PYR_TRY(cudaMemcpyAsync(d_htoff, htoff.data(), (n + 1) * sizeof(int64_t),
                                cudaMemcpyHostToDevice, s));
        PYR_TRY(cudaMemsetAsync(hkey, 0xFF, (size_t)htoff[n] * sizeof(unsigned long long), s));
        PYR_TRY(cudaMemsetAsync(hmin, 0x7F, (size_t)htoff[n] * sizeof(int32_t), s));
        PyrLevelArgs L;
        L.key = keyL[k];
        L.img = imgL[k];
        L.n = nk;
        L.htoff = d_htoff;
        L.hkey = hkey;
        L.hmin = hmin;
        L.slot = slot;
        L.flag = flag;
        L.id = idv;
        L.err = g->err;
        PYR_TRY(pyr_level_insert(L, s));
        PYR_TRY(scan_u32(flag, idv, nk, tmp, s));
        // next-level image starts: the ids at this level's image starts
        PYR_TRY(cudaMemcpyAsync(d_idx, ls.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        PYR_TRY(gather_u32(idv, d_idx, d_out, n + 1, s));
        PYR_TRY(cudaMemcpyAsync(hout.data(), d_out, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        PYR_TRY(cudaStreamSynchronize(s));
        lstart.push_back(hout);
        const int64_t nk1 = hout[n];
        keyL.push_back(nullptr);
        imgL.push_back(nullptr);
        parL.push_back(nullptr);
        PYR_TRY(dalloc(&keyL[k + 1], (size_t)nk1, s));
        PYR_TRY(dalloc(&imgL[k + 1], (size_t)nk1, s));
        PYR_TRY(dalloc(&parL[k], (size_t)nk, s));
        L.parent = parL[k];
        L.key1 = keyL[k + 1];
        L.img1 = imgL[k + 1];
        PYR_TRY(pyr_level_finish(L, s));
        level_tmp_free();
    }
    const int K = (int)lstart.size();
    int64_t off[kMaxLevels + 1];
    off[0] = 0;
    for (int k = 0; k < K; ++k) off[k + 1] = off[k] + lstart[k][n];
    const int64_t T = off[K];
    std::vector<int64_t> ioffa((size_t)K * (n + 1));
    for (int k = 0; k < K; ++k)
        for (int im = 0; im <= n; ++im) ioffa[(size_t)k * (n + 1) + im] = off[k] + lstart[k][im];
    std::vector<uint8_t> kimg(n, (uint8_t)K);
    for (int im = 0; im < n; ++im)
        for (int k = 0; k < K; ++k)
            if (lstart[k][im + 1] - lstart[k][im] == 1) {
                kimg[im] = (uint8_t)(k + 1);
                break;
            }
    // the concatenated arrays
    PYR_TRY(dalloc(&g->pyr_parent, (size_t)std::max<int64_t>(off[K - 1], 1), s));
    PYR_TRY(dalloc(&g->pyr_child_off, (size_t)(T - V + 1), s));
    PYR_TRY(dalloc(&g->pyr_child_idx, (size_t)std::max<int64_t>(off[K - 1], 1), s));
    PYR_TRY(dalloc(&g->pyr_vimg, (size_t)T, s));
    PYR_TRY(dalloc(&g->pyr_key, (size_t)T, s));
    PYR_TRY(dalloc(&g->pyr_ioff, ioffa.size(), s));
    PYR_TRY(dalloc(&g->pyr_kimg, kimg.size(), s));
    PYR_TRY(dalloc(&g->pyr_cnt, (size_t)T, s));
    PYR_TRY(dalloc(&g->pyr_cinit, (size_t)T, s));
    PYR_TRY(dalloc(&g->pyr_coef, (size_t)T, s));
    PYR_TRY(dalloc(&g->pyr_dg, (size_t)V, s));
    PYR_TRY(dalloc(&g->pyr_scv, (size_t)V, s));
    PYR_TRY(dalloc(&g->pyr_lv, (size_t)std::max<int64_t>(T - V, 1) * kPyrMaxNc, s));
    g->pyr_lv_nc = kPyrMaxNc;
    for (int k = 0; k < K; ++k) {
        PYR_TRY(cudaMemcpyAsync(g->pyr_vimg + off[k], imgL[k], lstart[k][n] * sizeof(uint16_t),
                                cudaMemcpyDeviceToDevice, s));
        PYR_TRY(cudaMemcpyAsync(g->pyr_key + off[k], keyL[k], lstart[k][n] * sizeof(uint64_t),
                                cudaMemcpyDeviceToDevice, s));
        if (k + 1 < K)
            PYR_TRY(cudaMemcpyAsync(g->pyr_parent + off[k], parL[k], lstart[k][n] * sizeof(int32_t),
                                    cudaMemcpyDeviceToDevice, s));
    }
    PYR_TRY(cudaMemcpyAsync(g->pyr_ioff, ioffa.data(), ioffa.size() * sizeof(int64_t),
                            cudaMemcpyHostToDevice, s));
    PYR_TRY(cudaMemcpyAsync(g->pyr_kimg, kimg.data(), kimg.size(), cudaMemcpyHostToDevice, s));
    PYR_TRY(dalloc(&d_off, (size_t)K + 1, s));
    PYR_TRY(cudaMemcpyAsync(d_off, off, (K + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    const int64_t np = T - V;
    PYR_TRY(dalloc(&tcnt, (size_t)3 * (np + 1), s));
    PYR_TRY(dalloc(&tscan, (size_t)(np / 1024 + 2), s));
    PYR_TRY(pyr_children(g->pyr_parent, d_off, K, T, V, g->pyr_child_off, g->pyr_child_idx, tcnt,
                         tscan, s));
    PYR_TRY(pyr_counts(g->pyr_child_off, g->pyr_child_idx, off, d_off, K, g->pyr_ioff, g->pyr_kimg, n,
                       g->pyr_cnt, g->pyr_cinit, s));
    // the host copies above are stream-ordered: finish before their sources go
    PYR_TRY(cudaStreamSynchronize(s));
    cleanup();
#undef PYR_TRY
    g->pyr_K = K;
    for (int k = 0; k <= K; ++k) g->pyr_off[k] = off[k];
    g->pyr_ioff_host = ioffa;
    return FBS_OK;
}

// Sizes the workspace, uploads the image descriptors (if they changed) and
// runs one solve plan.
fbs_status run(fbs_grid* g, std::vector<InstDev>& inst, SolvePlan plan, cudaStream_t s)
{
    int64_t cv = 0, cpart = 0;
    int pc = 0, cmax = 1;
    for (int k = 0; k < g->n_images; ++k) {
        InstDev& I = inst[k];
        I.voff = g->voff[k];
        I.V = (int)(g->voff[k + 1] - g->voff[k]);
        I.Cp = padded_channels(I.C);
        I.vec_base = cv;
        I.tile0 = g->vt0[k];
        I.ntiles = g->nvt_img[k];
        I.pc = pc;
        I.part_base = cpart;
        I.N = (int64_t)g->img[k].H * g->img[k].W;
        I.pix_base = g->img[k].pix_base;
        cv += ((int64_t)I.Cp * I.V + 31) / 32 * 32;  // 128-byte aligned image blocks
        cpart += (int64_t)I.C * I.ntiles;
        pc += I.C;
        cmax = std::max(cmax, I.C);
        plan.max_cv = std::max<int64_t>(plan.max_cv, (int64_t)I.C * I.V);
    }
    plan.max_pixels = g->max_pixels;
    plan.chan_block = std::min(cmax, kChanBlock);
    plan.cmax = cmax;
    // vector precision: FP32 state for forward and robust solves, the
    // compensated variant for the backward solve (whose right-hand side is
    // an arbitrary gradient) unless the caller chose otherwise
    if (g->precision == FBS_VECTORS_FP32) plan.comp = 0;
    else if (g->precision == FBS_VECTORS_COMPENSATED) plan.comp = 1;
    else plan.comp = plan.mode == kSplatBackward ? 1 : 0;
    // the robust solver in compensated precision also keeps y and a' as
    // double-float pairs: its IRLS loop amplifies their float32 rounding
    plan.dfy = plan.comp && plan.mode == kSplatRobust ? 1 : 0;
    // the whole PCG loop as one cooperative launch, except inside a caller's
    // stream capture (per-phase launches are captured instead)
    // the single-reduction form for FP32 vectors and images of at most 4
    // channels; it runs as per-phase launches
    plan.single = g->pcg_form == FBS_PCG_FORM_SINGLE && !plan.comp && cmax <= 4 ? 1 : 0;
    // hierarchical preconditioner: any channel count
    plan.hier = g->precond == FBS_PRECOND_HIERARCHICAL ? 1 : 0;
    if (plan.hier) plan.single = 0;
    plan.persistent = g->persistent && !capturing(s) && !plan.hier ? 1 : 0;
    plan.block_mult = g->phase_blocks;
    plan.force_persistent = g->force_persistent;
    plan.inject_timeout = plan.persistent ? g->inject_timeout : 0;
    if (plan.persistent) g->inject_timeout = 0;
    const bool cap = capturing(s);
    cudaError_t e = cudaSuccess;
    if ((size_t)cv > g->cap_vec || (size_t)pc > g->cap_scal || (size_t)cpart > g->cap_part ||
        !g->a) {
        if (cap) return FBS_ERR_STATE;   // size the workspace outside capture first
        free_graphs(g);
        dfree(g->vec, s); dfree(g->a, s); dfree(g->nm, s); dfree(g->scal, s);
        dfree(g->part, s); dfree(g->inst, s);
        g->inst_cached.clear();
        g->cap_vec = (size_t)std::max<int64_t>(cv, 32);
        g->cap_scal = (size_t)std::max(pc, 1);
        g->cap_part = (size_t)std::max<int64_t>(cpart, 1);
        if ((e = dalloc(&g->vec, 8 * g->cap_vec, s)) != cudaSuccess) return cuda_status(e);
        if ((e = dalloc(&g->a, g->Vtot, s)) != cudaSuccess) return cuda_status(e);
        if ((e = dalloc(&g->nm, g->Vtot, s)) != cudaSuccess) return cuda_status(e);
        if ((e = dalloc(&g->scal, g->cap_scal, s)) != cudaSuccess) return cuda_status(e);
        if ((e = dalloc(&g->part, 4 * g->cap_part, s)) != cudaSuccess) return cuda_status(e);
        if (!g->barrier && (e = dalloc(&g->barrier, kBarrierWords, s)) != cudaSuccess)
            return cuda_status(e);
        if ((e = dalloc(&g->inst, (size_t)g->n_images, s)) != cudaSuccess) return cuda_status(e);
    }
    if (g->inst_cached.size() != inst.size() ||
        memcmp(g->inst_cached.data(), inst.data(), inst.size() * sizeof(InstDev)) != 0) {
        if ((e = upload(g->inst, inst.data(), inst.size() * sizeof(InstDev), s)) != cudaSuccess)
            return cuda_status(e);
        g->inst_cached = inst;
    }
    SolveArgs A;
    memset(&A, 0, sizeof(A));
    A.vt = g->vt;
    A.nvt = g->nvt;
    A.inst = g->inst;
    A.ninst = g->n_images;
    A.nbr = g->nbr;
    A.nbr_stride = g->nbr_stride;
    A.nbrp = g->nbrp;
    A.Vtot = g->Vtot;
    A.n64 = g->n64;
    A.m = g->m;
    A.pstart = g->pstart;
    A.perm = g->perm;
    A.vid = g->vid;
    A.a = g->a;
    A.nm = g->nm;
    A.y = g->vec;
    A.r = g->vec + g->cap_vec;
    A.rlo = g->vec + 2 * g->cap_vec;
    A.d[0] = g->vec + 3 * g->cap_vec;
    A.d[1] = g->vec + 4 * g->cap_vec;
    A.q = g->vec + 5 * g->cap_vec;
    A.aux[0] = g->vec + 6 * g->cap_vec;
    A.aux[1] = g->vec + 7 * g->cap_vec;
    if (plan.dfy && !g->alo) {
        if (cap) return FBS_ERR_STATE;
        if ((e = dalloc(&g->alo, g->Vtot, s)) != cudaSuccess) return cuda_status(e);
    }
    A.alo = plan.dfy ? g->alo : nullptr;
    A.ylo = plan.dfy ? A.aux[1] : nullptr;
    A.zq = !plan.comp && !plan.hier && !plan.single ? A.aux[0] : nullptr;
    A.nf = g->nf;
    A.scal = g->scal;
    A.nscal = pc;
    plan.barrier = g->barrier;
    A.part_rs[0] = g->part;
    A.part_rs[1] = g->part + g->cap_part;
    A.part_dq = g->part + 2 * g->cap_part;
    A.part_mu[0] = A.part_dq;
    A.part_mu[1] = g->part + 3 * g->cap_part;
    A.err = g->err;
    if (plan.hier) {
        if (g->pyr_K == 0) {
            if (cap) return FBS_ERR_STATE;          // first hierarchical solve inside capture
            fbs_status pst = build_pyramid(g, s);
            if (pst) return pst;
        }
        A.pyr.K = g->pyr_K;
        A.pyr.W = 1;
        for (const InstDev& d : inst) A.pyr.W = std::max(A.pyr.W, d.Cp);
        if (A.pyr.W + 2 > g->pyr_lv_nc) {           // level vectors of a wider solve
            if (cap) return FBS_ERR_STATE;
            dfree(g->pyr_lv, s);
            const int64_t nup = std::max<int64_t>(g->pyr_off[g->pyr_K] - g->pyr_off[1], 1);
            if ((e = dalloc(&g->pyr_lv, (size_t)nup * (A.pyr.W + 2), s)) != cudaSuccess) {
                g->pyr_lv_nc = 0;
                return cuda_status(e);
            }
            g->pyr_lv_nc = A.pyr.W + 2;
        }
        for (int k = 0; k <= g->pyr_K; ++k) A.pyr.off[k] = g->pyr_off[k];
        A.pyr.parent = g->pyr_parent;
        A.pyr.child_off = g->pyr_child_off;
        A.pyr.child_idx = g->pyr_child_idx;
        A.pyr.vimg = g->pyr_vimg;
        A.pyr.ioff = g->pyr_ioff;
        A.pyr.kimg = g->pyr_kimg;
        A.pyr.cnt = g->pyr_cnt;
        A.pyr.cinit = g->pyr_cinit;
        A.pyr.coef = g->pyr_coef;
        A.pyr.dg = g->pyr_dg;
        A.pyr.scv = g->pyr_scv;
        A.pyr.lv = g->pyr_lv;
        A.pyr.z = A.aux[0];
    }
    // AUTO: the resident loop for small batches; per-phase (graph) otherwise
    if (plan.persistent && !plan.force_persistent && !resident_preferred(A, plan))
        plan.persistent = 0;
    // the resident loop finalises each phase's scalars in its barrier; the
    // initial residual then finalises delta_0 the same way
    A.fin = plan.persistent && resident_fits(A, plan) ? 1 : 0;
    return run_segments(g, A, plan, s);
}

std::vector<InstDev> base_instances(const fbs_grid* g, const fbs_problem_desc* probs)
{
    std::vector<InstDev> inst(g->n_images);
    for (int k = 0; k < g->n_images; ++k) {
        InstDev I;
        memset(&I, 0, sizeof(I));
        I.C = probs[k].channels;
        I.lam = probs[k].lambda;
        I.t = probs[k].t;
        I.c = probs[k].c;
        I.x = probs[k].x;
        I.yout = probs[k].y;
        inst[k] = I;
    }
    return inst;
}

// ------------------------------------------------ low-rank reduction ---
// The reduction of a wide B = S(c o T) (V x C) by a column-pivoted QR
// B P = Q R (supplement, multiple output channels).  R and P come from the
// pivoted Cholesky factorisation of G = B^T B: pivoting on the largest
// remaining diagonal of the Schur complement is pivoting on the largest
// remaining column norm, so R^T R = P^T G P gives the same R (rows with
// positive diagonal) as the QR.  Rows of R are ranked by their mass
// m_i = |R_i|^2 (stable: ties in pivot order); the t kept are the fewest
// leading ones whose mass reaches (1 - eps) of the total |B|_F^2 = trace G.
// Q's kept columns are Q_k = B P R^-1 e_k, so the reduced right-hand sides
// are B W with W = P R^-1 restricted to the kept columns (C x t), and
// Y = Y_reduced R~ with R~ = the kept rows of R P^T (t x C).
struct LrChoice {
    int t = 0;                  // rows kept (0: B = 0)
    std::vector<float> W;       // C x max(t, 1), row-major
    std::vector<float> Rt;      // max(t, 1) x C, row-major
};

LrChoice lr_choose(const double* G, int ld, int C, double eps)
{
    std::vector<double> S((size_t)C * C), R((size_t)C * C, 0.0);
    for (int i = 0; i < C; ++i)
        for (int j = 0; j < C; ++j) S[(size_t)i * C + j] = G[(size_t)i * ld + j];
    std::vector<int> piv(C);
    for (int j = 0; j < C; ++j) piv[j] = j;
    double dmax = 0.0, total = 0.0;
    for (int j = 0; j < C; ++j) {
        dmax = std::max(dmax, S[(size_t)j * C + j]);
        total += S[(size_t)j * C + j];
    }
    // numerical rank: a pivot at or below 1e-13 of the largest column mass
    // is rounding noise of an exactly dependent column
    const double tol = dmax * 1e-13;
    int r = 0;
    for (int k = 0; k < C; ++k) {
        int p = k;
        for (int j = k + 1; j < C; ++j)
            if (S[(size_t)j * C + j] > S[(size_t)p * C + p]) p = j;
        if (!(S[(size_t)p * C + p] > tol)) break;
        if (p != k) {
            std::swap(piv[k], piv[p]);
            for (int j = 0; j < C; ++j) std::swap(S[(size_t)k * C + j], S[(size_t)p * C + j]);
            for (int i = 0; i < C; ++i) std::swap(S[(size_t)i * C + k], S[(size_t)i * C + p]);
            for (int i = 0; i < k; ++i) std::swap(R[(size_t)i * C + k], R[(size_t)i * C + p]);
        }
        const double rkk = sqrt(S[(size_t)k * C + k]);
        R[(size_t)k * C + k] = rkk;
        for (int j = k + 1; j < C; ++j) R[(size_t)k * C + j] = S[(size_t)k * C + j] / rkk;
        for (int i = k + 1; i < C; ++i)
            for (int j = k + 1; j < C; ++j)
                S[(size_t)i * C + j] -= R[(size_t)k * C + i] * R[(size_t)k * C + j];
        r = k + 1;
    }
    LrChoice out;
    std::vector<double> mass(r, 0.0);
    for (int k = 0; k < r; ++k)
        for (int j = k; j < C; ++j) mass[k] += R[(size_t)k * C + j] * R[(size_t)k * C + j];
    std::vector<int> order(r);
    for (int k = 0; k < r; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return mass[a] > mass[b]; });
    int t = 0;
    if (total > 0.0) {
        double acc = 0.0;
        while (t < r && acc < (1.0 - eps) * total) acc += mass[order[t++]];
    }
    out.t = t;
    const int tc = std::max(t, 1);
    out.W.assign((size_t)C * tc, 0.0f);
    out.Rt.assign((size_t)tc * C, 0.0f);
    if (t == 0) return out;
    // R^-1 of the leading r x r block (upper triangular), column by column
    std::vector<double> Ri((size_t)r * r, 0.0);
    for (int k = 0; k < r; ++k) {
        Ri[(size_t)k * r + k] = 1.0 / R[(size_t)k * C + k];
        for (int i = k - 1; i >= 0; --i) {
            double acc = 0.0;
            for (int j = i + 1; j <= k; ++j) acc += R[(size_t)i * C + j] * Ri[(size_t)j * r + k];
            Ri[(size_t)i * r + k] = -acc / R[(size_t)i * C + i];
        }
    }
    for (int q = 0; q < t; ++q) {
        const int k = order[q];
        for (int j = 0; j <= k; ++j) out.W[(size_t)piv[j] * tc + q] = (float)Ri[(size_t)j * r + k];
        for (int j = k; j < C; ++j) out.Rt[(size_t)q * C + piv[j]] = (float)R[(size_t)k * C + j];
    }
    return out;
}

}  // namespace

extern "C" {

fbs_status fbs_solve_lowrank(fbs_grid* g, const fbs_problem_desc* probs, int pcg_iters,
                             double eps, int* ranks, void* stream)
{
    fbs_status st = check_problems(g, probs, pcg_iters);
    if (st) return st;
    if (!(eps >= 1e-12 && eps < 1.0)) return FBS_ERR_ARG;
    const int n = g->n_images;
    for (int k = 0; k < n; ++k)
        if (!probs[k].x || probs[k].y) return FBS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (capturing(s)) return FBS_ERR_STATE;
    int cmax = 1;
    for (int k = 0; k < n; ++k) cmax = std::max(cmax, probs[k].channels);
    // B and its Gram matrices
    std::vector<LrImg> li(n);
    int64_t bfl = 0;
    for (int k = 0; k < n; ++k) {
        LrImg& L = li[k];
        memset(&L, 0, sizeof(L));
        L.t = probs[k].t;
        L.c = probs[k].c;
        L.C = probs[k].channels;
        L.N = (int64_t)g->img[k].H * g->img[k].W;
        L.pix_base = g->img[k].pix_base;
        L.v0 = g->voff[k];
        L.nv = g->voff[k + 1] - g->voff[k];
        L.boff = bfl;
        bfl += L.nv * L.C;
    }
    LrImg* d_li = nullptr;
    int64_t* d_voff = nullptr;
    float* B = nullptr;
    float2* part = nullptr;
    double* G = nullptr;
    float *d_M = nullptr, *d_tr = nullptr, *d_xr = nullptr;
    std::vector<double> hG((size_t)n * cmax * cmax);
    std::vector<LrChoice> ch(n);
    cudaError_t e = cudaSuccess;
    auto cleanup = [&]() {
        dfree(d_li, s); dfree(d_voff, s); dfree(B, s); dfree(part, s); dfree(G, s);
        dfree(d_M, s); dfree(d_tr, s); dfree(d_xr, s);
    };
#define LR_TRY(x)                          \
    do {                                   \
        if ((e = (x)) != cudaSuccess) {    \
            cleanup();                     \
            return cuda_status(e);         \
        }                                  \
    } while (0)
    LR_TRY(dalloc(&d_li, (size_t)n, s));
    LR_TRY(dalloc(&d_voff, (size_t)n + 1, s));
    LR_TRY(dalloc(&B, (size_t)bfl, s));
    LR_TRY(dalloc(&part, (size_t)n * kLrGramBlocks * (cmax * (cmax + 1) / 2), s));
    LR_TRY(dalloc(&G, hG.size(), s));
    LR_TRY(cudaMemcpyAsync(d_li, li.data(), n * sizeof(LrImg), cudaMemcpyHostToDevice, s));
    LR_TRY(cudaMemcpyAsync(d_voff, g->voff.data(), (n + 1) * sizeof(int64_t),
                           cudaMemcpyHostToDevice, s));
    LR_TRY(lr_splat(d_li, n, g->Vtot, d_voff, g->pstart, g->m, g->perm, B, s));
    LR_TRY(lr_gram(d_li, n, B, part, G, cmax, s));
    LR_TRY(cudaMemcpyAsync(hG.data(), G, hG.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    LR_TRY(cudaStreamSynchronize(s));
    // ranks and the maps in and out of the reduced system
    int64_t mfl = 0, rfl = 0;
    std::vector<int64_t> moff(n), roff(n);
    for (int k = 0; k < n; ++k) {
        ch[k] = lr_choose(hG.data() + (size_t)k * cmax * cmax, cmax, li[k].C, eps);
        if (ranks) ranks[k] = ch[k].t;
        moff[k] = mfl;
        mfl += 2 * (int64_t)ch[k].W.size();
        roff[k] = rfl;
        rfl += li[k].N * std::max(ch[k].t, 1);
    }
    std::vector<float> hM((size_t)mfl);
    for (int k = 0; k < n; ++k) {
        std::copy(ch[k].W.begin(), ch[k].W.end(), hM.begin() + moff[k]);
        std::copy(ch[k].Rt.begin(), ch[k].Rt.end(), hM.begin() + moff[k] + ch[k].W.size());
    }
    LR_TRY(dalloc(&d_M, (size_t)mfl, s));
    LR_TRY(dalloc(&d_tr, (size_t)rfl, s));
    LR_TRY(dalloc(&d_xr, (size_t)rfl, s));
    LR_TRY(cudaMemcpyAsync(d_M, hM.data(), mfl * sizeof(float), cudaMemcpyHostToDevice, s));
    // reduced targets T W
    int64_t max_pixels = 1;
    for (int k = 0; k < n; ++k) {
        li[k].Cout = std::max(ch[k].t, 1);
        li[k].M = d_M + moff[k];
        li[k].out = d_tr + roff[k];
        max_pixels = std::max(max_pixels, li[k].N);
    }
    LR_TRY(cudaMemcpyAsync(d_li, li.data(), n * sizeof(LrImg), cudaMemcpyHostToDevice, s));
    LR_TRY(lr_map(d_li, n, max_pixels, s));
    // the reduced solve
    std::vector<fbs_problem_desc> rp(probs, probs + n);
    for (int k = 0; k < n; ++k) {
        rp[k].t = d_tr + roff[k];
        rp[k].x = d_xr + roff[k];
        rp[k].y = nullptr;
        rp[k].channels = li[k].Cout;
    }
    std::vector<InstDev> inst = base_instances(g, rp.data());
    SolvePlan plan;
    memset(&plan, 0, sizeof(plan));
    plan.mode = kSplatConfidence;
    plan.outer_iters = 1;
    plan.pcg_iters = pcg_iters;
    plan.sigma_gm = 1.0f;
    st = run(g, inst, plan, s);
    if (st) {
        cleanup();
        return st;
    }
    // x = x_reduced R~
    for (int k = 0; k < n; ++k) {
        li[k].t = d_xr + roff[k];
        li[k].C = li[k].Cout;
        li[k].Cout = probs[k].channels;
        li[k].M = d_M + moff[k] + ch[k].W.size();
        li[k].out = probs[k].x;
    }
    // (stream-ordered after the first map, which read the previous copy)
    if ((e = cudaMemcpyAsync(d_li, li.data(), n * sizeof(LrImg), cudaMemcpyHostToDevice, s)) ==
        cudaSuccess)
        e = lr_map(d_li, n, max_pixels, s);
    // the host copies above are stream-ordered: finish them before the
    // host vectors go out of scope
    const cudaError_t e2 = cudaStreamSynchronize(s);
    cleanup();
#undef LR_TRY
    if (e != cudaSuccess) return cuda_status(e);
    return e2 == cudaSuccess ? FBS_OK : cuda_status(e2);
}

fbs_status fbs_domain_transform(const float* guide, int height, int width, float* x, int channels,
                                float sigma_s, float sigma_r, int iterations, void* stream)
{
    if (!guide || !x || height < 1 || width < 1 || channels < 1 || channels > 65535 ||
        !(sigma_s > 0.f) || !isfinite(sigma_s) || !(sigma_r > 0.f) || !isfinite(sigma_r) ||
        iterations < 1 || iterations > 16 || width > domain_transform_max_width())
        return FBS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = (size_t)height * width;
    float *dh = nullptr, *dv = nullptr;
    cudaError_t e = dalloc(&dh, N, s);
    if (e == cudaSuccess) e = dalloc(&dv, N, s);
    if (e == cudaSuccess)
        e = domain_transform(guide, height, width, x, channels, sigma_s, sigma_r, iterations, dh,
                             dv, s);
    dfree(dh, s);
    dfree(dv, s);
    return e == cudaSuccess ? FBS_OK : cuda_status(e);
}

fbs_status fbs_solve(fbs_grid* g, const fbs_problem_desc* probs, int pcg_iters, void* stream)
{
    fbs_status st = check_problems(g, probs, pcg_iters);
    if (st) return st;
    std::vector<InstDev> inst = base_instances(g, probs);
    SolvePlan plan;
    memset(&plan, 0, sizeof(plan));
    plan.mode = kSplatConfidence;
    plan.outer_iters = 1;
    plan.pcg_iters = pcg_iters;
    plan.sigma_gm = 1.0f;
    plan.export_y = false;
    for (int k = 0; k < g->n_images; ++k) plan.export_y |= probs[k].y != nullptr;
    return run(g, inst, plan, (cudaStream_t)stream);
}

fbs_status fbs_solve_robust(fbs_grid* g, const fbs_problem_desc* probs, float sigma_gm,
                            int irls_iters, int pcg_iters, void* stream)
{
    fbs_status st = check_problems(g, probs, pcg_iters);
    if (st) return st;
    if (!(sigma_gm > 0.f) || !isfinite(sigma_gm) || irls_iters < 1) return FBS_ERR_ARG;
    for (int k = 0; k < g->n_images; ++k)
        if (probs[k].channels != 1) return FBS_ERR_ARG;
    std::vector<InstDev> inst = base_instances(g, probs);
    SolvePlan plan;
    memset(&plan, 0, sizeof(plan));
    plan.mode = kSplatRobust;
    plan.outer_iters = irls_iters;
    plan.pcg_iters = pcg_iters;
    plan.sigma_gm = sigma_gm;
    for (int k = 0; k < g->n_images; ++k) plan.export_y |= probs[k].y != nullptr;
    return run(g, inst, plan, (cudaStream_t)stream);
}

fbs_status fbs_solve_backward(fbs_grid* g, const fbs_problem_desc* probs,
                              const float* const* dL_dx, float* const* dL_dt,
                              float* const* dL_dc, int pcg_iters, void* stream)
{
    fbs_status st = check_problems(g, probs, pcg_iters);
    if (st) return st;
    if (!dL_dx || !dL_dt || !dL_dc) return FBS_ERR_ARG;
    std::vector<InstDev> inst = base_instances(g, probs);
    for (int k = 0; k < g->n_images; ++k) {
        if (!probs[k].y || !dL_dx[k]) return FBS_ERR_ARG;
        inst[k].x = nullptr;
        inst[k].yout = nullptr;
        inst[k].yhat = probs[k].y;
        inst[k].dx = dL_dx[k];
        inst[k].dt = dL_dt[k];
        inst[k].dc = dL_dc[k];
    }
    SolvePlan plan;
    memset(&plan, 0, sizeof(plan));
    plan.mode = kSplatBackward;
    plan.outer_iters = 1;
    plan.pcg_iters = pcg_iters;
    plan.sigma_gm = 1.0f;
    return run(g, inst, plan, (cudaStream_t)stream);
}

fbs_status fbs_set_option(fbs_grid* g, int option, int value)
{
    if (!g) return FBS_ERR_ARG;
    if (option == FBS_OPT_VECTOR_PRECISION) {
        if (value < FBS_VECTORS_AUTO || value > FBS_VECTORS_COMPENSATED) return FBS_ERR_ARG;
        g->precision = value;
        return FBS_OK;
    }
    if (option == FBS_OPT_INJECT_BARRIER_TIMEOUT) {
        if (value != 0 && value != 1) return FBS_ERR_ARG;
        g->inject_timeout = value;
        return FBS_OK;
    }
    if (option == FBS_OPT_PRECONDITIONER) {
        if (value != FBS_PRECOND_JACOBI && value != FBS_PRECOND_HIERARCHICAL) return FBS_ERR_ARG;
        g->precond = value;
        return FBS_OK;
    }
    if (option == FBS_OPT_PHASE_BLOCKS) {
        if (value != 1 && value != 2 && value != 4) return FBS_ERR_ARG;
        g->phase_blocks = value;
        return FBS_OK;
    }
    if (option == FBS_OPT_TUNE_SINGLE_SOLVE) {
        if (value != 0 && value != 1) return FBS_ERR_ARG;
        g->tune_single = value;
        return FBS_OK;
    }
    if (option == FBS_OPT_PCG_FORM) {
        if (value != FBS_PCG_FORM_STANDARD && value != FBS_PCG_FORM_SINGLE) return FBS_ERR_ARG;
        g->pcg_form = value;
        return FBS_OK;
    }
    if (option == FBS_OPT_PCG_LAUNCH) {
        if (value != FBS_PCG_AUTO && value != FBS_PCG_PERSISTENT && value != FBS_PCG_PER_PHASE)
            return FBS_ERR_ARG;
        g->persistent = value == FBS_PCG_PER_PHASE ? 0 : 1;
        g->force_persistent = value == FBS_PCG_PERSISTENT ? 1 : 0;
        return FBS_OK;
    }
    return FBS_ERR_ARG;
}

fbs_status fbs_autotune(fbs_grid* g, const fbs_problem_desc* probs, int pcg_iters, void* stream,
                        fbs_tune_result* out)
{
    if (!g) return FBS_ERR_ARG;
    fbs_status st = check_problems(g, probs, pcg_iters);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (capturing(s)) return FBS_ERR_STATE;
    struct Cand {
        int launch, form, blocks;
    };
    const Cand cands[] = {{FBS_PCG_PER_PHASE, FBS_PCG_FORM_STANDARD, 1},
                          {FBS_PCG_PER_PHASE, FBS_PCG_FORM_STANDARD, 2},
                          {FBS_PCG_PER_PHASE, FBS_PCG_FORM_STANDARD, 4},
                          {FBS_PCG_PER_PHASE, FBS_PCG_FORM_SINGLE, 1},
                          {FBS_PCG_PER_PHASE, FBS_PCG_FORM_SINGLE, 2},
                          {FBS_PCG_PERSISTENT, FBS_PCG_FORM_STANDARD, 1},
                          {FBS_PCG_PERSISTENT, FBS_PCG_FORM_SINGLE, 1}};
    const int n = (int)(sizeof(cands) / sizeof(cands[0]));
    const int saved_persistent = g->persistent, saved_force = g->force_persistent,
              saved_form = g->pcg_form, saved_blocks = g->phase_blocks;
    cudaEvent_t ev[4];
    for (int k = 0; k < 4; ++k)
        if (cudaEventCreate(&ev[k]) != cudaSuccess) return FBS_ERR_CUDA;
    int best = -1;
    float best_ms = 0.0f;
    for (int c = 0; c < n && !st; ++c) {
        g->persistent = cands[c].launch == FBS_PCG_PER_PHASE ? 0 : 1;
        g->force_persistent = cands[c].launch == FBS_PCG_PERSISTENT ? 1 : 0;
        g->pcg_form = cands[c].form;
        g->phase_blocks = cands[c].blocks;
        // single-solve timing: drop the graphs (after the work that may use
        // them has finished) so that each solve is a grid's first
        auto drop_graphs = [&]() {
            if (!g->tune_single) return;
            if (cudaStreamSynchronize(s) != cudaSuccess) st = FBS_ERR_CUDA;
            free_graphs(g);
        };
        for (int w = 0; w < 2 && !st; ++w) {
            drop_graphs();
            if (!st) st = fbs_solve(g, probs, pcg_iters, stream);
        }
        float t[3] = {0.0f, 0.0f, 0.0f};
        for (int r = 0; r < 3 && !st; ++r) {
            drop_graphs();
            if (cudaEventRecord(ev[0], s) != cudaSuccess) st = FBS_ERR_CUDA;
            if (!st) st = fbs_solve(g, probs, pcg_iters, stream);
            if (!st && cudaEventRecord(ev[1], s) != cudaSuccess) st = FBS_ERR_CUDA;
            if (!st && cudaEventSynchronize(ev[1]) != cudaSuccess) st = FBS_ERR_CUDA;
            if (!st && cudaEventElapsedTime(&t[r], ev[0], ev[1]) != cudaSuccess) st = FBS_ERR_CUDA;
        }
        if (st) break;
        std::sort(t, t + 3);
        if (best < 0 || t[1] < best_ms) {
            best = c;
            best_ms = t[1];
        }
    }
    for (int k = 0; k < 4; ++k) cudaEventDestroy(ev[k]);
    if (st || best < 0) {
        g->persistent = saved_persistent;
        g->force_persistent = saved_force;
        g->pcg_form = saved_form;
        g->phase_blocks = saved_blocks;
        return st ? st : FBS_ERR_STATE;
    }
    g->persistent = cands[best].launch == FBS_PCG_PER_PHASE ? 0 : 1;
    g->force_persistent = cands[best].launch == FBS_PCG_PERSISTENT ? 1 : 0;
    g->pcg_form = cands[best].form;
    g->phase_blocks = cands[best].blocks;
    st = fbs_solve(g, probs, pcg_iters, stream);
    if (out) {
        out->pcg_launch = cands[best].launch;
        out->pcg_form = cands[best].form;
        out->phase_blocks = cands[best].blocks;
        out->solve_ms = best_ms;
        out->candidates = n;
    }
    return st;
}

fbs_status fbs_grid_info(const fbs_grid* g, int image, int64_t* n_vertices, int64_t* vertex_offset)
{
    if (!g || image < 0 || image >= g->n_images) return FBS_ERR_ARG;
    if (n_vertices) *n_vertices = g->voff[image + 1] - g->voff[image];
    if (vertex_offset) *vertex_offset = g->voff[image];
    return FBS_OK;
}

fbs_status fbs_grid_export(const fbs_grid* g, int image, void* stream, uint64_t* host_keys,
                           uint32_t* host_vid, uint32_t* host_counts, int32_t* host_nbr,
                           double* host_n)
{
    if (!g || image < 0 || image >= g->n_images) return FBS_ERR_ARG;
    if (host_n && g->bistoch_iters < 1) return FBS_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t v0 = g->voff[image], V = g->voff[image + 1] - v0;
    const int64_t p0 = g->img[image].pix_base;
    const int64_t N = (int64_t)g->img[image].H * g->img[image].W;
    cudaError_t e = cudaSuccess;
    if (host_keys && e == cudaSuccess)
        e = cudaMemcpyAsync(host_keys, g->vkey + v0, V * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    if (host_vid && e == cudaSuccess)
        e = cudaMemcpyAsync(host_vid, g->vid + p0, N * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (host_counts && e == cudaSuccess)
        e = cudaMemcpyAsync(host_counts, g->m + v0, V * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    std::vector<int32_t> soa;
    if (host_nbr && e == cudaSuccess) {
        soa.resize((size_t)V * 10);
        for (int k = 0; k < 10 && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(soa.data() + (size_t)k * V, g->nbr + (size_t)k * g->nbr_stride + v0,
                                V * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    }
    if (host_n && e == cudaSuccess)
        e = cudaMemcpyAsync(host_n, g->n64 + v0, V * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    if (host_vid)
        for (int64_t i = 0; i < N; ++i) host_vid[i] = (uint32_t)(host_vid[i] - v0);
    if (host_nbr)
        for (int64_t v = 0; v < V; ++v)
            for (int k = 0; k < 10; ++k) {
                const int32_t u = soa[(size_t)k * V + v];
                host_nbr[v * 10 + k] = u >= 0 ? (int32_t)(u - v0) : -1;
            }
    return FBS_OK;
}

fbs_status fbs_pyramid_export(fbs_grid* g, int image, int level, void* stream, int* levels,
                              int64_t* n_vertices, uint64_t* host_keys, int32_t* host_parent,
                              float* host_count)
{
    if (!g || image < 0 || image >= g->n_images || level < 0) return FBS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->pyr_K == 0) {
        if (capturing(s)) return FBS_ERR_STATE;
        const fbs_status st = build_pyramid(g, s);
        if (st) return st;
    }
    const int K = g->pyr_K, n = g->n_images;
    if (levels) *levels = K;
    if (level >= K) return FBS_ERR_ARG;
    const int64_t g0 = g->pyr_ioff_host[(size_t)level * (n + 1) + image];
    const int64_t nv = g->pyr_ioff_host[(size_t)level * (n + 1) + image + 1] - g0;
    if (n_vertices) *n_vertices = nv;
    cudaError_t e = cudaSuccess;
    if (host_keys)
        e = cudaMemcpyAsync(host_keys, g->pyr_key + g0, nv * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    if (host_count && e == cudaSuccess)
        e = cudaMemcpyAsync(host_count, g->pyr_cnt + g0, nv * sizeof(float), cudaMemcpyDeviceToHost, s);
    const bool top = level + 1 >= K;
    if (host_parent && !top && e == cudaSuccess)
        e = cudaMemcpyAsync(host_parent, g->pyr_parent + g0, nv * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    if (host_parent) {
        // level-local ids of level + 1 -> indices within the image's range there
        const int64_t base = top ? 0
                                 : g->pyr_ioff_host[(size_t)(level + 1) * (n + 1) + image] -
                                       g->pyr_off[level + 1];
        for (int64_t i = 0; i < nv; ++i)
            host_parent[i] = top ? -1 : (int32_t)(host_parent[i] - base);
    }
    return FBS_OK;
}

fbs_status fbs_grid_sync(fbs_grid* g, void* stream)
{
    if (!g) return FBS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t bits = 0;
    cudaError_t e = cudaMemcpyAsync(&bits, g->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    if (bits) {
        cudaMemsetAsync(g->err, 0, sizeof(uint32_t), s);
        cudaStreamSynchronize(s);
    }
    return latched(bits);
}

fbs_status fbs_grid_destroy(fbs_grid* g, void* stream)
{
    if (!g) return FBS_ERR_ARG;
    free_grid_memory(g, (cudaStream_t)stream);
    delete g;
    return FBS_OK;
}

fbs_status fbs_profile_enable(int on)
{
    if (on < 0 || on > 2) return FBS_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_level = on;
    for (auto& f : families()) {
        for (auto& p : f.pending) {
            event_pool().push_back(p.first);
            event_pool().push_back(p.second);
        }
        f.pending.clear();
        f.launches = 0;
        f.ms = 0.0;
        if (f.open) {
            event_pool().push_back(f.open);
            f.open = nullptr;
        }
    }
    return FBS_OK;
}

fbs_status fbs_profile_read(int* count, const char** names, int64_t* launches, double* total_ms)
{
    if (!count) return FBS_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    auto& fams = families();
    for (auto& f : fams) {
        for (auto& p : f.pending) {
            if (cudaEventSynchronize(p.second) != cudaSuccess) return FBS_ERR_CUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p.first, p.second);
            f.ms += ms;
            f.launches += 1;
            event_pool().push_back(p.first);
            event_pool().push_back(p.second);
        }
        f.pending.clear();
    }
    const int n = std::min<int>(*count, (int)fams.size());
    for (int i = 0; i < n; ++i) {
        if (names) names[i] = fams[i].name.c_str();
        if (launches) launches[i] = fams[i].launches;
        if (total_ms) total_ms[i] = fams[i].ms;
    }
    *count = (int)fams.size();
    return FBS_OK;
}

}  // extern "C"

#include "grid_view.cuh"

namespace fbs {

bool grid_view(const fbs_grid* g, GridView* out)
{
    if (!g || !out) return false;
    out->n_images = g->n_images;
    out->Vtot = g->Vtot;
    out->max_pixels = g->max_pixels;
    out->nvt = g->nvt;
    out->bistoch_iters = g->bistoch_iters;
    out->precision = g->precision;
    out->persistent = g->persistent;
    out->force_persistent = g->force_persistent;
    out->phase_blocks = g->phase_blocks;
    out->img = g->img.data();
    out->voff = g->voff.data();
    out->vt0 = g->vt0.data();
    out->nvt_img = g->nvt_img.data();
    out->vt = g->vt;
    out->nbr = g->nbr;
    out->nbr_stride = g->nbr_stride;
    out->nbrp = g->nbrp;
    out->n64 = g->n64;
    out->nf = g->nf;
    out->m = g->m;
    out->pstart = g->pstart;
    out->perm = g->perm;
    out->vid = g->vid;
    out->err = g->err;
    return true;
}

}  // namespace fbs
