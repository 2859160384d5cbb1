// fbs_solve_static: the forward solve of fbs_solve for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc / cudaMallocAsync is not an
// option -- for example a host that hands the library a fixed memory budget
// up front, a real-time loop that must not hit an allocator (or its
// implicit synchronisation) between frames, or an embedding runtime whose
// own allocator owns all device memory.  fbs_solve sizes and allocates its
// workspace on first use; this entry point instead takes every piece of
// scratch from one array compiled into the library, so a solve allocates
// nothing at all.  The grid (fbs_grid_build) and every input and output
// buffer are still the caller's.
//
// The scratch array is a file-scope __device__ variable of
// kStaticScratchBytes; every GPU that loads the library holds it until the
// process exits.  Host code cannot use the array's name as a device address,
// so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it; that first
// call should therefore come before any stream capture.  All calls share the
// array and it keeps the last call's contents, so calls whose work overlaps
// on the GPU (different streams, or different grids at the same time) race:
// serialise them.
#include <map>
#include <mutex>
#include <string.h>
#include <vector>

#include "fbs_internal.cuh"
#include "grid_view.cuh"
#include "solve.cuh"

namespace fbs {
namespace {

constexpr size_t kStaticScratchBytes = 64ull << 20;   // 64 MiB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// device address of g_static_scratch on the current device (looked up once)
cudaError_t static_scratch(unsigned char** out)
{
    static std::mutex mu;
    static std::map<int, unsigned char*> addr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    auto it = addr.find(dev);
    if (it != addr.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr) return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    addr[dev] = static_cast<unsigned char*>(p);
    *out = static_cast<unsigned char*>(p);
    return cudaSuccess;
}

// byte offsets of the pieces of scratch, each 256-byte aligned
struct StaticLayout {
    size_t inst, vec, a, nm, scal, part, barrier, total;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

StaticLayout layout(int n_images, int64_t cv, int64_t Vtot, int pc, int64_t cpart)
{
    StaticLayout L;
    size_t o = 0;
    L.inst = o;    o = align256(o + sizeof(InstDev) * (size_t)n_images);
    L.vec = o;     o = align256(o + sizeof(float) * 8 * (size_t)cv);
    L.a = o;       o = align256(o + sizeof(float) * (size_t)Vtot);
    L.nm = o;      o = align256(o + sizeof(float2) * (size_t)Vtot);
    L.scal = o;    o = align256(o + sizeof(Scal) * (size_t)pc);
    L.part = o;    o = align256(o + sizeof(float2) * 4 * (size_t)cpart);
    L.barrier = o; o = align256(o + sizeof(unsigned) * kBarrierWords);
    L.total = o;
    return L;
}

// descriptors are copied in through kernel parameters (no staging buffer)
struct StaticChunk {
    unsigned char b[3968];
};
__global__ void static_upload_kernel(unsigned char* dst, StaticChunk c, int n)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = c.b[i];
}

}  // namespace
}  // namespace fbs

using namespace fbs;

extern "C" fbs_status fbs_solve_static(fbs_grid* g, const fbs_problem_desc* probs,
                                       int pcg_iters, void* stream)
{
    GridView G;
    if (!grid_view(g, &G) || !probs || pcg_iters < 0) return FBS_ERR_ARG;
    for (int k = 0; k < G.n_images; ++k) {
        const fbs_problem_desc& p = probs[k];
        if (!p.t || !p.c || p.channels < 1 || p.channels > kMaxChannels || !(p.lambda >= 0.f) ||
            !isfinite(p.lambda))
            return FBS_ERR_ARG;
    }
    if (G.bistoch_iters < 1) return FBS_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;

    // per-image descriptors and sizes, as fbs_solve lays them out
    std::vector<InstDev> inst(G.n_images);
    int64_t cv = 0, cpart = 0, max_cv = 0;
    int pc = 0, cmax = 1;
    for (int k = 0; k < G.n_images; ++k) {
        InstDev I;
        memset(&I, 0, sizeof(I));
        I.C = probs[k].channels;
        I.lam = probs[k].lambda;
        I.t = probs[k].t;
        I.c = probs[k].c;
        I.x = probs[k].x;
        I.yout = probs[k].y;
        I.voff = G.voff[k];
        I.V = (int)(G.voff[k + 1] - G.voff[k]);
        I.Cp = padded_channels(I.C);
        I.vec_base = cv;
        I.tile0 = G.vt0[k];
        I.ntiles = G.nvt_img[k];
        I.pc = pc;
        I.part_base = cpart;
        I.N = (int64_t)G.img[k].H * G.img[k].W;
        I.pix_base = G.img[k].pix_base;
        cv += ((int64_t)I.Cp * I.V + 31) / 32 * 32;  // 128-byte aligned image blocks
        cpart += (int64_t)I.C * I.ntiles;
        pc += I.C;
        cmax = cmax > I.C ? cmax : I.C;
        max_cv = max_cv > (int64_t)I.C * I.V ? max_cv : (int64_t)I.C * I.V;
        inst[k] = I;
    }
    const StaticLayout L = layout(G.n_images, cv, G.Vtot, pc, cpart);
    if (L.total > kStaticScratchBytes) return FBS_ERR_ARG;   // problem too large for the array

    unsigned char* base = nullptr;
    cudaError_t e = static_scratch(&base);
    if (e != cudaSuccess) return FBS_ERR_CUDA;

    const size_t bytes = inst.size() * sizeof(InstDev);
    const unsigned char* src = reinterpret_cast<const unsigned char*>(inst.data());
    for (size_t off = 0; off < bytes; off += sizeof(StaticChunk)) {
        StaticChunk c;
        const size_t n = bytes - off < sizeof(StaticChunk) ? bytes - off : sizeof(StaticChunk);
        memcpy(c.b, src + off, n);
        static_upload_kernel<<<1, 256, 0, s>>>(base + L.inst + off, c, (int)n);
    }
    // the only state a solve reads before writing it is the barrier (reset
    // by the PCG launch itself); clear it here too so no call depends on the
    // previous call's contents
    e = cudaMemsetAsync(base + L.barrier, 0, sizeof(unsigned) * kBarrierWords, s);
    if (e != cudaSuccess) return FBS_ERR_CUDA;

    float* vec = reinterpret_cast<float*>(base + L.vec);
    float2* part = reinterpret_cast<float2*>(base + L.part);
    SolveArgs A;
    memset(&A, 0, sizeof(A));
    A.vt = G.vt;
    A.nvt = G.nvt;
    A.inst = reinterpret_cast<const InstDev*>(base + L.inst);
    A.ninst = G.n_images;
    A.nbr = G.nbr;
    A.nbr_stride = G.nbr_stride;
    A.nbrp = G.nbrp;
    A.Vtot = G.Vtot;
    A.n64 = G.n64;
    A.m = G.m;
    A.pstart = G.pstart;
    A.perm = G.perm;
    A.vid = G.vid;
    A.a = reinterpret_cast<float*>(base + L.a);
    A.nm = reinterpret_cast<float2*>(base + L.nm);
    A.y = vec;
    A.r = vec + cv;
    A.rlo = vec + 2 * cv;
    A.d[0] = vec + 3 * cv;
    A.d[1] = vec + 4 * cv;
    A.q = vec + 5 * cv;
    A.aux[0] = vec + 6 * cv;
    A.aux[1] = vec + 7 * cv;
    A.scal = reinterpret_cast<Scal*>(base + L.scal);
    A.nscal = pc;
    A.part_rs[0] = part;
    A.part_rs[1] = part + cpart;
    A.part_dq = part + 2 * cpart;
    A.part_mu[0] = A.part_dq;
    A.part_mu[1] = part + 3 * cpart;
    A.err = G.err;

    SolvePlan P;
    memset(&P, 0, sizeof(P));
    P.mode = kSplatConfidence;
    P.outer_iters = 1;
    P.pcg_iters = pcg_iters;
    P.sigma_gm = 1.0f;
    P.chan_block = cmax < kChanBlock ? cmax : kChanBlock;
    P.cmax = cmax;
    P.max_pixels = G.max_pixels;
    P.max_cv = max_cv;
    for (int k = 0; k < G.n_images; ++k) P.export_y |= probs[k].y != nullptr;
    P.comp = G.precision == FBS_VECTORS_COMPENSATED ? 1 : 0;
    A.zq = P.comp ? nullptr : A.aux[0];
    A.nf = G.nf;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    P.persistent = G.persistent && cs == cudaStreamCaptureStatusNone ? 1 : 0;
    P.barrier = reinterpret_cast<unsigned*>(base + L.barrier);
    // the grid's launch options (fbs_set_option, fbs_autotune) as fbs_solve uses them
    P.block_mult = G.phase_blocks;
    P.force_persistent = G.force_persistent;
    if (P.persistent && !P.force_persistent && !resident_preferred(A, P)) P.persistent = 0;
    A.fin = P.persistent && resident_fits(A, P) ? 1 : 0;

    e = launch_segment(A, P, kSegSetup, kSplatConfidence, s);
    if (e == cudaSuccess) e = launch_segment(A, P, kSegLoop, kSplatConfidence, s);
    if (e == cudaSuccess) e = launch_segment(A, P, kSegOut, kSplatConfidence, s);
    return e == cudaSuccess ? FBS_OK : FBS_ERR_CUDA;
}
