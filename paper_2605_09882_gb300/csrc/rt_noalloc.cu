// Forward trace for callers that cannot allocate device memory.
//
// rt_trace_columns needs an rt_octree handle, and building one allocates (the
// coarse table, the statistics block) as does the first use of an nside (the
// direction table).  Some callers cannot do that: an application whose memory
// pool owns all of the device memory, or code that must not call cudaMalloc /
// cudaFree because they can synchronize the whole device in the middle of its
// stream work.  rt_trace_columns_noalloc runs the same forward kernel on a raw
// octree with all of its scratch (work-queue counter, statistics and status,
// the root lookup entry and the direction table) in one file-scope device
// array of fixed size, so the call itself allocates nothing.
#include <stddef.h>

#include <mutex>

#include "rt_host.h"

namespace rt {

// Largest direction table the static scratch holds: nside <= 8 (768 rays).
constexpr int kNoAllocMaxNside = 8;
constexpr int kNoAllocMaxDirs = 12 * kNoAllocMaxNside * kNoAllocMaxNside;

struct NoAllocScratch {
    DevStats stats;                 // queue counter, counters, status
    uint64_t root_entry;            // one-entry lookup table (level-0 cell)
    uint64_t pad[7];
    DirConst dirs[kNoAllocMaxDirs];
};

// The scratch of every call on this device (about 74 KiB, held until exit).
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Host sources of what every call uploads: one direction table per nside
// (index log2 nside), each computed on its first use and never changed after,
// and the possible one-entry lookup tables (entry l: the cube is one uniform
// level l, entry 22: search all keys).  Static storage, so staging allocates
// nothing either; the mutex serializes the host-side preparation.
static DirConst g_dirs_stage[4][kNoAllocMaxDirs];
static bool g_dirs_ready[4];
static double g_dirs_host[3 * kNoAllocMaxDirs];
static const uint64_t kRootEntries[23] = {0,  1,  2,  3,  4,  5,  6,  7,  8,  9,  10, 11,
                                          12, 13, 14, 15, 16, 17, 18, 19, 20, 21, (uint64_t)kCodeMixed};
static std::mutex g_noalloc_mu;
static NoAllocScratch* g_noalloc_ptr[64];  // device address of the array, per device

// Device address of the scratch for `dev` (the current device); looked up
// once per device with cudaGetSymbolAddress.
static NoAllocScratch* noalloc_scratch(int dev, int* status)
{
    if (dev < 0 || dev >= 64) {
        *status = set_error(RT_ERR_ARG, "rt_trace_columns_noalloc: device index out of range");
        return nullptr;
    }
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            *status = cuda_error("rt_trace_columns_noalloc: cudaGetSymbolAddress");
            return nullptr;
        }
        g_noalloc_ptr[dev] = (NoAllocScratch*)p;
    }
    return g_noalloc_ptr[dev];
}

// The direction constants of nside (1, 2, 4 or 8), computed once.
static const DirConst* staged_directions(int nside)
{
    const int l = nside == 1 ? 0 : nside == 2 ? 1 : nside == 4 ? 2 : 3;
    if (g_dirs_ready[l]) return g_dirs_stage[l];
    const int nd = 12 * nside * nside;
    rt_healpix_dirs(nside, g_dirs_host);
    for (int q = 0; q < nd; q++) {
        DirConst& d = g_dirs_stage[l][q];
        memset(&d, 0, sizeof d);
        for (int b = 0; b < 3; b++) {
            const double v = g_dirs_host[3 * q + b];
            d.m[b] = v;
            d.m32[b] = (float)v;
            if (v != 0.0) {
                d.inv[b] = 1.0 / v;
                d.ih[b] = (float)d.inv[b];
                d.il[b] = (float)(d.inv[b] - (double)d.ih[b]);
                d.flags |= 1 << b;
                if (v > 0.0) d.flags |= 8 << b;
            }
        }
        const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
        for (int k = 0; k < 3; k++)
            if ((d.flags & (1 << pa[k])) && (d.flags & (1 << pb[k])) &&
                fabs(d.inv[pa[k]]) == fabs(d.inv[pb[k]]))
                d.flags |= 1 << (6 + k);
    }
    g_dirs_ready[l] = true;
    return g_dirs_stage[l];
}

}  // namespace rt

using namespace rt;

extern "C" int rt_trace_columns_noalloc(const uint64_t* d_keys, const uint8_t* d_levels,
                                        int64_t n_leaves, const int32_t* h_extent, int max_level,
                                        const double* d_src, int64_t n_src, int nside,
                                        const void* d_dens, int n_species, int dens_dtype,
                                        int mode, void* d_out, rt_stats* h_stats, void* stream)
{
    if (!d_keys || !d_levels || n_leaves <= 0 || n_leaves >= (1ll << 32))
        return set_error(RT_ERR_ARG, "rt_trace_columns_noalloc: bad octree arrays");
    if (max_level < 0 || max_level > kDepth)
        return set_error(RT_ERR_ARG, "rt_trace_columns_noalloc: max_level outside [0, 21]");
    if (nside < 1 || nside > kNoAllocMaxNside || (nside & (nside - 1)))
        return set_error(RT_ERR_ARG, "rt_trace_columns_noalloc: nside must be 1, 2, 4 or 8 "
                                     "(the fixed scratch holds at most 768 directions)");
    if (n_species < 1 || n_species > kMaxSpecies)
        return set_error(RT_ERR_ARG, "rt_trace_columns_noalloc: n_species must be in [1, 8]");
    if (mode != RT_MODE_FP64 && mode != RT_MODE_F32_KAHAN)
        return set_error(RT_ERR_ARG, "rt_trace_columns_noalloc: unknown mode");
    if (dens_dtype != RT_F32 && dens_dtype != RT_F64)
        return set_error(RT_ERR_ARG, "rt_trace_columns_noalloc: bad dens_dtype");
    if (n_src < 0 || (n_src > 0 && (!d_src || !d_dens || !d_out)))
        return set_error(RT_ERR_ARG, "rt_trace_columns_noalloc: bad sources, densities or output");
    if (((uintptr_t)d_dens & 15u) || ((uintptr_t)d_out & 15u))
        return set_error(RT_ERR_ARG, "rt_trace_columns_noalloc: densities and output must be 16-byte aligned");
    uint32_t ext[3];
    for (int b = 0; b < 3; b++) {
        const int32_t e = h_extent ? h_extent[b] : (1 << kDepth);
        if (e <= 0 || e > (1 << kDepth))
            return set_error(RT_ERR_ARG, "rt_trace_columns_noalloc: extent outside [1, 2^21]");
        ext[b] = (uint32_t)e;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, status = RT_OK;
    cudaGetDevice(&dev);
    const int nd = 12 * nside * nside;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocScratch* sc = noalloc_scratch(dev, &status);
    if (!sc) return status;

    const bool full = ext[0] == (1u << kDepth) && ext[1] == (1u << kDepth) && ext[2] == (1u << kDepth);
    const bool uniform = full && max_level <= 10 && n_leaves == (int64_t)(1ll << (3 * max_level));
    // zeroed statistics, the level-0 lookup entry (O(1) index of a uniform
    // cube, else a key search over all leaves) and the directions, copied from
    // host data that never changes once computed
    if (cudaMemsetAsync(&sc->stats, 0, sizeof(DevStats), s) != cudaSuccess ||
        cudaMemcpyAsync(&sc->root_entry, &kRootEntries[uniform ? max_level : 22], sizeof(uint64_t),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(sc->dirs, staged_directions(nside), sizeof(DirConst) * nd, cudaMemcpyHostToDevice,
                        s) != cudaSuccess)
        return cuda_error("rt_trace_columns_noalloc: scratch upload");

    TraceArgs a;
    memset(&a, 0, sizeof a);
    a.t.keys = d_keys;
    a.t.levels = d_levels;
    a.t.table = &sc->root_entry;
    a.t.n = n_leaves;
    for (int b = 0; b < 3; b++) a.t.ext[b] = ext[b];
    a.t.T = 0;
    a.t.uniform_level = uniform ? max_level : -1;
    a.t.lmax = max_level;
    a.t.step_cap = 3 * (1ll << max_level) + 3;
    a.dirs = sc->dirs;
    a.nd = nd;
    a.src = d_src;
    a.n_src = n_src;
    a.n_src_pad = (n_src + 31) / 32 * 32;
    a.dens = d_dens;
    a.dens_f64 = dens_dtype == RT_F64;
    a.S = n_species;
    a.out = d_out;
    a.st = &sc->stats;
    // the launch shape and ray order of rt_trace_columns
    int block, bps, groups;
    launch_shape(&block, &bps, &groups);
    a.batch = groups;
    a.layout = ray_layout(n_src);
    if (n_src > 0) {
        const int fit = std::max(1, occupancy_fwd(0, mode, n_species, uniform, block));
        const int per_sm = bps > 0 ? std::min(bps, fit) : fit;
        if (launch_forward(a, mode, block, sm_count_of(dev) * per_sm, s) != cudaSuccess)
            return cuda_error("rt_trace_columns_noalloc: launch");
    }
    if (h_stats) {
        DevStats d;
        if (cudaMemcpyAsync(&d, &sc->stats, sizeof d, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return cuda_error("rt_trace_columns_noalloc: statistics readback");
        h_stats->rays = d.rays;
        h_stats->segments = d.segments;
        h_stats->exit_fallbacks = d.exit_fb;
        h_stats->lookup_fallbacks = d.lookup_fb;
        h_stats->status = d.status;
        h_stats->gathered = 0;
        h_stats->fault_ray = d.status ? d.fault_ray : -1;
    }
    clear_error();
    return RT_OK;
}
