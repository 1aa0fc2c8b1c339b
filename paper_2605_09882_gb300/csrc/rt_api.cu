// Public C ABI: argument checks, direction tables, launches, statistics.
#include <stdio.h>
#include <stdlib.h>

#include <mutex>
#include <string>

#include "rt_host.h"

namespace rt {

static thread_local std::string g_err;

int set_error(int code, const char* msg)
{
    g_err = msg;
    return code;
}

int cuda_error(const char* where)
{
    const cudaError_t e = cudaGetLastError();
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    g_err = buf;
    return (e == cudaErrorMemoryAllocation) ? RT_ERR_OOM : RT_ERR_CUDA;
}

void clear_error() { g_err.clear(); }

// ----------------------------------------------------------- launch shape

static int g_block = 256;
static int g_blocks_per_sm = 0;
static int g_batch = 4;
static int g_table_cap = -1;

int table_level_cap() { return g_table_cap; }

struct DeviceInfo {
    int sms = 0;
};
static std::mutex g_mu;
static DeviceInfo g_dev[64];
static DirConst* g_dirs[64][11];  // per device, per log2(nside); never freed

static int sm_count(int dev)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 64) return 0;
    if (!g_dev[dev].sms) cudaDeviceGetAttribute(&g_dev[dev].sms, cudaDevAttrMultiProcessorCount, dev);
    return g_dev[dev].sms;
}

static int ilog2_pow2(int v)
{
    int l = 0;
    while ((1 << l) < v) l++;
    return ((1 << l) == v) ? l : -1;
}

// Per-direction constants of the HEALPix table for nside, in device memory
// (uploaded on first use per device, kept until process exit).
static const DirConst* dir_table(int dev, int nside, int* status)
{
    const int l = ilog2_pow2(nside);
    if (nside < 1 || nside > 1024 || l < 0) {
        *status = set_error(RT_ERR_ARG, "nside must be a power of two in [1, 1024]");
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 64) {
        *status = set_error(RT_ERR_ARG, "device index out of range");
        return nullptr;
    }
    if (g_dirs[dev][l]) return g_dirs[dev][l];
    const int nd = 12 * nside * nside;
    double* m = (double*)malloc(sizeof(double) * 3 * nd);
    DirConst* h = (DirConst*)calloc(nd, sizeof(DirConst));
    rt_healpix_dirs(nside, m);
    for (int q = 0; q < nd; q++) {
        DirConst& d = h[q];
        d.flags = 0;
        for (int b = 0; b < 3; b++) {
            const double v = m[3 * q + b];
            d.m[b] = v;
            d.m32[b] = (float)v;
            if (v != 0.0) {
                d.inv[b] = 1.0 / v;
                d.ih[b] = (float)d.inv[b];
                d.il[b] = (float)(d.inv[b] - (double)d.ih[b]);
                d.flags |= 1 << b;
                if (v > 0.0) d.flags |= 8 << b;
            } else {
                d.inv[b] = 0.0;
                d.ih[b] = d.il[b] = 0.f;
            }
        }
        const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
        for (int k = 0; k < 3; k++)
            if ((d.flags & (1 << pa[k])) && (d.flags & (1 << pb[k])) && fabs(d.inv[pa[k]]) == fabs(d.inv[pb[k]]))
                d.flags |= 1 << (6 + k);
    }
    DirConst* dptr = nullptr;
    if (cudaMalloc(&dptr, sizeof(DirConst) * nd) != cudaSuccess ||
        cudaMemcpy(dptr, h, sizeof(DirConst) * nd, cudaMemcpyHostToDevice) != cudaSuccess) {
        *status = cuda_error("direction table upload");
        if (dptr) cudaFree(dptr);
        dptr = nullptr;
    } else {
        g_dirs[dev][l] = dptr;
    }
    free(m);
    free(h);
    return dptr;
}

void launch_shape(int* block, int* blocks_per_sm, int* groups_per_pop)
{
    *block = g_block;
    *blocks_per_sm = g_blocks_per_sm;
    *groups_per_pop = g_batch;
}

const DirConst* direction_table(int dev, int nside, int* status) { return dir_table(dev, nside, status); }

int sm_count_of(int dev) { return sm_count(dev); }

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Common argument handling of the trace entry points.
int prepare_trace(const rt_octree* t, const double* d_src, int64_t n_src, int nside, int S,
                   int mode, TraceArgs& a, const char* who)
{
    char buf[256];
    if (!t) {
        snprintf(buf, sizeof buf, "%s: null octree", who);
        return set_error(RT_ERR_ARG, buf);
    }
    if (n_src < 0 || (n_src > 0 && !d_src)) {
        snprintf(buf, sizeof buf, "%s: bad sources", who);
        return set_error(RT_ERR_ARG, buf);
    }
    if (S < 1 || S > kMaxSpecies) {
        snprintf(buf, sizeof buf, "%s: n_species must be in [1, %d]", who, kMaxSpecies);
        return set_error(RT_ERR_ARG, buf);
    }
    if (mode != RT_MODE_FP64 && mode != RT_MODE_F32_KAHAN) {
        snprintf(buf, sizeof buf, "%s: unknown mode", who);
        return set_error(RT_ERR_ARG, buf);
    }
    int status = RT_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != t->device) return set_error(RT_ERR_ARG, "octree was built on another device");
    const DirConst* dirs = dir_table(dev, nside, &status);
    if (!dirs) return status;
    memset(&a, 0, sizeof a);
    a.t = t->dev;
    if (!t->uniform_allowed) a.t.uniform_level = -1;
    a.dirs = dirs;
    a.nd = 12 * nside * nside;
    a.src = d_src;
    a.n_src = n_src;
    a.n_src_pad = (n_src + 31) / 32 * 32;
    a.S = S;
    a.st = t->st;
    a.batch = g_batch;
    a.layout = ray_layout(n_src);
    a.dgroup = 1;
    return RT_OK;
}

// Directions per group of the forward's direction-major order on a uniform
// cube: the most whose columns of one source fit in RT_DGROUP_BYTES (a divisor
// of nd).  At 64 bytes (4 directions of 4 FP32 species) a warp writes whole
// 64-byte DRAM bursts of every source row it touches, and the rest of the
// walk keeps its direction-major sweep (measured at 512^3, 4 species: 32 bytes
// 904.6 ms, 64 bytes 893.9 ms, a whole 192-byte row 901.3 ms per trace).  On
// general octrees the groups were slower (the differentiable workload's
// forward 12.4 -> 15.0 ms, the 64-cloud batch 1163 -> 1775 ms).
#ifndef RT_DGROUP_BYTES
#define RT_DGROUP_BYTES 64
#endif
static int output_dgroup(int nd, int S, int mode)
{
    const int row = S * (mode == RT_MODE_FP64 ? 8 : 4);
    int D = std::max(1, std::min(nd, RT_DGROUP_BYTES / row));
    while (D > 1 && nd % D) D--;
    return D;
}

static int grid_for(int blocks_per_sm_fit)
{
    int dev = 0;
    cudaGetDevice(&dev);
    int bps = g_blocks_per_sm > 0 ? std::min(g_blocks_per_sm, blocks_per_sm_fit) : blocks_per_sm_fit;
    if (bps < 1) bps = 1;
    return sm_count(dev) * bps;
}

}  // namespace rt

using namespace rt;

extern "C" {

const char* rt_last_error(void) { return g_err.c_str(); }

void rt_destroy_octree(rt_octree* t)
{
    if (!t) return;
    cudaDeviceSynchronize();
    if (t->table) cudaFree(t->table);
    if (t->st) cudaFree(t->st);
    if (t->adj_tab) cudaFree(t->adj_tab);
    free(t);
}

int rt_set_launch(int threads_per_block, int blocks_per_sm, int groups_per_pop)
{
    if (threads_per_block == 0) threads_per_block = 256;
    if (groups_per_pop == 0) groups_per_pop = 4;
    if (threads_per_block < 32 || threads_per_block > 256 || threads_per_block % 32)
        return set_error(RT_ERR_ARG, "rt_set_launch: threads_per_block must be a multiple of 32 in [32, 256]");
    if (blocks_per_sm < 0) return set_error(RT_ERR_ARG, "rt_set_launch: blocks_per_sm < 0");
    if (groups_per_pop < 1 || groups_per_pop > 64)
        return set_error(RT_ERR_ARG, "rt_set_launch: groups_per_pop must be in [1, 64]");
    g_block = threads_per_block;
    g_blocks_per_sm = blocks_per_sm;
    g_batch = groups_per_pop;
    return RT_OK;
}

int rt_set_step_cap(rt_octree* t, int64_t cap)
{
    if (!t || cap < 0) return set_error(RT_ERR_ARG, "rt_set_step_cap: bad argument");
    t->dev.step_cap = cap ? cap : t->default_cap;
    return RT_OK;
}

int rt_set_table_cap(int max_level)
{
    if (max_level < -1 || max_level > kMaxTableLevel)
        return set_error(RT_ERR_ARG, "rt_set_table_cap: max_level must be -1 or in [0, 10]");
    g_table_cap = max_level;
    return RT_OK;
}

int rt_set_lookup(rt_octree* t, int use_uniform_index)
{
    if (!t) return set_error(RT_ERR_ARG, "rt_set_lookup: null octree");
    t->uniform_allowed = use_uniform_index ? 1 : 0;
    return RT_OK;
}

int rt_octree_info(const rt_octree* t, int64_t* n_leaves, int* max_level, int* uniform_level)
{
    if (!t) return set_error(RT_ERR_ARG, "rt_octree_info: null octree");
    if (n_leaves) *n_leaves = t->dev.n;
    if (max_level) *max_level = t->dev.lmax;
    if (uniform_level) *uniform_level = t->dev.uniform_level;
    return RT_OK;
}

int rt_trace_columns(const rt_octree* t, const double* d_src, int64_t n_src, int nside,
                     const void* d_dens, int n_species, int dens_dtype, int mode, void* d_out,
                     void* stream)
{
    return trace_columns_impl(t, d_src, n_src, nside, d_dens, n_species, dens_dtype, mode, d_out, stream, true);
}

}  // extern "C"

int rt::trace_columns_impl(const rt_octree* t, const double* d_src, int64_t n_src, int nside, const void* d_dens,
                           int n_species, int dens_dtype, int mode, void* d_out, void* stream, bool check)
{
    TraceArgs a;
    int st = prepare_trace(t, d_src, n_src, nside, n_species, mode, a, "rt_trace_columns");
    if (st != RT_OK) return st;
    if (dens_dtype != RT_F32 && dens_dtype != RT_F64) return set_error(RT_ERR_ARG, "rt_trace_columns: bad dens_dtype");
    if (n_src == 0) return RT_OK;
    if (!d_dens || !d_out) return set_error(RT_ERR_ARG, "rt_trace_columns: null densities or output");
    if (!aligned16(d_dens) || !aligned16(d_out))
        return set_error(RT_ERR_ARG, "rt_trace_columns: densities and output must be 16-byte aligned");
    a.dens = d_dens;
    a.dens_f64 = dens_dtype == RT_F64;
    a.out = d_out;
    cudaStream_t s = (cudaStream_t)stream;
    if (check) {
        const int cs = check_densities(d_dens, t->dev.n, n_species, a.dens_f64, 0, t->st, s);
        if (cs != RT_OK) return cs;
    }
    // (a general octree keeps one direction per pop: there the direction-major
    // sweep's L2 reuse of the walk outweighs the output's partial bursts)
    if (a.t.uniform_level >= 0) a.dgroup = output_dgroup(a.nd, n_species, mode);
    // leaf centres of a uniform cube share their exit sequences: two rays per
    // lane (FP32 densities with 1, 2, 4 or 8 species, direction-major order)
    a.pair = mode == RT_MODE_F32_KAHAN && a.t.uniform_level >= 0 && a.layout == 0 && !a.dens_f64 &&
             (n_species == 1 || n_species == 2 || n_species == 4 || n_species == 8);
    if (a.pair) a.n_src_pad = (n_src + 63) / 64 * 64;
    const int fit = a.pair ? occupancy_pair(n_species, g_block)
                           : occupancy_fwd(0, mode, n_species, a.t.uniform_level >= 0, g_block);
    if (cudaMemsetAsync(&t->st->queue, 0, sizeof(unsigned long long), s) != cudaSuccess)
        return cuda_error("rt_trace_columns: queue reset");
    if (launch_forward(a, mode, g_block, grid_for(fit), s) != cudaSuccess)
        return cuda_error("rt_trace_columns: launch");
    return RT_OK;
}

extern "C" {

int rt_trace_paths(const rt_octree* t, const double* d_src, int64_t n_src, int nside, int mode,
                   uint32_t* d_nseg, uint64_t* d_hash, void* stream)
{
    TraceArgs a;
    int st = prepare_trace(t, d_src, n_src, nside, 1, mode, a, "rt_trace_paths");
    if (st != RT_OK) return st;
    if (n_src == 0) return RT_OK;
    a.nseg = d_nseg;
    a.hash = d_hash;
    cudaStream_t s = (cudaStream_t)stream;
    const int fit = occupancy_fwd(1, mode, 1, a.t.uniform_level >= 0, g_block);
    if (cudaMemsetAsync(&t->st->queue, 0, sizeof(unsigned long long), s) != cudaSuccess)
        return cuda_error("rt_trace_paths: queue reset");
    if (launch_paths(a, mode, g_block, grid_for(fit), s) != cudaSuccess)
        return cuda_error("rt_trace_paths: launch");
    return RT_OK;
}

int rt_get_stats(const rt_octree* t, rt_stats* h_out, void* stream)
{
    if (!t || !h_out) return set_error(RT_ERR_ARG, "rt_get_stats: null argument");
    DevStats d;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&d, t->st, sizeof d, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return cuda_error("rt_get_stats");
    h_out->rays = d.rays;
    h_out->segments = d.segments;
    h_out->exit_fallbacks = d.exit_fb;
    h_out->lookup_fallbacks = d.lookup_fb;
    h_out->status = d.status;
    h_out->gathered = d.gathered;
    h_out->fault_ray = d.status ? d.fault_ray : -1;
    return RT_OK;
}

int rt_reset_stats(rt_octree* t, void* stream)
{
    if (!t) return set_error(RT_ERR_ARG, "rt_reset_stats: null octree");
    if (cudaMemsetAsync(t->st, 0, sizeof(DevStats), (cudaStream_t)stream) != cudaSuccess)
        return cuda_error("rt_reset_stats");
    return RT_OK;
}

}  // extern "C"
