// Recorded paths: the (leaf, ds) sequence of every ray stored once, then the
// forward columns (a sparse product sum_j n[j] ds) and the adjoint (its
// transpose) evaluated from the record without walking again.  Useful when
// the same geometry is traced many times (finite differences, optimisation
// loops) and the record fits in memory (about 8 bytes per segment in
// F32-Kahan mode, 12 in FP64 mode).
//
// Layout: rays are grouped 32 at a time as the trace kernels walk them (32
// neighbouring sources, one direction); the group gets 32 * L slots, L its
// longest path, and segment k of lane i sits at slot off[g] + 32 k + i, so
// recording and replay both read and write whole sectors per warp.
#include <cub/cub.cuh>

#include "rt_host.h"
#include "rt_kernels.cuh"

namespace rt {

struct PathArgs {
    const long long* off;   // [n_groups + 1] slot offsets
    const uint32_t* nseg;   // [n_src * nd] segments per ray
    const uint32_t* leaf;   // [slots]
    const void* ds;         // [slots] float (F32-Kahan) or double (FP64)
    const void* dens;       // forward: densities
    const void* gin;        // adjoint: gradient of the columns
    void* out;              // forward: columns; adjoint: gradient of the densities (double)
    long long n_groups, gq, n_src;
    int nd, S, dens_f64, layout;
};

// Ray of lane `lane` in 32-ray group g of either ray order; false past the end.
__device__ __forceinline__ bool group_ray(long long g, int lane, long long gq, long long n_src, int nd, int layout,
                                          long long& ray)
{
    if (layout == 0) {
        const long long q = g / gq;
        const long long s = (g - q * gq) * 32 + lane;
        ray = s * nd + q;
        return s < n_src;
    }
    ray = g * 32 + lane;
    return ray < n_src * nd;
}

// 32 * (longest path in the group) for every 32-ray group.
__global__ void k_group_slots(const uint32_t* __restrict__ nseg, long long n_groups, long long gq, long long n_src,
                              int nd, int layout, long long* slots)
{
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long g = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; g < n_groups; g += warps) {
        long long ray;
        unsigned v = group_ray(g, lane, gq, n_src, nd, layout, ray) ? nseg[ray] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(RT_FULL, v, o));
        if (lane == 0) slots[g] = 32ll * (long long)v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) slots[n_groups] = 0;
}

template <int KIND, int MODE, int SM>
__global__ void __launch_bounds__(256) k_paths(const PathArgs p)
{
    using T = typename std::conditional<MODE == RT_MODE_FP64, double, float>::type;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const T* dsv = (const T*)p.ds;
    for (long long g = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; g < p.n_groups; g += warps) {
        long long ray;
        const bool valid = group_ray(g, lane, p.gq, p.n_src, p.nd, p.layout, ray);
        const unsigned ns = valid ? p.nseg[ray] : 0u;
        const long long base = p.off[g] + lane;
        const long long len = (p.off[g + 1] - p.off[g]) >> 5;
        if (KIND == 0) {
            if (MODE == RT_MODE_FP64) {
                FwdF64<SM> v;
                v.dens = p.dens; v.f64 = p.dens_f64; v.S = p.S;
                v.init();
                for (long long k = 0; k < len; k++)
                    if (k < ns) v.seg(__ldg(p.leaf + base + 32 * k), __ldg(dsv + base + 32 * k));
                if (valid) {
                    double* o = (double*)p.out + (size_t)ray * p.S;
                    for (int k = 0; k < SM; k++)
                        if (k < p.S) o[k] = v.col[k];
                }
            } else {
                FwdKahan<SM> v;
                v.dens = p.dens; v.f64 = p.dens_f64; v.S = p.S;
                v.init();
                for (long long k = 0; k < len; k++)
                    if (k < ns) v.seg(__ldg(p.leaf + base + 32 * k), __ldg(dsv + base + 32 * k));
                if (valid) {
                    float* o = (float*)p.out + (size_t)ray * p.S;
                    for (int k = 0; k < SM; k++)
                        if (k < p.S) o[k] = v.sum[k];
                }
            }
        } else {
            AdjScatter<SM> v;
            v.grad = (double*)p.out;
            v.S = p.S;
#pragma unroll
            for (int k = 0; k < SM; k++) {
                v.g[k] = 0.0;
                if (valid && k < p.S)
                    v.g[k] = (MODE == RT_MODE_FP64) ? __ldg((const double*)p.gin + (size_t)ray * p.S + k)
                                                    : (double)__ldg((const float*)p.gin + (size_t)ray * p.S + k);
            }
            for (long long k = 0; k < len; k++)
                if (k < ns) v.seg(__ldg(p.leaf + base + 32 * k), __ldg(dsv + base + 32 * k));
        }
    }
}

template <int KIND>
static cudaError_t launch_paths_kernel(const PathArgs& p, int mode, cudaStream_t s)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const long long want = (p.n_groups + 7) / 8;
    const int grid = (int)std::min<long long>(want, (long long)sm_count_of(dev) * 8);
    if (grid <= 0) return cudaSuccess;
#define RT_PATHS_GO(M, SMV) k_paths<KIND, M, SMV><<<grid, 256, 0, s>>>(p)
    if (mode == RT_MODE_FP64) {
        if (p.S <= 1) RT_PATHS_GO(RT_MODE_FP64, 1);
        else if (p.S <= 2) RT_PATHS_GO(RT_MODE_FP64, 2);
        else if (p.S <= 4) RT_PATHS_GO(RT_MODE_FP64, 4);
        else RT_PATHS_GO(RT_MODE_FP64, 8);
    } else {
        if (p.S <= 1) RT_PATHS_GO(RT_MODE_F32_KAHAN, 1);
        else if (p.S <= 2) RT_PATHS_GO(RT_MODE_F32_KAHAN, 2);
        else if (p.S <= 4) RT_PATHS_GO(RT_MODE_F32_KAHAN, 4);
        else RT_PATHS_GO(RT_MODE_F32_KAHAN, 8);
    }
#undef RT_PATHS_GO
    return cudaGetLastError();
}

static cudaError_t launch_record(const TraceArgs& a, int mode, int block, int grid, cudaStream_t s)
{
    const bool u = a.t.uniform_level >= 0;
    if (mode == RT_MODE_FP64) {
        if (u) k_trace<3, RT_MODE_FP64, true, 1><<<grid, block, 0, s>>>(a);
        else k_trace<3, RT_MODE_FP64, false, 1><<<grid, block, 0, s>>>(a);
    } else {
        if (u) k_trace<3, RT_MODE_F32_KAHAN, true, 1><<<grid, block, 0, s>>>(a);
        else k_trace<3, RT_MODE_F32_KAHAN, false, 1><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

static int record_occupancy(int mode, bool u, int block)
{
    int n = 0;
    if (mode == RT_MODE_FP64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, u ? k_trace<3, RT_MODE_FP64, true, 1>
                                                            : k_trace<3, RT_MODE_FP64, false, 1>, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, u ? k_trace<3, RT_MODE_F32_KAHAN, true, 1>
                                                            : k_trace<3, RT_MODE_F32_KAHAN, false, 1>, block, 0);
    return n;
}

}  // namespace rt

using namespace rt;

struct rt_paths {
    int device, mode, nd, layout;
    int64_t n_src, n_src_pad, n_groups, slots, segments;
    long long* off;
    uint32_t* nseg;
    uint32_t* leaf;
    void* ds;
};

extern "C" {

void rt_destroy_paths(rt_paths* p)
{
    if (!p) return;
    cudaDeviceSynchronize();
    cudaFree(p->off);
    cudaFree(p->nseg);
    cudaFree(p->leaf);
    cudaFree(p->ds);
    free(p);
}

int rt_record_paths(const rt_octree* tree, const double* d_src, int64_t n_src, int nside, int mode,
                    void* stream, rt_paths** out)
{
    if (out) *out = nullptr;
    if (!out) return set_error(RT_ERR_ARG, "rt_record_paths: null output");
    cudaStream_t s = (cudaStream_t)stream;
    // pass 1: segments per ray (the fingerprint walk)
    rt_paths* p = (rt_paths*)calloc(1, sizeof(rt_paths));
    p->mode = mode;
    p->n_src = n_src;
    p->nd = 12 * nside * nside;
    p->n_src_pad = (n_src + 31) / 32 * 32;
    p->layout = ray_layout(n_src);
    p->n_groups = p->layout ? (n_src * p->nd + 31) / 32 : p->n_src_pad * p->nd / 32;
    cudaGetDevice(&p->device);
    int status = RT_OK;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    long long total = 0;
    rt_stats st;
    long long* slots = nullptr;
    if (n_src < 0 || nside < 1) { status = set_error(RT_ERR_ARG, "rt_record_paths: bad sources or nside"); goto fail; }
    if (cudaMalloc(&p->nseg, sizeof(uint32_t) * (size_t)std::max<int64_t>(1, n_src * p->nd)) != cudaSuccess ||
        cudaMalloc(&p->off, sizeof(long long) * (size_t)(p->n_groups + 1)) != cudaSuccess ||
        cudaMalloc(&slots, sizeof(long long) * (size_t)(p->n_groups + 1)) != cudaSuccess) {
        status = set_error(RT_ERR_OOM, "rt_record_paths: allocation");
        goto fail;
    }
    if (rt_reset_stats((rt_octree*)tree, stream) != RT_OK) { status = RT_ERR_CUDA; goto fail; }
    status = rt_trace_paths(tree, d_src, n_src, nside, mode, p->nseg, nullptr, stream);
    if (status != RT_OK) goto fail;
    if (p->n_groups > 0) {
        int dev = p->device;
        const int grid = (int)std::min<long long>((p->n_groups + 7) / 8, (long long)sm_count_of(dev) * 8);
        k_group_slots<<<grid, 256, 0, s>>>(p->nseg, p->n_groups, p->n_src_pad / 32, n_src, p->nd, p->layout, slots);
        cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, slots, p->off, p->n_groups + 1, s);
        if (cudaMalloc(&tmp, tmp_bytes) != cudaSuccess) { status = set_error(RT_ERR_OOM, "rt_record_paths: scan scratch"); goto fail; }
        cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, slots, p->off, p->n_groups + 1, s);
        if (cudaMemcpyAsync(&total, p->off + p->n_groups, sizeof total, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            status = cuda_error("rt_record_paths: size readback");
            goto fail;
        }
    }
    if (rt_get_stats(tree, &st, stream) != RT_OK) { status = RT_ERR_CUDA; goto fail; }  // synchronizes
    if (st.status != RT_OK) {
        status = set_error(st.status, "rt_record_paths: a walk failed while counting segments");
        goto fail;
    }
    p->segments = (int64_t)st.segments;
    p->slots = total;
    if (cudaMalloc(&p->leaf, sizeof(uint32_t) * (size_t)std::max<long long>(1, total)) != cudaSuccess ||
        cudaMalloc(&p->ds, (mode == RT_MODE_FP64 ? 8 : 4) * (size_t)std::max<long long>(1, total)) != cudaSuccess) {
        status = set_error(RT_ERR_OOM, "rt_record_paths: the record does not fit in device memory");
        goto fail;
    }
    // pass 2: record
    if (n_src > 0) {
        TraceArgs a;
        memset(&a, 0, sizeof a);
        int dev = p->device;
        a.t = tree->dev;
        if (!tree->uniform_allowed) a.t.uniform_level = -1;
        a.dirs = direction_table(dev, nside, &status);
        if (!a.dirs) goto fail;
        a.nd = p->nd;
        a.src = d_src;
        a.n_src = n_src;
        a.n_src_pad = p->n_src_pad;
        a.S = 1;
        a.st = tree->st;
        a.batch = 4;
        a.layout = p->layout;
        a.rec_off = p->off;
        a.rec_leaf = p->leaf;
        a.rec_ds = p->ds;
        int block, bps, groups;
        launch_shape(&block, &bps, &groups);
        a.batch = groups;
        const int fit = record_occupancy(mode, a.t.uniform_level >= 0, block);
        const int grid = sm_count_of(dev) * std::max(1, bps > 0 ? std::min(bps, fit) : fit);
        if (cudaMemsetAsync(&tree->st->queue, 0, sizeof(unsigned long long), s) != cudaSuccess ||
            launch_record(a, mode, block, grid, s) != cudaSuccess) {
            status = cuda_error("rt_record_paths: record launch");
            goto fail;
        }
    }
    cudaFree(tmp);
    cudaFree(slots);
    *out = p;
    clear_error();
    return RT_OK;
fail:
    if (tmp) cudaFree(tmp);
    if (slots) cudaFree(slots);
    rt_destroy_paths(p);
    return status;
}

int rt_paths_info(const rt_paths* p, int64_t* n_rays, int64_t* n_segments, int64_t* bytes)
{
    if (!p) return set_error(RT_ERR_ARG, "rt_paths_info: null paths");
    if (n_rays) *n_rays = p->n_src * p->nd;
    if (n_segments) *n_segments = p->segments;
    if (bytes)
        *bytes = p->slots * (int64_t)(4 + (p->mode == RT_MODE_FP64 ? 8 : 4)) + 8 * (p->n_groups + 1) +
                 4 * p->n_src * p->nd;
    return RT_OK;
}

static int paths_args(const rt_paths* p, int S, PathArgs& a, const char* who)
{
    char buf[160];
    if (!p || S < 1 || S > kMaxSpecies) {
        snprintf(buf, sizeof buf, "%s: null paths or n_species outside [1, 8]", who);
        return set_error(RT_ERR_ARG, buf);
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != p->device) return set_error(RT_ERR_ARG, "paths were recorded on another device");
    memset(&a, 0, sizeof a);
    a.off = p->off;
    a.nseg = p->nseg;
    a.leaf = p->leaf;
    a.ds = p->ds;
    a.n_groups = p->n_groups;
    a.gq = p->n_src_pad / 32;
    a.n_src = p->n_src;
    a.nd = p->nd;
    a.S = S;
    a.layout = p->layout;
    return RT_OK;
}

int rt_paths_columns(const rt_paths* p, const void* d_dens, int n_species, int dens_dtype, void* d_out,
                     void* stream)
{
    PathArgs a;
    const int st = paths_args(p, n_species, a, "rt_paths_columns");
    if (st != RT_OK) return st;
    if (dens_dtype != RT_F32 && dens_dtype != RT_F64) return set_error(RT_ERR_ARG, "rt_paths_columns: bad dens_dtype");
    if (p->n_src == 0) return RT_OK;
    if (!d_dens || !d_out || ((uintptr_t)d_dens & 15u) || ((uintptr_t)d_out & 15u))
        return set_error(RT_ERR_ARG, "rt_paths_columns: densities and output must be non-null and 16-byte aligned");
    a.dens = d_dens;
    a.dens_f64 = dens_dtype == RT_F64;
    a.out = d_out;
    if (launch_paths_kernel<0>(a, p->mode, (cudaStream_t)stream) != cudaSuccess)
        return cuda_error("rt_paths_columns: launch");
    return RT_OK;
}

int rt_paths_adjoint(const rt_paths* p, const void* d_grad_out, int n_species, double* d_grad_dens, void* stream)
{
    PathArgs a;
    const int st = paths_args(p, n_species, a, "rt_paths_adjoint");
    if (st != RT_OK) return st;
    if (p->n_src == 0) return RT_OK;
    if (!d_grad_out || !d_grad_dens || ((uintptr_t)d_grad_out & 15u) || ((uintptr_t)d_grad_dens & 15u))
        return set_error(RT_ERR_ARG, "rt_paths_adjoint: gradients must be non-null and 16-byte aligned");
    a.gin = d_grad_out;
    a.out = d_grad_dens;
    if (launch_paths_kernel<1>(a, p->mode, (cudaStream_t)stream) != cudaSuccess)
        return cuda_error("rt_paths_adjoint: launch");
    return RT_OK;
}

}  // extern "C"
