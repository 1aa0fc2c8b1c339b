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

// Sort keys of the record's slots: the leaf of every valid slot, n_leaves (a
// key past every leaf) for the padding slots of shorter paths; and each
// slot's ray.
__global__ void k_slot_keys(const long long* __restrict__ off, const uint32_t* __restrict__ nseg,
                            const uint32_t* __restrict__ leaf, long long n_groups, long long gq, long long n_src,
                            int nd, int layout, uint32_t n_leaves, uint32_t* key, uint32_t* slot, uint32_t* slot_ray)
{
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    for (long long g = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; g < n_groups; g += warps) {
        long long ray;
        const bool valid = group_ray(g, lane, gq, n_src, nd, layout, ray);
        const unsigned ns = valid ? nseg[ray] : 0u;
        const long long base = off[g] + lane, len = (off[g + 1] - off[g]) >> 5;
        for (long long k = 0; k < len; k++) {
            const long long sl = base + 32 * k;
            key[sl] = k < ns ? leaf[sl] : n_leaves;
            slot[sl] = (uint32_t)sl;
            slot_ray[sl] = valid ? (uint32_t)ray : 0u;
        }
    }
}

// First sorted position of every leaf (and of the padding key past them).
__global__ void k_leaf_start(const uint32_t* __restrict__ skey, long long n_keys, long long n_leaves,
                             long long* start)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j <= n_leaves;
         j += (long long)gridDim.x * blockDim.x) {
        long long lo = 0, hi = n_keys;
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if ((long long)skey[mid] < j) lo = mid + 1;
            else hi = mid;
        }
        start[j] = lo;
    }
}

// Ordered adjoint: one thread per leaf sums g[ray, k] ds over the leaf's slots
// in record order (FP64 products of the recorded length and the gradient),
// then adds the sums to the gradient: the same bits on every run.
template <int MODE, int SM>
__global__ void k_paths_ordered(const long long* __restrict__ start, const uint32_t* __restrict__ t_slot,
                                const uint32_t* __restrict__ slot_ray, const void* __restrict__ ds,
                                const void* __restrict__ gin, long long n_leaves, int S, double* grad)
{
    using T = typename std::conditional<MODE == RT_MODE_FP64, double, float>::type;
    const T* dsv = (const T*)ds;
    const T* gv = (const T*)gin;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n_leaves;
         j += (long long)gridDim.x * blockDim.x) {
        double acc[SM];
#pragma unroll
        for (int k = 0; k < SM; k++) acc[k] = 0.0;
        const long long t1 = start[j + 1];
        for (long long t = start[j]; t < t1; t++) {
            const uint32_t sl = __ldg(t_slot + t);
            const double d = (double)__ldg(dsv + sl);
            const size_t r = (size_t)__ldg(slot_ray + sl) * S;
#pragma unroll
            for (int k = 0; k < SM; k++)
                if (k < S) acc[k] = __dadd_rn(acc[k], __dmul_rn((double)__ldg(gv + r + k), d));
        }
        double* gp = grad + (size_t)j * S;
#pragma unroll
        for (int k = 0; k < SM; k++)
            if (k < S) gp[k] = __dadd_rn(gp[k], acc[k]);
    }
}

}  // namespace rt

using namespace rt;

struct rt_paths {
    int device, mode, nd, layout;
    int64_t n_src, n_src_pad, n_groups, slots, segments, n_leaves;
    long long* off;
    uint32_t* nseg;
    uint32_t* leaf;
    void* ds;
    // leaf-major index of the record (built by the first ordered adjoint):
    // the record's slots sorted by leaf (stable, so each leaf's slots stay in
    // record order), each slot's ray, and each leaf's first sorted position
    uint32_t* t_slot;     // [slots]
    uint32_t* slot_ray;   // [slots]
    long long* t_start;   // [n_leaves + 1]
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
    cudaFree(p->t_slot);
    cudaFree(p->slot_ray);
    cudaFree(p->t_start);
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
    p->n_leaves = tree->dev.n;
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

// Builds the leaf-major index of a record (once).
static int build_transpose(rt_paths* p, cudaStream_t s)
{
    if (p->t_start) return RT_OK;
    if (p->slots >= (1ll << 32) || p->n_leaves >= 0xffffffffll)
        return set_error(RT_ERR_ARG, "rt_paths_adjoint_ordered: the record has 2^32 or more slots");
    const long long n = std::max<long long>(1, p->slots);
    uint32_t *key = nullptr, *key2 = nullptr, *slot = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    int bits = 1;
    while (bits < 32 && (1ull << bits) <= (unsigned long long)p->n_leaves) bits++;
    int st = RT_OK;
    if (cudaMalloc(&key, sizeof(uint32_t) * n) != cudaSuccess || cudaMalloc(&key2, sizeof(uint32_t) * n) != cudaSuccess ||
        cudaMalloc(&slot, sizeof(uint32_t) * n) != cudaSuccess ||
        cudaMalloc(&p->t_slot, sizeof(uint32_t) * n) != cudaSuccess ||
        cudaMalloc(&p->slot_ray, sizeof(uint32_t) * n) != cudaSuccess ||
        cudaMalloc(&p->t_start, sizeof(long long) * (p->n_leaves + 1)) != cudaSuccess) {
        st = set_error(RT_ERR_OOM, "rt_paths_adjoint_ordered: the leaf-major index does not fit in device memory");
    }
    if (st == RT_OK && p->n_groups > 0) {
        const int grid = (int)std::min<long long>((p->n_groups + 7) / 8, (long long)sm_count_of(p->device) * 8);
        k_slot_keys<<<grid, 256, 0, s>>>(p->off, p->nseg, p->leaf, p->n_groups, p->n_src_pad / 32, p->n_src, p->nd,
                                         p->layout, (uint32_t)p->n_leaves, key, slot, p->slot_ray);
        cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, key, key2, slot, p->t_slot, (long long)p->slots, 0, bits, s);
        if (cudaMalloc(&tmp, tmp_bytes) != cudaSuccess)
            st = set_error(RT_ERR_OOM, "rt_paths_adjoint_ordered: sort scratch");
        else if (cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, key, key2, slot, p->t_slot, (long long)p->slots, 0, bits,
                                                 s) != cudaSuccess)
            st = cuda_error("rt_paths_adjoint_ordered: sort");
    }
    if (st == RT_OK) {
        const int grid = (int)std::min<long long>((p->n_leaves + 256) / 256, 4096);
        k_leaf_start<<<grid, 256, 0, s>>>(key2, p->slots, p->n_leaves, p->t_start);
        if (cudaGetLastError() != cudaSuccess) st = cuda_error("rt_paths_adjoint_ordered: index");
    }
    cudaStreamSynchronize(s);
    cudaFree(tmp);
    cudaFree(key);
    cudaFree(key2);
    cudaFree(slot);
    if (st != RT_OK) {
        cudaFree(p->t_slot);
        cudaFree(p->slot_ray);
        cudaFree(p->t_start);
        p->t_slot = p->slot_ray = nullptr;
        p->t_start = nullptr;
    }
    return st;
}

int rt_paths_adjoint_ordered(rt_paths* p, const void* d_grad_out, int n_species, double* d_grad_dens, void* stream)
{
    PathArgs a;
    int st = paths_args(p, n_species, a, "rt_paths_adjoint_ordered");
    if (st != RT_OK) return st;
    if (p->n_src == 0) return RT_OK;
    if (!d_grad_out || !d_grad_dens)
        return set_error(RT_ERR_ARG, "rt_paths_adjoint_ordered: null gradient pointer");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = build_transpose(p, s)) != RT_OK) return st;
    const int grid = (int)std::min<long long>((p->n_leaves + 255) / 256, (long long)sm_count_of(p->device) * 16);
#define RT_ORD_GO(M, SMV)                                                                                          \
    k_paths_ordered<M, SMV><<<grid, 256, 0, s>>>(p->t_start, p->t_slot, p->slot_ray, p->ds, d_grad_out, p->n_leaves, \
                                                 n_species, d_grad_dens)
    if (p->mode == RT_MODE_FP64) {
        if (n_species <= 1) RT_ORD_GO(RT_MODE_FP64, 1);
        else if (n_species <= 2) RT_ORD_GO(RT_MODE_FP64, 2);
        else if (n_species <= 4) RT_ORD_GO(RT_MODE_FP64, 4);
        else RT_ORD_GO(RT_MODE_FP64, 8);
    } else {
        if (n_species <= 1) RT_ORD_GO(RT_MODE_F32_KAHAN, 1);
        else if (n_species <= 2) RT_ORD_GO(RT_MODE_F32_KAHAN, 2);
        else if (n_species <= 4) RT_ORD_GO(RT_MODE_F32_KAHAN, 4);
        else RT_ORD_GO(RT_MODE_F32_KAHAN, 8);
    }
#undef RT_ORD_GO
    if (cudaGetLastError() != cudaSuccess) return cuda_error("rt_paths_adjoint_ordered: launch");
    return RT_OK;
}

}  // extern "C"
