// Octree handle: device-side validation of a leaf-only linear octree and the
// coarse Morton table that turns most leaf lookups into one table read
// (Sec. 2.2.1: leaves in compact Morton/level arrays, found by array lookup).
#include <stdlib.h>

#include <atomic>

#include "rt_device.cuh"
#include "rt_host.h"

namespace rt {

struct ValOut {
    unsigned int flags;  // 1 level > 21, 2 misaligned, 4 unsorted, 8 overlap / outside the box
    unsigned int lmax;
    unsigned int lmin;
    unsigned int pad;
    unsigned long long vol;  // sum of leaf volumes (depth-21 cells), wraps on overlap
};

__global__ void k_validate(const uint64_t* __restrict__ keys, const uint8_t* __restrict__ levels,
                           int64_t n, uint32_t ex, uint32_t ey, uint32_t ez, ValOut* out)
{
    unsigned flags = 0, lmax = 0, lmin = 255;
    unsigned long long vol = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const unsigned l = levels[j];
        const uint64_t k = keys[j];
        uint64_t span = 0;
        if (l > kDepth) {
            flags |= 1u;
        } else {
            span = 1ull << (3 * (kDepth - l));
            lmax = max(lmax, l);
            lmin = min(lmin, l);
            vol += span;
            if ((k >> 63) || (k & (span - 1))) {
                flags |= 2u;
            } else {
                const uint32_t size = 1u << (kDepth - l);
                if ((uint64_t)compact21(k) + size > ex || (uint64_t)compact21(k >> 1) + size > ey ||
                    (uint64_t)compact21(k >> 2) + size > ez)
                    flags |= 8u;
            }
        }
        if (j + 1 < n) {
            const uint64_t k2 = keys[j + 1];
            if (k2 <= k) flags |= 4u;
            else if (l <= kDepth && k2 - k < span) flags |= 8u;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        flags |= __shfl_xor_sync(RT_FULL, flags, o);
        lmax = max(lmax, __shfl_xor_sync(RT_FULL, lmax, o));
        lmin = min(lmin, __shfl_xor_sync(RT_FULL, lmin, o));
        vol += __shfl_xor_sync(RT_FULL, vol, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (flags) atomicOr(&out->flags, flags);
        atomicMax(&out->lmax, lmax);
        atomicMin(&out->lmin, lmin);
        atomicAdd(&out->vol, vol);
    }
}

// Level range of the leaves finer than the table inside each coarse cell.
__global__ void k_cell_levels(const uint64_t* __restrict__ keys, const uint8_t* __restrict__ levels,
                              int64_t n, int T, unsigned* lvmin, unsigned* lvmax)
{
    const int csh = 3 * (kDepth - T);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const unsigned l = levels[j];
        if ((int)l > T) {
            const uint64_t cell = keys[j] >> csh;
            atomicMin(lvmin + cell, l);
            atomicMax(lvmax + cell, l);
        }
    }
}

__device__ __forceinline__ int64_t lower_bound_keys(const uint64_t* keys, int64_t n, uint64_t v)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One entry per coarse cell C (Morton index at level T):
//   code l <= T : the cell lies in leaf `first` (level l);
//   code l > T  : every leaf in the cell has level l, leaf = first + local index;
//   kCodeMixed  : binary search in [first, next cell's first);
//   kCodeHole   : the cell starts outside the domain box.
__global__ void k_fill_table(const uint64_t* __restrict__ keys, const uint8_t* __restrict__ levels,
                             int64_t n, int T, uint32_t ex, uint32_t ey, uint32_t ez,
                             const unsigned* lvmin, const unsigned* lvmax, uint64_t* table)
{
    const int csh = 3 * (kDepth - T);
    const uint64_t ncell = 1ull << (3 * T);
    for (uint64_t C = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; C < ncell;
         C += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t base = C << csh;
        const int64_t j0 = lower_bound_keys(keys, n, base);
        int code;
        int64_t first = j0;
        if (compact21(base) >= ex || compact21(base >> 1) >= ey || compact21(base >> 2) >= ez) {
            code = kCodeHole;
        } else if (j0 > 0 && keys[j0 - 1] + (1ull << (3 * (kDepth - levels[j0 - 1]))) > base) {
            code = levels[j0 - 1];
            first = j0 - 1;
        } else if (j0 < n && keys[j0] == base && (int)levels[j0] <= T) {
            code = levels[j0];
        } else if (lvmin[C] == lvmax[C]) {
            const int l = (int)lvmin[C];
            const int64_t j1 = lower_bound_keys(keys, n, base + (1ull << csh));
            code = (j1 - j0 == (int64_t)(1ull << (3 * (l - T)))) ? l : kCodeMixed;
        } else {
            code = kCodeMixed;
        }
        table[C] = ((uint64_t)first << 6) | (uint64_t)code;
    }
}

// Densities are number densities: finite and non-negative.  The first NaN,
// infinite or negative value found sets RT_ERR_NONFINITE in the status word,
// with the index of its leaf (base + i / S) as the fault position.
__global__ void k_check_dens(const void* __restrict__ dens, long long count, int f64, int S, long long base,
                             DevStats* st)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (!f64) {
        const float* p = (const float*)dens;
        const long long nv = count / 4;
        for (long long i = t0; i < nv; i += stride) {
            const float4 v = __ldg((const float4*)p + i);
            const float w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (!(w[k] >= 0.f && w[k] <= 3.402823466e38f)) report_fault(st, RT_ERR_NONFINITE, base + (4 * i + k) / S);
        }
        for (long long i = 4 * nv + t0; i < count; i += stride) {
            const float w = __ldg(p + i);
            if (!(w >= 0.f && w <= 3.402823466e38f)) report_fault(st, RT_ERR_NONFINITE, base + i / S);
        }
    } else {
        const double* p = (const double*)dens;
        const long long nv = count / 2;
        for (long long i = t0; i < nv; i += stride) {
            const double2 v = __ldg((const double2*)p + i);
            if (!(v.x >= 0.0 && v.x <= 1.7976931348623157e308)) report_fault(st, RT_ERR_NONFINITE, base + (2 * i) / S);
            if (!(v.y >= 0.0 && v.y <= 1.7976931348623157e308)) report_fault(st, RT_ERR_NONFINITE, base + (2 * i + 1) / S);
        }
        for (long long i = 2 * nv + t0; i < count; i += stride) {
            const double w = __ldg(p + i);
            if (!(w >= 0.0 && w <= 1.7976931348623157e308)) report_fault(st, RT_ERR_NONFINITE, base + i / S);
        }
    }
}

int check_densities(const void* dens, long long n_leaves, int S, int f64, long long base, DevStats* st,
                    cudaStream_t s)
{
    const long long count = n_leaves * S;
    if (count <= 0) return RT_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    const long long want = (count / (f64 ? 2 : 4) + 255) / 256 + 1;
    const int grid = (int)std::min<long long>(want, (long long)sm_count_of(dev) * 8);
    k_check_dens<<<grid, 256, 0, s>>>(dens, count, f64, S, base, st);
    if (cudaGetLastError() != cudaSuccess) return cuda_error("density check launch");
    return RT_OK;
}

}  // namespace rt

using namespace rt;

extern "C" int rt_build_octree(const uint64_t* d_keys, const uint8_t* d_levels, int64_t n_leaves,
                               const int32_t* h_extent, void* stream, rt_octree** out)
{
    if (out) *out = nullptr;
    if (!out || !d_keys || !d_levels) return set_error(RT_ERR_ARG, "rt_build_octree: null pointer");
    if (n_leaves <= 0 || n_leaves >= (1ll << 32))
        return set_error(RT_ERR_ARG, "rt_build_octree: n_leaves must be in [1, 2^32)");
    uint32_t ext[3];
    for (int b = 0; b < 3; b++) {
        const int32_t e = h_extent ? h_extent[b] : (1 << kDepth);
        if (e <= 0 || e > (1 << kDepth)) return set_error(RT_ERR_ARG, "rt_build_octree: extent outside [1, 2^21]");
        ext[b] = (uint32_t)e;
    }
    cudaStream_t s = (cudaStream_t)stream;
    rt_octree* t = (rt_octree*)calloc(1, sizeof(rt_octree));
    if (!t) return set_error(RT_ERR_OOM, "rt_build_octree: host allocation");
    cudaGetDevice(&t->device);
    ValOut* vo = nullptr;
    ValOut hv;
    unsigned *lvmin = nullptr, *lvmax = nullptr;
    int status = RT_OK;
    const int blocks = (int)std::min<int64_t>((n_leaves + 255) / 256, 4096);
    if (cudaMalloc(&t->st, sizeof(DevStats)) != cudaSuccess || cudaMalloc(&vo, sizeof(ValOut)) != cudaSuccess) {
        status = set_error(RT_ERR_OOM, "rt_build_octree: device allocation");
        goto fail;
    }
    cudaMemsetAsync(t->st, 0, sizeof(DevStats), s);
    memset(&hv, 0, sizeof hv);
    hv.lmin = 255;
    cudaMemcpyAsync(vo, &hv, sizeof hv, cudaMemcpyHostToDevice, s);
    k_validate<<<blocks, 256, 0, s>>>(d_keys, d_levels, n_leaves, ext[0], ext[1], ext[2], vo);
    cudaMemcpyAsync(&hv, vo, sizeof hv, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        status = cuda_error("rt_build_octree: validation");
        goto fail;
    }
    if (hv.flags & 1u) status = set_error(RT_ERR_ARG, "rt_build_octree: a level exceeds 21");
    else if (hv.flags & 2u) status = set_error(RT_ERR_MISALIGNED, "rt_build_octree: a key is not aligned to its level");
    else if (hv.flags & 4u) status = set_error(RT_ERR_UNSORTED, "rt_build_octree: keys are not strictly ascending");
    else if (hv.flags & 8u) status = set_error(RT_ERR_OVERLAP_OR_GAP, "rt_build_octree: leaves overlap or leave the domain box");
    else if (hv.vol != (unsigned long long)ext[0] * ext[1] * ext[2])
        status = set_error(RT_ERR_OVERLAP_OR_GAP, "rt_build_octree: leaves do not tile the domain box");
    if (status != RT_OK) goto fail;
    {
        const int lmax = (int)hv.lmax, lmin = (int)hv.lmin;
        const bool full = ext[0] == (1u << kDepth) && ext[1] == (1u << kDepth) && ext[2] == (1u << kDepth);
        const bool uniform = lmin == lmax && lmax <= 10 && full && n_leaves == (int64_t)(1ll << (3 * lmax));
        // Coarse table level: deep enough that most lookups are one table read
        // (at lmax - 1 no coarse cell mixes levels), within 8 entries per leaf
        // (never less than 8^7); a uniform cube uses the O(1) index instead.
        int T = std::min(lmax, kBaseTableLevel);
        if (!uniform) {
            const uint64_t budget = std::max<uint64_t>(1ull << (3 * kBaseTableLevel), 8ull * (uint64_t)n_leaves);
            while (T < std::min(lmax, kMaxTableLevel) && (1ull << (3 * (T + 1))) <= budget) T++;
        }
        const int cap = table_level_cap();
        if (cap >= 0) T = std::min(T, cap);
        const uint64_t ncell = 1ull << (3 * T);
        if (cudaMalloc(&t->table, ncell * sizeof(uint64_t)) != cudaSuccess ||
            cudaMalloc(&lvmin, ncell * sizeof(unsigned)) != cudaSuccess ||
            cudaMalloc(&lvmax, ncell * sizeof(unsigned)) != cudaSuccess) {
            status = set_error(RT_ERR_OOM, "rt_build_octree: table allocation");
            goto fail;
        }
        cudaMemsetAsync(lvmin, 0xff, ncell * sizeof(unsigned), s);
        cudaMemsetAsync(lvmax, 0, ncell * sizeof(unsigned), s);
        k_cell_levels<<<blocks, 256, 0, s>>>(d_keys, d_levels, n_leaves, T, lvmin, lvmax);
        const int cblocks = (int)std::min<uint64_t>((ncell + 255) / 256, 4096);
        k_fill_table<<<cblocks, 256, 0, s>>>(d_keys, d_levels, n_leaves, T, ext[0], ext[1], ext[2],
                                             lvmin, lvmax, t->table);
        if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            status = cuda_error("rt_build_octree: table build");
            goto fail;
        }
        cudaFree(lvmin);
        cudaFree(lvmax);
        lvmin = lvmax = nullptr;
        DevTree& d = t->dev;
        d.keys = d_keys;
        d.levels = d_levels;
        d.table = t->table;
        d.n = n_leaves;
        for (int b = 0; b < 3; b++) d.ext[b] = ext[b];
        d.T = T;
        d.lmax = lmax;
        d.uniform_level = uniform ? lmax : -1;
        static std::atomic<unsigned long long> builds{0};
        t->gen = ++builds;
        t->uniform_allowed = 1;
        t->default_cap = 3 * (1ll << lmax) + 3;
        d.step_cap = t->default_cap;
    }
    cudaFree(vo);
    *out = t;
    clear_error();
    return RT_OK;
fail:
    if (vo) cudaFree(vo);
    if (lvmin) cudaFree(lvmin);
    if (lvmax) cudaFree(lvmax);
    if (t->table) cudaFree(t->table);
    if (t->st) cudaFree(t->st);
    free(t);
    return status;
}
