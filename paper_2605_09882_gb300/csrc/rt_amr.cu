// Contribution-grid construction on the GPU: the leaf-only linear octree
// built from a uniform source grid by recursive refinement (Sec. 2.2.1) with
// the 3D-PDR criterion (Sec. 2.4: split a cell iff n_max >= n_PDR and
// (n_max - n_min) / n_max >= 1 %, down to a maximum depth).
//
// The source grid arrives in Morton order at level L, so every coarser cell is
// a contiguous run of 8^(L-l) source cells.  A min/max/sum pyramid is reduced
// bottom-up, the split flag of each cell follows from its min and max, and
// every source cell finds the level of the leaf containing it (the first
// level whose cell does not split).  Source cells that start a leaf are
// compacted with a scan, which emits the leaves already sorted by key.
#include <cub/cub.cuh>

#include "rt_device.cuh"
#include "rt_host.h"

namespace rt {

__device__ __forceinline__ double load_as_double(const void* p, int f64, size_t i)
{
    return f64 ? __ldg((const double*)p + i) : (double)__ldg((const float*)p + i);
}

// One pyramid level: cells of level l from their 8 children (level l + 1,
// or the source grid when l + 1 == L); the split flag uses the same FP64
// expression as the plain construction.
__global__ void k_pyramid(int l, int L, const void* nref, int nref_f64, const void* vals, int vals_f64, int S,
                          const double* cmn, const double* cmx, const double* csum, double* mn, double* mx, double* sum,
                          uint8_t* split, double n_pdr, double rel_var, int max_level)
{
    const long long ncell = 1ll << (3 * l);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
        double lo = 0.0, hi = 0.0;
        double acc[kMaxSpecies];
        for (int k = 0; k < S; k++) acc[k] = 0.0;
        for (int i = 0; i < 8; i++) {
            const long long ch = 8 * c + i;
            double a, b;
            if (l + 1 == L) {
                a = b = load_as_double(nref, nref_f64, (size_t)ch);
                for (int k = 0; k < S; k++)
                    acc[k] += vals ? load_as_double(vals, vals_f64, (size_t)ch * S + k) : a;
            } else {
                a = cmn[ch];
                b = cmx[ch];
                for (int k = 0; k < S; k++) acc[k] += csum[ch * S + k];
            }
            lo = (i == 0) ? a : fmin(lo, a);
            hi = (i == 0) ? b : fmax(hi, b);
        }
        mn[c] = lo;
        mx[c] = hi;
        for (int k = 0; k < S; k++) sum[c * S + k] = acc[k];
        split[c] = (hi != 0.0 && l < max_level && hi >= n_pdr && __ddiv_rn(__dsub_rn(hi, lo), hi) >= rel_var) ? 1 : 0;
    }
}

struct PyrPtrs {
    const uint8_t* split[kMaxTableLevel + 1];
    const double* sum[kMaxTableLevel + 1];
};

// Level of the leaf holding each source cell, and whether the cell starts it.
__global__ void k_leaf_levels(int L, long long n, PyrPtrs p, uint8_t* lvl, int* start)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int l = 0;
        while (l < L && p.split[l][i >> (3 * (L - l))]) l++;
        lvl[i] = (uint8_t)l;
        start[i] = (i & ((1ll << (3 * (L - l))) - 1)) == 0 ? 1 : 0;
    }
}

__global__ void k_emit(int L, long long n, PyrPtrs p, const void* nref, int nref_f64, const void* vals, int vals_f64,
                       int S, const uint8_t* lvl, const int* start, const long long* pos, uint64_t* keys,
                       uint8_t* levels, void* out, int out_f64)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (!start[i]) continue;
        const int l = lvl[i];
        const long long j = pos[i];
        keys[j] = (uint64_t)i << (3 * (kDepth - L));
        levels[j] = (uint8_t)l;
        const long long c = i >> (3 * (L - l));
        const double inv = 1.0 / (double)(1ll << (3 * (L - l)));
        for (int k = 0; k < S; k++) {
            double s;
            if (l == L) s = vals ? load_as_double(vals, vals_f64, (size_t)i * S + k) : load_as_double(nref, nref_f64, (size_t)i);
            else s = p.sum[l][c * S + k];
            const double m = s * inv;
            if (out_f64) ((double*)out)[j * S + k] = m;
            else ((float*)out)[j * S + k] = (float)m;
        }
    }
}

}  // namespace rt

using namespace rt;

extern "C" int rt_build_amr(const void* d_nref, int nref_dtype, const void* d_vals, int n_species, int vals_dtype,
                            int level, double n_pdr, double rel_var, int max_level, uint64_t* d_keys,
                            uint8_t* d_levels, void* d_leaf_vals, int64_t capacity, int64_t* h_n_leaves,
                            void* stream)
{
    if (!d_nref || !d_keys || !d_levels || !d_leaf_vals || !h_n_leaves)
        return set_error(RT_ERR_ARG, "rt_build_amr: null pointer");
    if (level < 1 || level > kMaxTableLevel) return set_error(RT_ERR_ARG, "rt_build_amr: level must be in [1, 10]");
    if (n_species < 1 || n_species > kMaxSpecies) return set_error(RT_ERR_ARG, "rt_build_amr: n_species must be in [1, 8]");
    if (!d_vals && n_species != 1) return set_error(RT_ERR_ARG, "rt_build_amr: without values n_species must be 1");
    if ((nref_dtype != RT_F32 && nref_dtype != RT_F64) || (vals_dtype != RT_F32 && vals_dtype != RT_F64))
        return set_error(RT_ERR_ARG, "rt_build_amr: bad dtype");
    const int L = level;
    const long long n = 1ll << (3 * L);
    if (capacity < n) return set_error(RT_ERR_ARG, "rt_build_amr: capacity below 8^level");
    const int S = n_species;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    const int gmax = sm_count_of(dev) * 8;
    // pyramid of levels 0 .. L-1
    double *mn[kMaxTableLevel + 1] = {}, *mx[kMaxTableLevel + 1] = {}, *sum[kMaxTableLevel + 1] = {};
    uint8_t* split[kMaxTableLevel + 1] = {};
    uint8_t* lvl = nullptr;
    int* start = nullptr;
    long long* pos = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    int status = RT_OK;
    long long last_pos = 0;
    int last_start = 0;
    PyrPtrs pp;
    memset(&pp, 0, sizeof pp);
    for (int l = 0; l < L; l++) {
        const long long nc = 1ll << (3 * l);
        if (cudaMalloc(&mn[l], sizeof(double) * nc) != cudaSuccess || cudaMalloc(&mx[l], sizeof(double) * nc) != cudaSuccess ||
            cudaMalloc(&sum[l], sizeof(double) * nc * S) != cudaSuccess || cudaMalloc(&split[l], nc) != cudaSuccess) {
            status = set_error(RT_ERR_OOM, "rt_build_amr: pyramid allocation");
            goto done;
        }
    }
    if (cudaMalloc(&lvl, n) != cudaSuccess || cudaMalloc(&start, sizeof(int) * n) != cudaSuccess ||
        cudaMalloc(&pos, sizeof(long long) * n) != cudaSuccess) {
        status = set_error(RT_ERR_OOM, "rt_build_amr: allocation");
        goto done;
    }
    for (int l = L - 1; l >= 0; l--) {
        const long long nc = 1ll << (3 * l);
        const int grid = (int)std::min<long long>((nc + 255) / 256, gmax);
        k_pyramid<<<grid, 256, 0, s>>>(l, L, d_nref, nref_dtype == RT_F64, d_vals, vals_dtype == RT_F64, S,
                                       l + 1 < L ? mn[l + 1] : nullptr, l + 1 < L ? mx[l + 1] : nullptr,
                                       l + 1 < L ? sum[l + 1] : nullptr, mn[l], mx[l], sum[l], split[l], n_pdr,
                                       rel_var, max_level);
    }
    for (int l = 0; l < L; l++) {
        pp.split[l] = split[l];
        pp.sum[l] = sum[l];
    }
    {
        const int grid = (int)std::min<long long>((n + 255) / 256, gmax);
        k_leaf_levels<<<grid, 256, 0, s>>>(L, n, pp, lvl, start);
        cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, start, pos, n, s);
        if (cudaMalloc(&tmp, tmp_bytes) != cudaSuccess) {
            status = set_error(RT_ERR_OOM, "rt_build_amr: scan scratch");
            goto done;
        }
        cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, start, pos, n, s);
        k_emit<<<grid, 256, 0, s>>>(L, n, pp, d_nref, nref_dtype == RT_F64, d_vals, vals_dtype == RT_F64, S, lvl, start,
                                    pos, d_keys, d_levels, d_leaf_vals, vals_dtype == RT_F64);
        cudaMemcpyAsync(&last_pos, pos + (n - 1), sizeof last_pos, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&last_start, start + (n - 1), sizeof last_start, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            status = cuda_error("rt_build_amr");
            goto done;
        }
        *h_n_leaves = last_pos + last_start;
    }
done:
    for (int l = 0; l < L; l++) {
        if (mn[l]) cudaFree(mn[l]);
        if (mx[l]) cudaFree(mx[l]);
        if (sum[l]) cudaFree(sum[l]);
        if (split[l]) cudaFree(split[l]);
    }
    if (lvl) cudaFree(lvl);
    if (start) cudaFree(start);
    if (pos) cudaFree(pos);
    if (tmp) cudaFree(tmp);
    if (status == RT_OK) clear_error();
    return status;
}
