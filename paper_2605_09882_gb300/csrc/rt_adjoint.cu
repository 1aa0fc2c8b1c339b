// Adjoint: the entry point (policy: leaf gather, scatter over recomputed or
// recorded paths, deterministic), and the scatter's kernel instantiations.
#include "rt_host.h"
#include "rt_kernels.cuh"

namespace rt {

template <int MODE, bool U>
static cudaError_t go(const TraceArgs& a, int block, int grid, cudaStream_t s)
{
    if (a.S <= 1) k_trace<2, MODE, U, 1><<<grid, block, 0, s>>>(a);
    else if (a.S <= 2) k_trace<2, MODE, U, 2><<<grid, block, 0, s>>>(a);
    else if (a.S <= 4) k_trace<2, MODE, U, 4><<<grid, block, 0, s>>>(a);
    else k_trace<2, MODE, U, 8><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const TraceArgs& a, int mode, int block, int grid, cudaStream_t s)
{
    const bool u = a.t.uniform_level >= 0;
    if (mode == RT_MODE_FP64) return u ? go<RT_MODE_FP64, true>(a, block, grid, s) : go<RT_MODE_FP64, false>(a, block, grid, s);
    return u ? go<RT_MODE_F32_KAHAN, true>(a, block, grid, s) : go<RT_MODE_F32_KAHAN, false>(a, block, grid, s);
}

template <int MODE, bool U, int SM>
static int occ(int block)
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<2, MODE, U, SM>, block, 0);
    return n;
}

template <int MODE, bool U>
static int occ_s(int S, int block)
{
    if (S <= 1) return occ<MODE, U, 1>(block);
    if (S <= 2) return occ<MODE, U, 2>(block);
    if (S <= 4) return occ<MODE, U, 4>(block);
    return occ<MODE, U, 8>(block);
}

int occupancy_adj(int mode, int S, bool u, int block)
{
    if (mode == RT_MODE_FP64) return u ? occ_s<RT_MODE_FP64, true>(S, block) : occ_s<RT_MODE_FP64, false>(S, block);
    return u ? occ_s<RT_MODE_F32_KAHAN, true>(S, block) : occ_s<RT_MODE_F32_KAHAN, false>(S, block);
}

}  // namespace rt

using namespace rt;

extern "C" {

int rt_trace_columns_adjoint(const rt_octree* t, const double* d_src, int64_t n_src, int nside,
                             const void* d_grad_out, int n_species, int mode, double* d_grad_dens,
                             int path_policy, void* stream)
{
    TraceArgs a;
    int st = prepare_trace(t, d_src, n_src, nside, n_species, mode, a, "rt_trace_columns_adjoint");
    if (st != RT_OK) return st;
    if (path_policy < 0 || path_policy > 3)
        return set_error(RT_ERR_ARG, "rt_trace_columns_adjoint: path_policy must be 0, 1, 2 or 3");
    if (n_src == 0) return RT_OK;
    if (!d_grad_out || !d_grad_dens) return set_error(RT_ERR_ARG, "rt_trace_columns_adjoint: null gradient pointer");
    if (((uintptr_t)d_grad_out & 15u) || ((uintptr_t)d_grad_dens & 15u))
        return set_error(RT_ERR_ARG, "rt_trace_columns_adjoint: gradients must be 16-byte aligned");
    if (path_policy == 2) {
        rt_paths* p = nullptr;
        st = rt_record_paths(t, d_src, n_src, nside, mode, stream, &p);
        if (st != RT_OK) return st;
        st = rt_paths_adjoint(p, d_grad_out, n_species, d_grad_dens, stream);
        rt_destroy_paths(p);
        return st;
    }
    a.gin = d_grad_out;
    a.out = d_grad_dens;
    cudaStream_t s = (cudaStream_t)stream;
    if (path_policy == 3) {
        // deterministic: the leaf gather if the sources have its layout, else
        // the ordered adjoint over a record of the paths
        if (gather_applies(t, a)) {
            st = launch_adjoint_gather((rt_octree*)t, a, mode, s);
            if (st != RT_OK) return st;
            int off = 1;
            if (cudaMemcpyAsync(&off, &t->st->gather_off, sizeof off, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return cuda_error("rt_trace_columns_adjoint: gather flag readback");
            if (off == 0) return RT_OK;
        }
        rt_paths* p = nullptr;
        st = rt_record_paths(t, d_src, n_src, nside, mode, stream, &p);
        if (st != RT_OK) return st;
        st = rt_paths_adjoint_ordered(p, d_grad_out, n_species, d_grad_dens, stream);
        rt_destroy_paths(p);
        return st;
    }
    if (path_policy == 0 && gather_applies(t, a)) {
        // the leaf gather, with the scatter below as the fallback the device
        // takes when the sources do not have the gather's layout
        st = launch_adjoint_gather((rt_octree*)t, a, mode, s);
        if (st != RT_OK) return st;
        a.gate = &t->st->gather_off;
    }
    int block, bps, groups;
    launch_shape(&block, &bps, &groups);
    int dev = 0;
    cudaGetDevice(&dev);
    const int fit = occupancy_adj(mode, n_species, a.t.uniform_level >= 0, block);
    const int grid = sm_count_of(dev) * std::max(1, bps > 0 ? std::min(bps, fit) : fit);
    if (cudaMemsetAsync(&t->st->queue, 0, sizeof(unsigned long long), s) != cudaSuccess)
        return cuda_error("rt_trace_columns_adjoint: queue reset");
    if (launch_adjoint(a, mode, block, grid, s) != cudaSuccess)
        return cuda_error("rt_trace_columns_adjoint: launch");
    return RT_OK;
}

}  // extern "C"
