// Adjoint scatter: kernel instantiations and dispatch.
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
