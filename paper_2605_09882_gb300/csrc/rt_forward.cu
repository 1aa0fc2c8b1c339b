// Forward columns and path fingerprints: kernel instantiations and dispatch.
#include "rt_kernels.cuh"

namespace rt {

template <int KIND, int MODE, bool U>
static cudaError_t go(const TraceArgs& a, int block, int grid, cudaStream_t s)
{
    if (KIND == 1) {
        k_trace<1, MODE, U, 1><<<grid, block, 0, s>>>(a);
        return cudaGetLastError();
    }
    if (a.S <= 1) k_trace<KIND, MODE, U, 1><<<grid, block, 0, s>>>(a);
    else if (a.S <= 2) k_trace<KIND, MODE, U, 2><<<grid, block, 0, s>>>(a);
    else if (a.S <= 4) k_trace<KIND, MODE, U, 4><<<grid, block, 0, s>>>(a);
    else k_trace<KIND, MODE, U, 8><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <int KIND>
static cudaError_t dispatch(const TraceArgs& a, int mode, int block, int grid, cudaStream_t s)
{
    const bool u = a.t.uniform_level >= 0;
    if (mode == RT_MODE_FP64)
        return u ? go<KIND, RT_MODE_FP64, true>(a, block, grid, s) : go<KIND, RT_MODE_FP64, false>(a, block, grid, s);
    return u ? go<KIND, RT_MODE_F32_KAHAN, true>(a, block, grid, s)
             : go<KIND, RT_MODE_F32_KAHAN, false>(a, block, grid, s);
}

cudaError_t launch_forward(const TraceArgs& a, int mode, int block, int grid, cudaStream_t s)
{
    if (a.pair) {
        switch (a.S) {
        case 1: k_trace_pair<1><<<grid, block, 0, s>>>(a); break;
        case 2: k_trace_pair<2><<<grid, block, 0, s>>>(a); break;
        case 4: k_trace_pair<4><<<grid, block, 0, s>>>(a); break;
        case 8: k_trace_pair<8><<<grid, block, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    return dispatch<0>(a, mode, block, grid, s);
}

cudaError_t launch_paths(const TraceArgs& a, int mode, int block, int grid, cudaStream_t s)
{
    return dispatch<1>(a, mode, block, grid, s);
}

template <int KIND, int MODE, bool U, int SM>
static int occ(int block)
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<KIND, MODE, U, SM>, block, 0);
    return n;
}

template <int KIND, int MODE, bool U>
static int occ_s(int S, int block)
{
    if (KIND == 1 || S <= 1) return occ<KIND, MODE, U, 1>(block);
    if (S <= 2) return occ<KIND, MODE, U, 2>(block);
    if (S <= 4) return occ<KIND, MODE, U, 4>(block);
    return occ<KIND, MODE, U, 8>(block);
}

template <int KIND>
static int occ_kind(int mode, int S, bool u, int block)
{
    if (mode == RT_MODE_FP64) return u ? occ_s<KIND, RT_MODE_FP64, true>(S, block) : occ_s<KIND, RT_MODE_FP64, false>(S, block);
    return u ? occ_s<KIND, RT_MODE_F32_KAHAN, true>(S, block) : occ_s<KIND, RT_MODE_F32_KAHAN, false>(S, block);
}

int occupancy_fwd(int kind, int mode, int S, bool uniform, int block)
{
    return kind == 0 ? occ_kind<0>(mode, S, uniform, block) : occ_kind<1>(mode, S, uniform, block);
}

int occupancy_pair(int S, int block)
{
    int n = 0;
    if (S == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace_pair<1>, block, 0);
    else if (S == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace_pair<2>, block, 0);
    else if (S == 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace_pair<4>, block, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace_pair<8>, block, 0);
    return n;
}

}  // namespace rt
