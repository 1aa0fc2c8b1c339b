// Fused per-source epilogues: kernel instantiations, the finishing kernel and
// the entry point.
#include "rt_host.h"
#include "rt_kernels.cuh"

namespace rt {

template <int MODE, bool U>
static cudaError_t go(const TraceArgs& a, int block, int grid, cudaStream_t s)
{
    if (a.S <= 1) k_trace<4, MODE, U, 1><<<grid, block, 0, s>>>(a);
    else if (a.S <= 2) k_trace<4, MODE, U, 2><<<grid, block, 0, s>>>(a);
    else if (a.S <= 4) k_trace<4, MODE, U, 4><<<grid, block, 0, s>>>(a);
    else k_trace<4, MODE, U, 8><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_epilogue(const TraceArgs& a, int mode, int block, int grid, cudaStream_t s)
{
    const bool u = a.t.uniform_level >= 0;
    if (mode == RT_MODE_FP64) return u ? go<RT_MODE_FP64, true>(a, block, grid, s) : go<RT_MODE_FP64, false>(a, block, grid, s);
    return u ? go<RT_MODE_F32_KAHAN, true>(a, block, grid, s) : go<RT_MODE_F32_KAHAN, false>(a, block, grid, s);
}

template <int MODE, bool U, int SM>
static int occ(int block)
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<4, MODE, U, SM>, block, 0);
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

int occupancy_epi(int mode, int S, bool u, int block)
{
    if (mode == RT_MODE_FP64) return u ? occ_s<RT_MODE_FP64, true>(S, block) : occ_s<RT_MODE_FP64, false>(S, block);
    return u ? occ_s<RT_MODE_F32_KAHAN, true>(S, block) : occ_s<RT_MODE_F32_KAHAN, false>(S, block);
}

// out[p] <- -(1/gamma) ln(out[p] / n_dirs) (A_V,eff) or out[p] / n_dirs (beta).
__global__ void k_epilogue_finish(double* out, long long n, int kind, double inv_nd, double inv_gamma)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const double m = out[p] * inv_nd;
        out[p] = (kind == RT_EPI_AV_EFF) ? -log(m) * inv_gamma : m;
    }
}

}  // namespace rt

using namespace rt;

extern "C" int rt_trace_epilogue(const rt_octree* t, const double* d_src, int64_t n_src, int nside, const void* d_dens,
                                 int n_species, int dens_dtype, int mode, const rt_epilogue* h_epi, double* d_out,
                                 void* stream)
{
    if (!h_epi || (h_epi->kind != RT_EPI_AV_EFF && h_epi->kind != RT_EPI_BETA && h_epi->kind != RT_EPI_ATTENUATION))
        return set_error(RT_ERR_ARG, "rt_trace_epilogue: unknown epilogue");
    if (h_epi->kind == RT_EPI_AV_EFF && !(h_epi->gamma > 0.0))
        return set_error(RT_ERR_ARG, "rt_trace_epilogue: gamma must be positive");
    if (dens_dtype != RT_F32 && dens_dtype != RT_F64) return set_error(RT_ERR_ARG, "rt_trace_epilogue: bad dens_dtype");
    TraceArgs a;
    int st = prepare_trace(t, d_src, n_src, nside, n_species, mode, a, "rt_trace_epilogue");
    if (st != RT_OK) return st;
    if (n_src == 0) return RT_OK;
    if (!d_dens || !d_out || ((uintptr_t)d_dens & 15u) || ((uintptr_t)d_out & 7u))
        return set_error(RT_ERR_ARG, "rt_trace_epilogue: null or misaligned densities or output");
    a.dens = d_dens;
    a.dens_f64 = dens_dtype == RT_F64;
    a.out = d_out;
    a.epi_kind = h_epi->kind;
    for (int k = 0; k < kMaxSpecies; k++) a.epi_w[k] = k < n_species ? h_epi->weights[k] : 0.0;
    a.epi_a = h_epi->a;
    a.epi_gamma = h_epi->gamma;
    a.epi_coef = h_epi->d_coef;
    cudaStream_t s = (cudaStream_t)stream;
    if (h_epi->kind != RT_EPI_ATTENUATION &&
        cudaMemsetAsync(d_out, 0, sizeof(double) * (size_t)n_src, s) != cudaSuccess)
        return cuda_error("rt_trace_epilogue: clear");
    const int cs = check_densities(d_dens, t->dev.n, n_species, a.dens_f64, 0, t->st, s);
    if (cs != RT_OK) return cs;
    int block, bps, groups;
    launch_shape(&block, &bps, &groups);
    int dev = 0;
    cudaGetDevice(&dev);
    const int fit = occupancy_epi(mode, n_species, a.t.uniform_level >= 0, block);
    const int grid = sm_count_of(dev) * std::max(1, bps > 0 ? std::min(bps, fit) : fit);
    if (cudaMemsetAsync(&t->st->queue, 0, sizeof(unsigned long long), s) != cudaSuccess ||
        launch_epilogue(a, mode, block, grid, s) != cudaSuccess)
        return cuda_error("rt_trace_epilogue: launch");
    if (h_epi->kind != RT_EPI_ATTENUATION) {
        const int g2 = (int)std::min<long long>((n_src + 255) / 256, 4096);
        k_epilogue_finish<<<g2, 256, 0, s>>>(d_out, n_src, h_epi->kind, 1.0 / a.nd,
                                             h_epi->kind == RT_EPI_AV_EFF ? 1.0 / h_epi->gamma : 0.0);
        if (cudaGetLastError() != cudaSuccess) return cuda_error("rt_trace_epilogue: finish");
    }
    return RT_OK;
}
