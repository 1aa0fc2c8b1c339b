// End-to-end forward trace from host buffers: the octree, densities and
// sources are copied in, the octree is indexed, and the sources are traced in
// chunks whose input copy, trace and output copy run on three streams, so the
// host<->device traffic of one chunk hides under the trace of another.  The
// device buffers, streams and events persist per device between calls (they
// grow on demand) until rt_trace_columns_host_release.
#include <map>
#include <mutex>
#include <vector>

#include "rt_host.h"

using namespace rt;

namespace {

enum { kKeys, kLevels, kDens, kSrc, kOut0, kOut1, kBufs };

struct Workspace {
    void* buf[kBufs] = {};
    size_t cap[kBufs] = {};
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t dens_in = nullptr;
    std::vector<cudaEvent_t> ev;  // per chunk: source in, traced, output out

    void release()
    {
        if (up) cudaStreamSynchronize(up);
        if (down) cudaStreamSynchronize(down);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        ev.clear();
        if (dens_in) cudaEventDestroy(dens_in);
        if (up) cudaStreamDestroy(up);
        if (down) cudaStreamDestroy(down);
        up = down = nullptr;
        dens_in = nullptr;
        for (int i = 0; i < kBufs; i++) {
            cudaFree(buf[i]);
            buf[i] = nullptr;
            cap[i] = 0;
        }
    }
};

std::mutex g_mu;
std::map<int, Workspace> g_ws;

// Buffer i of at least `need` bytes (contents not kept when it grows).
bool reserve(Workspace& w, int i, size_t need)
{
    if (w.cap[i] >= need) return true;
    cudaFree(w.buf[i]);
    w.buf[i] = nullptr;
    w.cap[i] = 0;
    if (cudaMalloc(&w.buf[i], need) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    w.cap[i] = need;
    return true;
}

// Destroys the per-call octree and waits for the copy streams on every exit.
struct CallGuard {
    Workspace& w;
    cudaStream_t cs;
    rt_octree* tree = nullptr;
    ~CallGuard()
    {
        cudaStreamSynchronize(cs);
        if (w.up) cudaStreamSynchronize(w.up);
        if (w.down) cudaStreamSynchronize(w.down);
        if (tree) rt_destroy_octree(tree);
    }
};

}  // namespace

extern "C" int rt_trace_columns_host(const uint64_t* h_keys, const uint8_t* h_levels, int64_t n_leaves,
                                     const int32_t* h_extent, const double* h_src, int64_t n_src, int nside,
                                     const void* h_dens, int n_species, int dens_dtype, int mode, void* h_out,
                                     int64_t chunk_src, rt_stats* h_stats, void* stream)
{
    const char* who = "rt_trace_columns_host";
    if (!h_keys || !h_levels || !h_dens || (n_src > 0 && (!h_src || !h_out)))
        return set_error(RT_ERR_ARG, "rt_trace_columns_host: null host pointer");
    if (n_leaves <= 0 || n_src < 0 || chunk_src < 0)
        return set_error(RT_ERR_ARG, "rt_trace_columns_host: bad sizes");
    if (n_species < 1 || n_species > kMaxSpecies)
        return set_error(RT_ERR_ARG, "rt_trace_columns_host: n_species must be in [1, 8]");
    if (dens_dtype != RT_F32 && dens_dtype != RT_F64) return set_error(RT_ERR_ARG, "rt_trace_columns_host: bad dens_dtype");
    if (mode != RT_MODE_FP64 && mode != RT_MODE_F32_KAHAN) return set_error(RT_ERR_ARG, "rt_trace_columns_host: unknown mode");
    if (nside < 1 || nside > 8192) return set_error(RT_ERR_ARG, "rt_trace_columns_host: bad nside");
    const int S = n_species;
    const int64_t nd = 12ll * nside * nside;
    const size_t dsz = dens_dtype == RT_F64 ? 8 : 4;
    const size_t osz = mode == RT_MODE_FP64 ? 8 : 4;
    // chunk: a multiple of 32 sources, about an eighth of them by default and
    // never more than 1024 chunks
    int64_t chunk = chunk_src ? chunk_src : (n_src + 7) / 8;
    chunk = std::max<int64_t>(chunk, (n_src + 1023) / 1024);
    chunk = std::max<int64_t>(32, (chunk + 31) / 32 * 32);
    const int64_t n_chunks = n_src ? (n_src + chunk - 1) / chunk : 0;
    const size_t out_chunk = (size_t)std::min<int64_t>(chunk, n_src) * nd * S * osz;

    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace& w = g_ws[dev];
    cudaStream_t cs = (cudaStream_t)stream;
    CallGuard guard{w, cs};
    if (!w.up && (cudaStreamCreateWithFlags(&w.up, cudaStreamNonBlocking) != cudaSuccess ||
                  cudaStreamCreateWithFlags(&w.down, cudaStreamNonBlocking) != cudaSuccess ||
                  cudaEventCreateWithFlags(&w.dens_in, cudaEventDisableTiming) != cudaSuccess))
        return cuda_error(who);
    while ((int64_t)w.ev.size() < 3 * n_chunks) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return cuda_error(who);
        w.ev.push_back(e);
    }
    if (!reserve(w, kKeys, sizeof(uint64_t) * n_leaves) || !reserve(w, kLevels, n_leaves) ||
        !reserve(w, kDens, dsz * S * n_leaves) || (n_src && !reserve(w, kSrc, sizeof(double) * 3 * n_src)) ||
        (n_src && !reserve(w, kOut0, out_chunk)) || (n_chunks > 1 && !reserve(w, kOut1, out_chunk)))
        return set_error(RT_ERR_OOM, "rt_trace_columns_host: device allocation");
    uint64_t* keys = (uint64_t*)w.buf[kKeys];
    uint8_t* levels = (uint8_t*)w.buf[kLevels];
    void* dens = w.buf[kDens];
    double* src = (double*)w.buf[kSrc];
    void* out[2] = {w.buf[kOut0], w.buf[kOut1]};

    // octree in on the compute stream, densities alongside on the upload
    // stream; the index build waits for both (it synchronizes the device)
    if (cudaMemcpyAsync(keys, h_keys, sizeof(uint64_t) * n_leaves, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaMemcpyAsync(levels, h_levels, n_leaves, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaMemcpyAsync(dens, h_dens, dsz * S * n_leaves, cudaMemcpyHostToDevice, w.up) != cudaSuccess ||
        cudaEventRecord(w.dens_in, w.up) != cudaSuccess)
        return cuda_error(who);
    int st = rt_build_octree(keys, levels, n_leaves, h_extent, stream, &guard.tree);
    if (st != RT_OK) return st;
    // the source chunks follow on the upload stream, in order, under the
    // traces of the chunks before them
    for (int64_t c = 0; c < n_chunks; c++) {
        const int64_t s0 = c * chunk, n = std::min(chunk, n_src - s0);
        if (cudaMemcpyAsync(src + 3 * s0, h_src + 3 * s0, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, w.up) !=
                cudaSuccess ||
            cudaEventRecord(w.ev[3 * c], w.up) != cudaSuccess)
            return cuda_error(who);
    }
    if ((st = rt_reset_stats(guard.tree, stream)) != RT_OK) return st;
    if (cudaStreamWaitEvent(cs, w.dens_in, 0) != cudaSuccess) return cuda_error(who);
    if ((st = check_densities(dens, n_leaves, S, dens_dtype == RT_F64, 0, guard.tree->st, cs)) != RT_OK) return st;
    for (int64_t c = 0; c < n_chunks; c++) {
        const int64_t s0 = c * chunk, n = std::min(chunk, n_src - s0);
        void* slot = out[c & 1];
        // the trace of chunk c waits for its sources and for its output slot
        // to have been copied out (chunk c - 2)
        if (cudaStreamWaitEvent(cs, w.ev[3 * c], 0) != cudaSuccess ||
            (c >= 2 && cudaStreamWaitEvent(cs, w.ev[3 * (c - 2) + 2], 0) != cudaSuccess))
            return cuda_error(who);
        st = trace_columns_impl(guard.tree, src + 3 * s0, n, nside, dens, S, dens_dtype, mode, slot, stream, false);
        if (st != RT_OK) return st;
        const size_t bytes = (size_t)n * nd * S * osz;
        if (cudaEventRecord(w.ev[3 * c + 1], cs) != cudaSuccess ||
            cudaStreamWaitEvent(w.down, w.ev[3 * c + 1], 0) != cudaSuccess ||
            cudaMemcpyAsync((char*)h_out + (size_t)s0 * nd * S * osz, slot, bytes, cudaMemcpyDeviceToHost, w.down) !=
                cudaSuccess ||
            cudaEventRecord(w.ev[3 * c + 2], w.down) != cudaSuccess)
            return cuda_error(who);
    }
    if (cudaStreamSynchronize(w.down) != cudaSuccess || cudaStreamSynchronize(cs) != cudaSuccess)
        return cuda_error(who);
    rt_stats stats;
    if ((st = rt_get_stats(guard.tree, &stats, stream)) != RT_OK) return st;
    if (h_stats) *h_stats = stats;
    if (stats.status == RT_ERR_NONFINITE)
        return set_error(stats.status, "rt_trace_columns_host: a density is NaN, infinite or negative (its leaf is "
                                       "the statistics' fault position)");
    if (stats.status != RT_OK)
        return set_error(stats.status, "rt_trace_columns_host: a ray faulted (its columns are zero; see the statistics)");
    clear_error();
    return RT_OK;
}

extern "C" void rt_trace_columns_host_release(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& kv : g_ws) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(kv.first);
        kv.second.release();
        cudaSetDevice(cur);
    }
    g_ws.clear();
}
