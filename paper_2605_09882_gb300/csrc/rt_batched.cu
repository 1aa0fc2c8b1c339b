// Batched multi-cloud trace: many independent octrees of uneven size and
// depth traced in ONE persistent launch over a single work queue, replayed as
// a CUDA graph {queue reset (memset node), kernel node}; plus the autotuner
// that picks the launch shape (threads per block, blocks per SM, 32-ray
// groups per queue pop) by timing, cached as JSON per (GPU, batch signature).
#include <stdio.h>
#include <stdlib.h>

#include <mutex>
#include <string>
#include <vector>

#include "rt_host.h"
#include "rt_kernels.cuh"

namespace rt {

struct CloudArgs {
    DevTree t;
    const DirConst* dirs;
    const double* src;
    const void* dens;
    void* out;
    int64_t n_src;
    int64_t n_src_pad;
    int nd;
    int S;
    int dens_f64;
    int pad;
};

struct BatchArgs {
    const CloudArgs* clouds;
    const unsigned long long* ray_off;  // [n_clouds + 1] prefix of the padded ray counts
    unsigned long long total;
    DevStats* st;
    int n_clouds;
    int batch;
};

constexpr int kSmemClouds = 1024;  // ray offsets kept in shared memory up to this many clouds

// Resident 256-thread blocks per SM the register budget is sized for.
#ifndef RT_MIN_BLOCKS_BATCHED
#define RT_MIN_BLOCKS_BATCHED 3
#endif

template <int MODE, int SM>
__global__ void __launch_bounds__(256, RT_MIN_BLOCKS_BATCHED) k_batched(const BatchArgs b)
{
    __shared__ unsigned long long s_off[kSmemClouds + 1];
    const bool in_smem = b.n_clouds <= kSmemClouds;
    if (in_smem)
        for (int i = threadIdx.x; i <= b.n_clouds; i += blockDim.x) s_off[i] = b.ray_off[i];
    if (MODE == RT_MODE_F32_KAHAN) fill_spread_table();  // its barrier covers s_off too
    else __syncthreads();
    const unsigned long long* off = in_smem ? s_off : b.ray_off;
    const int lane = threadIdx.x & 31;
    unsigned long long n_rays = 0, n_segs = 0, n_efb = 0, n_lfb = 0;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&b.st->queue, 32ull * (unsigned)b.batch);
        base = __shfl_sync(RT_FULL, base, 0);
        if (base >= b.total) break;
        for (int kk = 0; kk < b.batch; kk++) {
            const unsigned long long g0 = base + 32ull * kk;
            if (g0 >= b.total) break;
            // cloud of this 32-ray group: last c with off[c] <= g0
            int lo = 0, hi = b.n_clouds;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (off[mid] <= g0) lo = mid;
                else hi = mid;
            }
            const CloudArgs& C = b.clouds[lo];
            const unsigned long long local = g0 - off[lo];
            const int64_t pad = C.n_src_pad;
            const int q = (int)(local / (unsigned long long)pad);
            const long long s = (long long)(local - (unsigned long long)q * pad) + lane;
            if (s >= C.n_src) continue;
            const DevTree t = C.t;
            const DirConst* d = C.dirs + q;
            const long long ray = s * C.nd + q;
            const double* src = C.src + 3 * s;
            WalkCounters wc = {0u, 0u, 0u};
            if (MODE == RT_MODE_FP64) {
                FwdF64<SM> v;
                v.dens = C.dens; v.f64 = C.dens_f64; v.S = C.S;
                v.init();
                const int st = t.uniform_level >= 0 ? walk<MODE, true>(t, d, src, t.step_cap, v, wc)
                                                    : walk<MODE, false>(t, d, src, t.step_cap, v, wc);
                if (st != RT_OK) { report_fault(b.st, st, ray); v.init(); }
                double* o = (double*)C.out + (size_t)ray * C.S;
                for (int k = 0; k < SM; k++)
                    if (k < C.S) o[k] = v.col[k];
            } else {
                FwdKahan<SM> v;
                v.dens = C.dens; v.f64 = C.dens_f64; v.S = C.S;
                v.init();
                const int st = t.uniform_level >= 0 ? walk<MODE, true>(t, d, src, t.step_cap, v, wc)
                                                    : walk<MODE, false>(t, d, src, t.step_cap, v, wc);
                if (st != RT_OK) { report_fault(b.st, st, ray); v.init(); }
                float* o = (float*)C.out + (size_t)ray * C.S;
                for (int k = 0; k < SM; k++)
                    if (k < C.S) o[k] = v.sum[k];
            }
            n_rays++;
            n_segs += wc.nseg;
            n_efb += wc.exit_fb;
            n_lfb += wc.lookup_fb;
        }
    }
    flush_counters(b.st, n_rays, n_segs, n_efb, n_lfb);
}

typedef void (*batched_fn)(const BatchArgs);

static batched_fn kernel_for(int mode, int smax)
{
    if (mode == RT_MODE_FP64) {
        if (smax <= 1) return k_batched<RT_MODE_FP64, 1>;
        if (smax <= 2) return k_batched<RT_MODE_FP64, 2>;
        if (smax <= 4) return k_batched<RT_MODE_FP64, 4>;
        return k_batched<RT_MODE_FP64, 8>;
    }
    if (smax <= 1) return k_batched<RT_MODE_F32_KAHAN, 1>;
    if (smax <= 2) return k_batched<RT_MODE_F32_KAHAN, 2>;
    if (smax <= 4) return k_batched<RT_MODE_F32_KAHAN, 4>;
    return k_batched<RT_MODE_F32_KAHAN, 8>;
}

}  // namespace rt

using namespace rt;

struct rt_batch {
    int device, mode, n_clouds, smax;
    unsigned long long total;
    CloudArgs* d_clouds;
    unsigned long long* d_off;
    DevStats* st;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int g_block, g_grid, g_batch;  // launch shape the graph was built with
};

extern "C" {

int rt_batch_create(const rt_cloud_desc* h_desc, int n_clouds, int mode, rt_batch** out)
{
    if (out) *out = nullptr;
    if (!out || !h_desc || n_clouds < 1) return set_error(RT_ERR_ARG, "rt_batch_create: bad arguments");
    if (mode != RT_MODE_FP64 && mode != RT_MODE_F32_KAHAN) return set_error(RT_ERR_ARG, "rt_batch_create: unknown mode");
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<CloudArgs> h(n_clouds);
    std::vector<unsigned long long> off(n_clouds + 1, 0);
    int smax = 1;
    for (int i = 0; i < n_clouds; i++) {
        const rt_cloud_desc& c = h_desc[i];
        char buf[160];
        if (!c.tree || c.tree->device != dev || c.n_src < 0 || c.n_species < 1 || c.n_species > kMaxSpecies ||
            (c.dens_dtype != RT_F32 && c.dens_dtype != RT_F64) ||
            (c.n_src > 0 && (!c.d_src || !c.d_dens || !c.d_out)) ||
            ((uintptr_t)c.d_dens & 15u) || ((uintptr_t)c.d_out & 15u)) {
            snprintf(buf, sizeof buf, "rt_batch_create: cloud %d has a bad descriptor", i);
            return set_error(RT_ERR_ARG, buf);
        }
        int status = RT_OK;
        const DirConst* dirs = direction_table(dev, c.nside, &status);
        if (!dirs) return status;
        CloudArgs& a = h[i];
        memset(&a, 0, sizeof a);
        a.t = c.tree->dev;
        if (!c.tree->uniform_allowed) a.t.uniform_level = -1;
        a.dirs = dirs;
        a.src = c.d_src;
        a.dens = c.d_dens;
        a.out = c.d_out;
        a.n_src = c.n_src;
        a.n_src_pad = (c.n_src + 31) / 32 * 32;
        a.nd = 12 * c.nside * c.nside;
        a.S = c.n_species;
        a.dens_f64 = c.dens_dtype == RT_F64;
        off[i + 1] = off[i] + (unsigned long long)a.n_src_pad * (unsigned long long)a.nd;
        smax = std::max(smax, c.n_species);
    }
    rt_batch* b = (rt_batch*)calloc(1, sizeof(rt_batch));
    b->device = dev;
    b->mode = mode;
    b->n_clouds = n_clouds;
    b->smax = smax;
    b->total = off[n_clouds];
    if (cudaMalloc(&b->d_clouds, sizeof(CloudArgs) * n_clouds) != cudaSuccess ||
        cudaMalloc(&b->d_off, sizeof(unsigned long long) * (n_clouds + 1)) != cudaSuccess ||
        cudaMalloc(&b->st, sizeof(DevStats)) != cudaSuccess ||
        cudaMemcpy(b->d_clouds, h.data(), sizeof(CloudArgs) * n_clouds, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_off, off.data(), sizeof(unsigned long long) * (n_clouds + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->st, 0, sizeof(DevStats)) != cudaSuccess) {
        const int st = cuda_error("rt_batch_create: device allocation");
        if (b->d_clouds) cudaFree(b->d_clouds);
        if (b->d_off) cudaFree(b->d_off);
        if (b->st) cudaFree(b->st);
        free(b);
        return st;
    }
    *out = b;
    clear_error();
    return RT_OK;
}

void rt_batch_destroy(rt_batch* b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_clouds);
    cudaFree(b->d_off);
    cudaFree(b->st);
    free(b);
}

// (Re)builds the graph {memset(queue) -> kernel} for the current launch shape.
static int build_graph(rt_batch* b)
{
    int block, bps, groups;
    launch_shape(&block, &bps, &groups);
    batched_fn fn = kernel_for(b->mode, b->smax);
    int fit = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, block, 0);
    if (fit < 1) fit = 1;
    const int use = bps > 0 ? std::min(bps, fit) : fit;
    const int grid = sm_count_of(b->device) * use;
    if (b->exec && b->g_block == block && b->g_grid == grid && b->g_batch == groups) return RT_OK;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    BatchArgs args;
    args.clouds = b->d_clouds;
    args.ray_off = b->d_off;
    args.total = b->total;
    args.st = b->st;
    args.n_clouds = b->n_clouds;
    args.batch = groups;
    cudaGraphNode_t mset, kern;
    cudaMemsetParams mp;
    memset(&mp, 0, sizeof mp);
    mp.dst = &b->st->queue;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = 2;
    mp.height = 1;
    mp.pitch = 0;
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof kp);
    void* params[1] = {&args};
    kp.func = (void*)fn;
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(block);
    kp.sharedMemBytes = 0;
    kp.kernelParams = params;
    if (cudaGraphCreate(&b->graph, 0) != cudaSuccess ||
        cudaGraphAddMemsetNode(&mset, b->graph, nullptr, 0, &mp) != cudaSuccess ||
        cudaGraphAddKernelNode(&kern, b->graph, &mset, 1, &kp) != cudaSuccess ||
        cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
        return cuda_error("rt_batch_launch: graph build");
    b->g_block = block;
    b->g_grid = grid;
    b->g_batch = groups;
    return RT_OK;
}

int rt_batch_launch(rt_batch* b, void* stream)
{
    if (!b) return set_error(RT_ERR_ARG, "rt_batch_launch: null batch");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != b->device) return set_error(RT_ERR_ARG, "rt_batch_launch: batch was built on another device");
    const int st = build_graph(b);
    if (st != RT_OK) return st;
    if (cudaGraphLaunch(b->exec, (cudaStream_t)stream) != cudaSuccess) return cuda_error("rt_batch_launch: graph launch");
    return RT_OK;
}

int rt_batch_stats(const rt_batch* b, rt_stats* h_out, void* stream)
{
    if (!b || !h_out) return set_error(RT_ERR_ARG, "rt_batch_stats: null argument");
    DevStats d;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&d, b->st, sizeof d, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return cuda_error("rt_batch_stats");
    h_out->rays = d.rays;
    h_out->segments = d.segments;
    h_out->exit_fallbacks = d.exit_fb;
    h_out->lookup_fallbacks = d.lookup_fb;
    h_out->status = d.status;
    h_out->gathered = 0;
    h_out->fault_ray = d.status ? d.fault_ray : -1;
    return RT_OK;
}

int rt_batch_reset_stats(rt_batch* b, void* stream)
{
    if (!b) return set_error(RT_ERR_ARG, "rt_batch_reset_stats: null batch");
    if (cudaMemsetAsync(b->st, 0, sizeof(DevStats), (cudaStream_t)stream) != cudaSuccess)
        return cuda_error("rt_batch_reset_stats");
    return RT_OK;
}

// ----------------------------------------------------------------- autotune

static std::string signature(const rt_batch* b)
{
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, b->device);
    char buf[512];
    snprintf(buf, sizeof buf, "%.255s|%d|mode%d|clouds%d|rays%llu|S%d", p.name, p.multiProcessorCount, b->mode,
             b->n_clouds, (unsigned long long)b->total, b->smax);
    return buf;
}

// Cache file: one entry per line,
//   "<signature>": {"threads": T, "blocks_per_sm": B, "groups_per_pop": G, "seg_per_s": R},
// inside a JSON object.
static bool cache_lookup(const char* path, const std::string& key, int best[3], double* rate)
{
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    const std::string pre = "\"" + key + "\":";
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        const char* p = strstr(line, pre.c_str());
        if (!p) continue;
        if (sscanf(p + pre.size(), " {\"threads\": %d, \"blocks_per_sm\": %d, \"groups_per_pop\": %d, \"seg_per_s\": %lf",
                   &best[0], &best[1], &best[2], rate) == 4) {
            found = true;
            break;
        }
    }
    fclose(f);
    return found;
}

static void cache_store(const char* path, const std::string& key, const int best[3], double rate)
{
    std::vector<std::string> keep;
    FILE* f = fopen(path, "r");
    char line[1024];
    const std::string pre = "\"" + key + "\":";
    if (f) {
        while (fgets(line, sizeof line, f)) {
            std::string l(line);
            while (!l.empty() && (l.back() == '\n' || l.back() == ',' || l.back() == ' ')) l.pop_back();
            if (l.empty() || l == "{" || l == "}" || l.find(pre) != std::string::npos) continue;
            keep.push_back(l);
        }
        fclose(f);
    }
    char buf[512];
    snprintf(buf, sizeof buf, "  %s {\"threads\": %d, \"blocks_per_sm\": %d, \"groups_per_pop\": %d, \"seg_per_s\": %.6e}",
             pre.c_str(), best[0], best[1], best[2], rate);
    keep.push_back(buf);
    const std::string tmp = std::string(path) + ".tmp";
    f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    for (size_t i = 0; i < keep.size(); i++) fprintf(f, "%s%s\n", keep[i].c_str(), i + 1 < keep.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

static double time_launches(rt_batch* b, cudaStream_t s, int reps)
{
    if (rt_batch_launch(b, s) != RT_OK) return -1.0;  // warm-up, also rebuilds the graph
    rt_batch_reset_stats(b, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; r++) rt_batch_launch(b, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    rt_stats st;
    if (rt_batch_stats(b, &st, s) != RT_OK || st.status != RT_OK || ms <= 0.f) return -1.0;
    return (double)st.segments / (ms * 1e-3);
}

int rt_batch_autotune(rt_batch* b, const char* cache_json, int* h_best, double* h_rate, void* stream)
{
    if (!b) return set_error(RT_ERR_ARG, "rt_batch_autotune: null batch");
    cudaStream_t s = (cudaStream_t)stream;
    const std::string key = signature(b);
    int best[3] = {256, 0, 4};
    double rate = 0.0;
    if (!(cache_json && cache_lookup(cache_json, key, best, &rate))) {
        const int blocks[3] = {64, 128, 256};
        for (int bi = 0; bi < 3; bi++) {
            int fit = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kernel_for(b->mode, b->smax), blocks[bi], 0);
            for (int bps = 1; bps <= fit; bps = (bps < 4) ? bps + 1 : bps * 2) {
                rt_set_launch(blocks[bi], bps, 4);
                const double r = time_launches(b, s, 2);
                if (r > rate) { rate = r; best[0] = blocks[bi]; best[1] = bps; best[2] = 4; }
            }
        }
        const int groups[5] = {1, 2, 8, 16, 32};
        for (int gi = 0; gi < 5; gi++) {
            rt_set_launch(best[0], best[1], groups[gi]);
            const double r = time_launches(b, s, 2);
            if (r > rate) { rate = r; best[2] = groups[gi]; }
        }
        if (rate <= 0.0) {
            rt_set_launch(0, 0, 0);
            return set_error(RT_ERR_CUDA, "rt_batch_autotune: no configuration ran");
        }
        if (cache_json) cache_store(cache_json, key, best, rate);
    }
    rt_set_launch(best[0], best[1], best[2]);
    if (h_best) { h_best[0] = best[0]; h_best[1] = best[1]; h_best[2] = best[2]; }
    if (h_rate) *h_rate = rate;
    return RT_OK;
}

// The batch of the last rt_trace_batched call, kept for replays while the
// same descriptors come back (a batch is built synchronously, its graph on
// the first launch).
static std::mutex g_tb_mu;
static rt_batch* g_tb_batch = nullptr;
static std::vector<rt_cloud_desc> g_tb_desc;
static std::vector<unsigned long long> g_tb_gen;  // build numbers of the batch's octrees
static int g_tb_mode = -1;

int rt_trace_batched(const rt_cloud_desc* h_desc, int n_clouds, int mode, void* stream)
{
    if (!h_desc || n_clouds < 1) return set_error(RT_ERR_ARG, "rt_trace_batched: bad arguments");
    std::lock_guard<std::mutex> lk(g_tb_mu);
    int dev = 0;
    cudaGetDevice(&dev);
    bool same = g_tb_batch && g_tb_mode == mode && g_tb_batch->device == dev && (int)g_tb_desc.size() == n_clouds &&
                memcmp(g_tb_desc.data(), h_desc, sizeof(rt_cloud_desc) * n_clouds) == 0;
    for (int i = 0; same && i < n_clouds; i++) same = h_desc[i].tree && h_desc[i].tree->gen == g_tb_gen[i];
    if (!same) {
        rt_batch_destroy(g_tb_batch);
        g_tb_batch = nullptr;
        g_tb_desc.clear();
        g_tb_gen.clear();
        const int st = rt_batch_create(h_desc, n_clouds, mode, &g_tb_batch);
        if (st != RT_OK) return st;
        g_tb_desc.assign(h_desc, h_desc + n_clouds);
        for (int i = 0; i < n_clouds; i++) g_tb_gen.push_back(h_desc[i].tree->gen);
        g_tb_mode = mode;
    }
    return rt_batch_launch(g_tb_batch, stream);
}

int rt_autotune(const rt_cloud_desc* h_desc, int n_clouds, int mode, const char* cache_json)
{
    rt_batch* b = nullptr;
    int st = rt_batch_create(h_desc, n_clouds, mode, &b);
    if (st != RT_OK) return st;
    st = rt_batch_autotune(b, cache_json, nullptr, nullptr, nullptr);
    rt_batch_destroy(b);
    return st;
}

}  // extern "C"
