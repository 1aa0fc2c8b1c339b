// Forward trace over a chunked contribution grid (Alg. 1 of arXiv 2605.09882:
// the contribution grid is split into chunks, the chunks are traversed one at
// a time, every ray from a source inside the cloud walks the part of its path
// that lies in the current chunk and adds that chunk's partial integral to
// I(p, q); sources outside the cloud get I(p, q) = 0).
//
// Chunks are contiguous ranges of the Morton-sorted leaf array (so each is the
// union of aligned octree cells).  The octree index (keys, levels, coarse
// table) stays on the device; the densities, which dominate the tree's
// memory for many species, are streamed one chunk at a time from host memory
// through two device buffers (the next chunk's copy overlaps the current
// chunk's pass), or read in place if they are already on the device.
//
// Instead of restarting a ray at its entry into each chunk, every ray keeps
// the state of its walk at the top of the step loop (leaf, box, entry time,
// segment count, path hash) and its running column sums between passes: it
// stops when its next leaf lies outside the chunk and resumes there when that
// chunk comes round.  The walk and the order of the additions are therefore
// exactly those of the unchunked trace, and so are the paths and the columns
// (bit for bit).  A ray may leave a chunk and come back to it later, so the
// chunks are swept in order until every ray has finished.
#include <vector>

#include "rt_host.h"
#include "rt_kernels.cuh"

namespace rt {

struct ChunkArgs {
    DevTree t;
    const DirConst* dirs;
    int nd;
    const double* src;
    int64_t n_src, n_src_pad;
    const uint8_t* mask;    // [n_src] nonzero: the source is inside the cloud; NULL: all are
    const void* dens;       // densities of the chunk's leaves [j1 - j0][S]
    int dens_f64, S;
    long long j0, j1;       // the chunk: leaves [j0, j1)
    void* out;              // running columns [n_src][nd][S]
    float* cmp;             // F32-Kahan compensations [n_src * nd][S]
    RayState* rs;           // [n_src * nd]
    uint32_t* nseg;         // optional per-ray outputs, written when a ray finishes
    uint64_t* hash;
    DevStats* st;
    unsigned long long* done;  // rays finished
    // per-chunk queues of the rays waiting at a leaf of that chunk: the pass of
    // chunk c walks queue c (the first pass of all walks every ray); a ray
    // that stops appends itself to the queue of its next leaf's chunk
    uint32_t* queues;          // [n_chunks][n_rays]
    unsigned long long* qcount;  // [n_chunks]
    const long long* bounds;   // [n_chunks + 1] first leaf of every chunk
    long long n_rays;
    int n_chunks, chunk, fresh;
    int batch, layout;
};

// Chunk of leaf j: the last c with bounds[c] <= j.
__device__ __forceinline__ int chunk_of(const long long* __restrict__ bounds, int n_chunks, long long j)
{
    int lo = 0, hi = n_chunks;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(bounds + mid) <= j) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Column sums that continue from the ray's running values, reading the
// densities of chunk leaves (index j - j0 in the chunk buffer), and the path
// fingerprint.
template <int MODE, int SM>
struct ChunkCols {
    using T = typename std::conditional<MODE == RT_MODE_FP64, double, float>::type;
    T sum[SM], cmp[SM], n[SM];
    uint64_t h;
    const void* dens;
    long long j0;
    int f64, S;
    __device__ __forceinline__ void pre(uint32_t j)
    {
        h = (h ^ (uint64_t)j) * 0x100000001b3ull;
        load_dens<SM, T>(dens, f64, S, (uint32_t)((long long)j - j0), n);
    }
    template <class F>
    __device__ __forceinline__ void acc(F dsin)
    {
        if (MODE == RT_MODE_FP64) {
            const double ds = (double)dsin;
#pragma unroll
            for (int k = 0; k < SM; k++) sum[k] = __dadd_rn((double)sum[k], __dmul_rn((double)n[k], ds));
        } else {
            const float ds = (float)dsin;
#pragma unroll
            for (int k = 0; k < SM; k++) {
                const float y = __fmaf_rn((float)n[k], ds, -(float)cmp[k]);
                const float tt = __fadd_rn((float)sum[k], y);
                cmp[k] = __fsub_rn(__fsub_rn(tt, (float)sum[k]), y);
                sum[k] = tt;
            }
        }
    }
    template <class F>
    __device__ __forceinline__ void seg(uint32_t j, F ds) { pre(j); acc(ds); }
};

// One pass: every unfinished ray whose walk is at a leaf of the chunk (or that
// has not started) walks until its next leaf lies outside the chunk or the ray
// leaves the domain.
#ifndef RT_MIN_BLOCKS_CHUNK
#define RT_MIN_BLOCKS_CHUNK 3
#endif
template <int MODE, int SM>
__global__ void __launch_bounds__(256, RT_MIN_BLOCKS_CHUNK) k_chunk_pass(const ChunkArgs a)
{
    using T = typename std::conditional<MODE == RT_MODE_FP64, double, float>::type;
    if (MODE == RT_MODE_F32_KAHAN) fill_spread_table();
    const int lane = threadIdx.x & 31;
    const unsigned long long total = a.fresh ? (unsigned long long)(a.layout ? a.n_src : a.n_src_pad) * (unsigned long long)a.nd
                                             : *(volatile unsigned long long*)(a.qcount + a.chunk);
    const uint32_t* myq = a.queues + (size_t)a.chunk * (size_t)a.n_rays;
    unsigned long long n_rays = 0, n_segs = 0, n_efb = 0, n_lfb = 0, n_done = 0;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&a.st->queue, 32ull * (unsigned)a.batch);
        base = __shfl_sync(RT_FULL, base, 0);
        if (base >= total) break;
        for (int kk = 0; kk < a.batch; kk++) {
            const unsigned long long g0 = base + 32ull * kk;
            if (g0 >= total) break;
            int q;
            long long s;
            if (!a.fresh) {
                if (g0 + lane >= total) continue;
                const long long r = (long long)__ldg(myq + g0 + lane);
                s = r / a.nd;
                q = (int)(r - s * a.nd);
            } else if (a.layout == 0) {
                q = (int)(g0 / (unsigned long long)a.n_src_pad);
                s = (long long)(g0 - (unsigned long long)q * a.n_src_pad) + lane;
                if (s >= a.n_src) continue;
            } else {
                const unsigned long long r = g0 + lane;
                if (r >= total) continue;
                s = (long long)(r / (unsigned long long)a.nd);
                q = (int)(r - (unsigned long long)s * a.nd);
            }
            const long long ray = s * a.nd + q;
            RayState* rp = a.rs + ray;
            const uint32_t jw = rp->j;
            const uint8_t status = rp->status;
            if (status == 2) continue;                                 // finished
            if (status == 1 && ((long long)jw < a.j0 || (long long)jw >= a.j1)) continue;  // waits for its chunk
            T* o = (T*)a.out + (size_t)ray * a.S;
            if (status == 0 && a.mask && !__ldg(a.mask + s)) {         // outside the cloud: I = 0
#pragma unroll
                for (int k = 0; k < SM; k++)
                    if (k < a.S) o[k] = (T)0;
                if (a.nseg) a.nseg[ray] = 0u;
                if (a.hash) a.hash[ray] = 0ull;
                rp->status = 2;
                n_done++;
                continue;
            }
            RayState rs = *rp;
            ChunkCols<MODE, SM> v;
            v.dens = a.dens; v.j0 = a.j0; v.f64 = a.dens_f64; v.S = a.S;
            float* cp = a.cmp ? a.cmp + (size_t)ray * a.S : nullptr;
#pragma unroll
            for (int k = 0; k < SM; k++) {
                v.sum[k] = v.cmp[k] = (T)0;
                if (status == 1 && k < a.S) {
                    v.sum[k] = o[k];
                    if (MODE != RT_MODE_FP64) v.cmp[k] = (T)cp[k];
                }
            }
            v.h = status == 1 ? rs.hash : 0xcbf29ce484222325ull;
            if (status == 0) rs.nseg = 0;
            WalkCounters wc = {rs.nseg, 0u, 0u};
            ChunkResume cr = {&rs, a.j0, a.j1};
            const int st = walk_chunk<MODE>(a.t, a.dirs + q, a.src + 3 * s, a.t.step_cap, v, wc, &cr);
            n_segs += wc.nseg - (status == 1 ? rp->nseg : 0u);
            n_efb += wc.exit_fb;
            n_lfb += wc.lookup_fb;
            if (st == kSuspended) {
                rs.status = 1;
                rs.hash = v.h;
                // join the queue of the next leaf's chunk (one atomic per
                // chunk per warp)
                const int cn = chunk_of(a.bounds, a.n_chunks, (long long)rs.j);
                const unsigned am = __activemask();
                const unsigned peers = __match_any_sync(am, cn);
                const int leader = __ffs(peers) - 1;
                unsigned long long slot = 0;
                if (lane == leader) slot = atomicAdd(a.qcount + cn, (unsigned long long)__popc(peers));
                slot = __shfl_sync(peers, slot, leader) + __popc(peers & ((1u << lane) - 1u));
                a.queues[(size_t)cn * (size_t)a.n_rays + slot] = (uint32_t)ray;
#pragma unroll
                for (int k = 0; k < SM; k++) {
                    if (k < a.S) {
                        o[k] = v.sum[k];
                        if (MODE != RT_MODE_FP64) cp[k] = (float)v.cmp[k];
                    }
                }
                *rp = rs;
                continue;
            }
            if (st != RT_OK) {
                report_fault(a.st, st, ray);
#pragma unroll
                for (int k = 0; k < SM; k++) v.sum[k] = (T)0;
                v.h = 0ull;
                wc.nseg = 0;
            }
#pragma unroll
            for (int k = 0; k < SM; k++)
                if (k < a.S) o[k] = v.sum[k];
            if (a.nseg) a.nseg[ray] = wc.nseg;
            if (a.hash) a.hash[ray] = v.h;
            rp->status = 2;
            n_rays++;
            n_done++;
        }
    }
    flush_counters(a.st, n_rays, n_segs, n_efb, n_lfb);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_done += __shfl_down_sync(RT_FULL, n_done, o);
    if (lane == 0 && n_done) atomicAdd(a.done, n_done);
}

template <int MODE>
static cudaError_t launch_pass(const ChunkArgs& a, int grid, cudaStream_t s)
{
    if (a.S <= 1) k_chunk_pass<MODE, 1><<<grid, 256, 0, s>>>(a);
    else if (a.S <= 2) k_chunk_pass<MODE, 2><<<grid, 256, 0, s>>>(a);
    else if (a.S <= 4) k_chunk_pass<MODE, 4><<<grid, 256, 0, s>>>(a);
    else k_chunk_pass<MODE, 8><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <int MODE, int SM>
static int pass_occ()
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_chunk_pass<MODE, SM>, 256, 0);
    return n;
}

static int pass_occupancy(int mode, int S)
{
    const int sm = S <= 1 ? 1 : S <= 2 ? 2 : S <= 4 ? 4 : 8;
    if (mode == RT_MODE_FP64)
        return sm == 1 ? pass_occ<RT_MODE_FP64, 1>() : sm == 2 ? pass_occ<RT_MODE_FP64, 2>()
             : sm == 4 ? pass_occ<RT_MODE_FP64, 4>() : pass_occ<RT_MODE_FP64, 8>();
    return sm == 1 ? pass_occ<RT_MODE_F32_KAHAN, 1>() : sm == 2 ? pass_occ<RT_MODE_F32_KAHAN, 2>()
         : sm == 4 ? pass_occ<RT_MODE_F32_KAHAN, 4>() : pass_occ<RT_MODE_F32_KAHAN, 8>();
}

}  // namespace rt

using namespace rt;

extern "C" int rt_trace_columns_chunked(const rt_octree* t, const double* d_src, int64_t n_src, int nside,
                                        const void* dens, int n_species, int dens_dtype, int mode,
                                        const uint8_t* d_mask, int n_chunks, void* d_out, uint32_t* d_nseg,
                                        uint64_t* d_hash, void* stream)
{
    TraceArgs a;
    int st = prepare_trace(t, d_src, n_src, nside, n_species, mode, a, "rt_trace_columns_chunked");
    if (st != RT_OK) return st;
    if (dens_dtype != RT_F32 && dens_dtype != RT_F64)
        return set_error(RT_ERR_ARG, "rt_trace_columns_chunked: bad dens_dtype");
    if (n_chunks < 1 || (int64_t)n_chunks > t->dev.n)
        return set_error(RT_ERR_ARG, "rt_trace_columns_chunked: n_chunks must be in [1, n_leaves]");
    if (n_src == 0) return RT_OK;
    if (!dens || !d_out || ((uintptr_t)d_out & 15u) || ((uintptr_t)dens & 15u))
        return set_error(RT_ERR_ARG, "rt_trace_columns_chunked: densities and output must be non-null and 16-byte aligned");
    cudaPointerAttributes pa;
    bool on_device = false;
    if (cudaPointerGetAttributes(&pa, dens) == cudaSuccess)
        on_device = pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
    cudaGetLastError();  // an unregistered host pointer may leave an error behind
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = t->dev.n;
    const int64_t n_rays = n_src * a.nd;
    const size_t dsz = dens_dtype == RT_F64 ? 8 : 4;
    int64_t max_chunk = 0;
    for (int c = 0; c < n_chunks; c++)
        max_chunk = std::max<int64_t>(max_chunk, n * (c + 1) / n_chunks - n * c / n_chunks);
    const size_t rs_bytes = ((size_t)n_rays * sizeof(RayState) + 255) / 256 * 256;
    const size_t cmp_bytes = mode == RT_MODE_FP64 ? 0 : ((size_t)n_rays * n_species * 4 + 255) / 256 * 256;
    const size_t buf_bytes = on_device ? 0 : ((size_t)max_chunk * n_species * dsz + 255) / 256 * 256;
    if (n_rays >= (1ll << 32))
        return set_error(RT_ERR_ARG, "rt_trace_columns_chunked: 2^32 or more rays in one call");
    const size_t head_bytes = ((size_t)(2 * n_chunks + 2) * 8 + 255) / 256 * 256;  // done, counts, bounds
    const size_t q_bytes = ((size_t)n_chunks * n_rays * 4 + 255) / 256 * 256;
    char* scratch = nullptr;
    if (cudaMalloc(&scratch, head_bytes + rs_bytes + cmp_bytes + q_bytes + 2 * buf_bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_error(RT_ERR_OOM, "rt_trace_columns_chunked: the ray states do not fit in device memory");
    }
    unsigned long long* done = (unsigned long long*)scratch;
    unsigned long long* qcount = done + 1;
    long long* bounds = (long long*)(qcount + n_chunks);
    RayState* rs = (RayState*)(scratch + head_bytes);
    float* cmp = mode == RT_MODE_FP64 ? nullptr : (float*)(scratch + head_bytes + rs_bytes);
    uint32_t* queues = (uint32_t*)(scratch + head_bytes + rs_bytes + cmp_bytes);
    char* buf[2] = {scratch + head_bytes + rs_bytes + cmp_bytes + q_bytes,
                    scratch + head_bytes + rs_bytes + cmp_bytes + q_bytes + buf_bytes};
    std::vector<long long> h_bounds(n_chunks + 1);
    for (int c = 0; c <= n_chunks; c++) h_bounds[c] = n * c / n_chunks;
    cudaStream_t cs = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, used[2] = {nullptr, nullptr};
    if (!on_device) {
        cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        for (int i = 0; i < 2; i++) {
            cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming);
            cudaEventCreateWithFlags(&used[i], cudaEventDisableTiming);
        }
    }
    ChunkArgs c;
    memset(&c, 0, sizeof c);
    c.t = a.t;
    c.t.uniform_level = -1;  // the general-octree walk (the same leaves and lengths as the grid walks)
    c.dirs = a.dirs;
    c.nd = a.nd;
    c.src = d_src;
    c.n_src = n_src;
    c.n_src_pad = a.n_src_pad;
    c.mask = d_mask;
    c.dens_f64 = dens_dtype == RT_F64;
    c.S = n_species;
    c.out = d_out;
    c.cmp = cmp;
    c.rs = rs;
    c.nseg = d_nseg;
    c.hash = d_hash;
    c.st = t->st;
    c.done = done;
    c.queues = queues;
    c.qcount = qcount;
    c.bounds = bounds;
    c.n_rays = n_rays;
    c.n_chunks = n_chunks;
    c.batch = a.batch;
    c.layout = a.layout;
    int dev = 0;
    cudaGetDevice(&dev);
    const int grid = sm_count_of(dev) * std::max(1, pass_occupancy(mode, n_species));
    unsigned long long h_done = 0, last_done = 0, h_segs = 0, last_segs = ~0ull;
    DevStats hst;
    st = RT_OK;
    if (cudaMemsetAsync(scratch, 0, head_bytes + rs_bytes, s) != cudaSuccess ||
        cudaMemcpyAsync(bounds, h_bounds.data(), sizeof(long long) * (n_chunks + 1), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        st = cuda_error("rt_trace_columns_chunked: state reset");
    for (int sweep = 0; st == RT_OK; sweep++) {
        for (int k = 0; k < n_chunks && st == RT_OK; k++) {
            const int64_t j0 = n * k / n_chunks, j1 = n * (k + 1) / n_chunks;
            c.j0 = j0;
            c.j1 = j1;
            c.chunk = k;
            c.fresh = sweep == 0 && k == 0;
            if (on_device) {
                c.dens = (const char*)dens + (size_t)j0 * n_species * dsz;
            } else {
                // copy chunk k into buffer k % 2 once the pass that last read it is done
                const int b = k & 1;
                cudaStreamWaitEvent(cs, used[b], 0);
                if (cudaMemcpyAsync(buf[b], (const char*)dens + (size_t)j0 * n_species * dsz,
                                    (size_t)(j1 - j0) * n_species * dsz, cudaMemcpyHostToDevice, cs) != cudaSuccess) {
                    st = cuda_error("rt_trace_columns_chunked: density chunk copy");
                    break;
                }
                cudaEventRecord(copied[b], cs);
                cudaStreamWaitEvent(s, copied[b], 0);
                c.dens = buf[b];
            }
            if (sweep == 0 &&
                (st = check_densities(c.dens, j1 - j0, n_species, c.dens_f64, j0, t->st, s)) != RT_OK)
                break;
            if (cudaMemsetAsync(&t->st->queue, 0, sizeof(unsigned long long), s) != cudaSuccess ||
                (mode == RT_MODE_FP64 ? launch_pass<RT_MODE_FP64>(c, grid, s)
                                      : launch_pass<RT_MODE_F32_KAHAN>(c, grid, s)) != cudaSuccess) {
                st = cuda_error("rt_trace_columns_chunked: pass launch");
                break;
            }
            // queue k has been walked; rays that come back to chunk k join it anew
            if (cudaMemsetAsync(qcount + k, 0, sizeof(unsigned long long), s) != cudaSuccess) {
                st = cuda_error("rt_trace_columns_chunked: queue reset");
                break;
            }
            if (!on_device) cudaEventRecord(used[k & 1], s);
        }
        if (st != RT_OK) break;
        if (cudaMemcpyAsync(&h_done, done, sizeof h_done, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&hst, t->st, sizeof hst, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = cuda_error("rt_trace_columns_chunked: progress readback");
            break;
        }
        h_segs = hst.segments;
        if (h_done >= (unsigned long long)n_rays) break;
        if (h_done == last_done && h_segs == last_segs) {  // a sweep that moved no ray: never for a valid octree
            st = set_error(RT_ERR_CUDA, "rt_trace_columns_chunked: a sweep over the chunks made no progress");
            break;
        }
        last_done = h_done;
        last_segs = h_segs;
    }
    if (cs) {
        cudaStreamSynchronize(cs);
        cudaStreamDestroy(cs);
        for (int i = 0; i < 2; i++) {
            cudaEventDestroy(copied[i]);
            cudaEventDestroy(used[i]);
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(scratch);
    if (st == RT_OK) clear_error();
    return st;
}
