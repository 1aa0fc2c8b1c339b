// Adjoint as a per-leaf gather, for the geometry where the walk is
// translation invariant: a full cube of equal-level leaves with one source in
// every leaf, source s in leaf s, all at the same offset inside their leaf
// (every leaf-centre source set is one).  The slab exits of the definition,
// t_b = (F_b - Q_b) / m_b, then depend only on F_b - Q_b, which is the same
// list of distances for every source, so along direction q every ray takes the
// same exit-axis sets E_i and the same segment lengths ds_i in the same order;
// only the step at which it leaves the cube depends on the source.  The ray from
// source s therefore visits leaf s + o_i at step i (o_i the summed steps), and
// the transpose of the trace is
//   grad[j,k] = sum_q sum_i [j - o_{q,i} in the cube] g[j - o_{q,i}, q, k] ds_{q,i}.
// Each leaf is summed by one thread in a fixed order (directions, then steps),
// so the result needs no atomics and is the same bits on every run.
//
// The per-direction tables (E_i, ds_i) come from the walk itself, run once per
// direction from the source whose path is the longest (the corner the ray
// starts from), so every ds is bitwise the one the forward walk and the
// scatter adjoint use.  A device check of the sources decides whether the form
// applies; the scatter kernel launched after it runs only if it did not.
//
// Layout: the gradient of the columns arrives as [source (Morton)][q][S].  For
// each direction its slice is first copied into x-major order [z][y][x][S], so
// that the 32 lanes of a warp, which take 32 neighbouring leaves of one x row,
// read 32 neighbouring sources (one contiguous run of 32 S values) at every
// step instead of 32 separate records.  Rows are handed out in 32^3-leaf
// blocks taken in Morton order, so the leaves in flight form a few compact
// blocks and the sources behind them stay in L2.
//
// Tables per direction, from the walk of the corner source: ds_i, the offset
// D_i of the step-i source from the leaf in the x-major index (the summed
// steps against the ray), and for each axis b and each r the first step P_b[r]
// that would put the source more than r cells behind the leaf on b.  A leaf
// with r_b cells of the cube behind it on each axis then gathers the steps
// i < min_b P_b[r_b], with no per-step bounds test.
#include "rt_host.h"
#include "rt_kernels.cuh"

namespace rt {

// 10-bit coordinate of axis 0 of a 30-bit Morton index (inverse of spread10).
__device__ __forceinline__ uint32_t compact10(uint32_t v)
{
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030c30c3u;
    v = (v | (v >> 4)) & 0x0300f00fu;
    v = (v | (v >> 8)) & 0x030000ffu;
    v = (v | (v >> 16)) & 0x3ffu;
    return v;
}

// Per-direction tables, one row of each per direction.
struct GatherTables {
    int* len;        // [nd] steps of the corner source's walk
    int* D;          // [nd][lcap] x-major index offset of the step-i source from the leaf
    void* ds;        // [nd][lcap] segment lengths (float or double)
    int* P;          // [nd][3][pcap] first step beyond r cells behind on axis b
    int lcap, pcap;
};

// Visitor that writes a direction's tables while the walk runs.  Leaf indices
// are level-L Morton indices; an axis stepped when its bits of the index
// changed.  dstep[b] is the x-major index change of one cell against the ray
// on axis b.
template <class T>
struct StepTable {
    T* ds;
    int* D;
    int* P;          // [3][pcap]
    int n, cap, pcap;
    uint32_t prev;
    int cnt[3], dstep[3], off;
    __device__ __forceinline__ void pre(uint32_t j)
    {
        if (n > 0) {
#pragma unroll
            for (int b = 0; b < 3; b++) {
                if ((prev ^ j) & (kDilX << b)) {
                    if (cnt[b] < pcap) P[b * pcap + cnt[b]] = n;
                    cnt[b]++;
                    off += dstep[b];
                }
            }
        }
        if (n < cap) D[n] = off;
        prev = j;
    }
    template <class F>
    __device__ __forceinline__ void acc(F d)
    {
        if (n < cap) ds[n] = (T)d;
        n++;
    }
    template <class F>
    __device__ __forceinline__ void seg(uint32_t j, F d) { pre(j); acc(d); }
};

struct GatherArgs {
    const void* gin;        // [n][nd][S]: float (F32-Kahan) or double (FP64)
    double* grad;           // [n][S], accumulated into
    GatherTables tab;
    unsigned long long* queue;  // [nd] work-queue counters, one per direction
    void* gl;               // [N^3][S] scratch: one direction's slice in x-major order
    const DirConst* dirs;
    DevStats* st;
    long long n;            // leaves = sources
    int nd, S, L;
};

// Sets st->gather_off unless source s lies in leaf s (the Morton index at the
// uniform level L) at the offset source 0 has inside its leaf.
__global__ void k_adj_check(const double* __restrict__ src, long long n, int L, DevStats* st)
{
    const int lane = threadIdx.x & 31;
    const int sh = kDepth - L;
    const long long fmask = (1ll << (sh + 32)) - 1;
    long long f0[3];
#pragma unroll
    for (int b = 0; b < 3; b++) {
        long long q = -1;
        fixed_source(__ldg(src + b), q);
        f0[b] = q & fmask;
    }
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long base = ((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5) * 32; base < n;
         base += warps * 32) {
        const int off = *(volatile int*)&st->gather_off;
        if (__any_sync(RT_FULL, off != 0)) return;  // already decided
        const long long s = base + lane;
        bool bad = false;
        if (s < n) {
#pragma unroll
            for (int b = 0; b < 3; b++) {
                long long q;
                if (!fixed_source(__ldg(src + 3 * s + b), q)) {
                    bad = true;
                } else {
                    const uint32_t cell = compact10((uint32_t)s >> b);
                    bad |= (q >> (sh + 32)) != (long long)cell || (q & fmask) != f0[b];
                }
            }
        }
        if (__any_sync(RT_FULL, bad)) {
            if (lane == 0) atomicOr(&st->gather_off, 1);
            return;
        }
    }
}

// One thread per direction (blocks of one warp, lane 0 only): walks the ray
// from the corner leaf the direction starts from, at source 0's offset inside
// its leaf, and writes the direction's tables.
template <int MODE>
__global__ void k_adj_table(const DevTree t, const DirConst* __restrict__ dirs, int nd, const double* __restrict__ src,
                            GatherTables tab, DevStats* st)
{
    using T = typename std::conditional<MODE == RT_MODE_FP64, double, float>::type;
    const int q = blockIdx.x;
    if (threadIdx.x != 0 || q >= nd) return;
    if (*(volatile int*)&st->gather_off) return;
    const int L = t.uniform_level;
    const int sh = kDepth - L;
    const long long fmask = (1ll << (sh + 32)) - 1;
    const int N = 1 << L;
    const int flags = __ldg(&dirs[q].flags);
    double x[3];
    StepTable<T> rec;
    rec.ds = (T*)tab.ds + (size_t)q * tab.lcap;
    rec.D = tab.D + (size_t)q * tab.lcap;
    rec.P = tab.P + (size_t)q * 3 * tab.pcap;
    rec.n = 0;
    rec.cap = tab.lcap;
    rec.pcap = tab.pcap;
    rec.prev = 0u;
    rec.off = 0;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        long long q0 = 0;
        fixed_source(__ldg(src + b), q0);
        const bool moving = flags & (1 << b), up = (flags >> (3 + b)) & 1;
        const long long cell = (moving && !up) ? N - 1 : 0;
        x[b] = __dmul_rn(__ll2double_rn((cell << (sh + 32)) | (q0 & fmask)), 0x1p-53);  // exact
        const int stride = b == 0 ? 1 : (b == 1 ? N : N * N);
        rec.dstep[b] = up ? -stride : stride;
        rec.cnt[b] = 0;
    }
    WalkCounters wc = {0u, 0u, 0u};
    const int status = walk<MODE, true>(t, dirs + q, x, t.step_cap, rec, wc);
    if (status != RT_OK || rec.n > tab.lcap) atomicOr(&st->gather_off, 2);
    const int n = min(rec.n, tab.lcap);
    tab.len[q] = n;
    // steps an axis never reaches within the walk end every leaf's range at n
#pragma unroll
    for (int b = 0; b < 3; b++)
        for (int r = min(rec.cnt[b], tab.pcap); r < tab.pcap; r++) rec.P[b * tab.pcap + r] = n;
}

// Direction q's slice of the column gradient in x-major order:
// gl[(z N + y) N + x][k] = g[(morton(x, y, z) nd + q) S + k].
template <class T, int SM>
__global__ void k_adj_slice(const T* __restrict__ g, int q, int nd, int L, T* __restrict__ gl)
{
    const uint32_t N = 1u << L;
    const unsigned long long n = 1ull << (3 * L);
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)i & (N - 1u), y = (uint32_t)(i >> L) & (N - 1u), z = (uint32_t)(i >> (2 * L));
        const uint32_t j = spread10(x) | (spread10(y) << 1) | (spread10(z) << 2);
        const T* src = g + ((size_t)j * nd + q) * SM;
        T* dst = gl + (size_t)i * SM;
        if (sizeof(T) == 4 && SM % 4 == 0) {
#pragma unroll
            for (int h = 0; h < SM / 4; h++) ((float4*)dst)[h] = __ldg((const float4*)src + h);
        } else if (sizeof(T) == 4 && SM == 2) {
            *(float2*)dst = __ldg((const float2*)src);
        } else if (sizeof(T) == 8 && SM % 2 == 0) {
#pragma unroll
            for (int h = 0; h < SM / 2; h++) ((double2*)dst)[h] = __ldg((const double2*)src + h);
        } else {
#pragma unroll
            for (int k = 0; k < SM; k++) dst[k] = __ldg(src + k);
        }
    }
}

template <class T, int SM>
__device__ __forceinline__ void load_g(const T* __restrict__ p, T v[SM])
{
    if (sizeof(T) == 4 && SM == 4) {
        const float4 w = __ldg((const float4*)p);
        v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
    } else if (sizeof(T) == 4 && SM == 2) {
        const float2 w = __ldg((const float2*)p);
        v[0] = w.x; v[1] = w.y;
    } else if (sizeof(T) == 8 && SM >= 2) {
#pragma unroll
        for (int h = 0; h < SM / 2; h++) {
            const double2 w = __ldg((const double2*)p + h);
            v[2 * h] = w.x; v[2 * h + 1] = w.y;
        }
    } else if (sizeof(T) == 4 && SM == 8) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const float4 w = __ldg((const float4*)p + h);
            v[4 * h] = w.x; v[4 * h + 1] = w.y; v[4 * h + 2] = w.z; v[4 * h + 3] = w.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < SM; k++) v[k] = __ldg(p + k);
    }
}

// Steps per group of independent gradient loads.
constexpr int kGatherU = 4;

// Accumulates a group of U terms sum_u g[u][k] ds[u]: F32-Kahan forms the
// group's sum with fused multiply-adds and adds it to the accumulator with one
// Kahan step; FP64 takes one fused multiply-add per term.
template <int MODE, int SM, int U, class T>
__device__ __forceinline__ void acc_group(T sum[SM], T cmp[SM], const T gv[U][SM], const T dv[U])
{
#pragma unroll
    for (int k = 0; k < SM; k++) {
        if (MODE == RT_MODE_FP64) {
#pragma unroll
            for (int u = 0; u < U; u++) sum[k] = __fma_rn((double)gv[u][k], (double)dv[u], (double)sum[k]);
        } else {
            float part = __fmul_rn((float)gv[0][k], (float)dv[0]);
#pragma unroll
            for (int u = 1; u < U; u++) part = __fmaf_rn((float)gv[u][k], (float)dv[u], part);
            const float y = __fsub_rn(part, (float)cmp[k]);
            const float tt = __fadd_rn((float)sum[k], y);
            cmp[k] = (T)__fsub_rn(__fsub_rn(tt, (float)sum[k]), y);
            sum[k] = (T)tt;
        }
    }
}

// One thread per leaf and one launch per direction q (launches on one stream
// run in order, so each leaf's gradient takes its directions in a fixed order
// and no two threads update it at once).  A warp takes one x row of 32 leaves;
// each lane gathers g[s_i, q, k] ds_i over the steps i of its range from the
// x-major slice, then adds the sum to the FP64 gradient of its leaf.  S == SM
// exactly.
template <int MODE, int SM>
__global__ void __launch_bounds__(256, 4) k_adj_gather(const GatherArgs a, const int q)
{
    using T = typename std::conditional<MODE == RT_MODE_FP64, double, float>::type;
    if (*(volatile int*)&a.st->gather_off) return;
    if (q == 0 && blockIdx.x == 0 && threadIdx.x == 0) a.st->gathered = 1;
    const int lane = threadIdx.x & 31;
    const int L = a.L;
    const int N = 1 << L;
    const int TY = min(32, N);                       // rows of a block: TY x TY
    const int GX = (N + 31) >> 5;                    // x rows per leaf row of the cube
    const unsigned long long rows = (unsigned long long)GX * N * N;
    const int flags = __ldg(&a.dirs[q].flags);
    const int* __restrict__ Dq = a.tab.D + (size_t)q * a.tab.lcap;
    const T* __restrict__ dq = (const T*)a.tab.ds + (size_t)q * a.tab.lcap;
    const int* __restrict__ Pq = a.tab.P + (size_t)q * 3 * a.tab.pcap;
    const int len = __ldg(a.tab.len + q);
    const T* __restrict__ gl = (const T*)a.gl;
    unsigned long long n_segs = 0, n_rays = 0;
    for (;;) {
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(a.queue + q, 1ull);
        w = __shfl_sync(RT_FULL, w, 0);
        if (w >= rows) break;
        const uint32_t blk = (uint32_t)(w / (unsigned long long)(TY * TY));
        const uint32_t r = (uint32_t)(w % (unsigned long long)(TY * TY));
        const int x = 32 * (int)compact10(blk) + lane;
        const int y = TY * (int)compact10(blk >> 1) + (int)(r % (uint32_t)TY);
        const int z = TY * (int)compact10(blk >> 2) + (int)(r / (uint32_t)TY);
        if (x < N) {  // lanes past the cube's edge (N < 32) sit out
            // the steps whose source stays inside the cube: fewer than the
            // cells behind the leaf on every moving axis
            int ell = len;
            const int c[3] = {x, y, z};
#pragma unroll
            for (int b = 0; b < 3; b++) {
                if (flags & (1 << b)) {
                    const int room = ((flags >> (3 + b)) & 1) ? c[b] : N - 1 - c[b];
                    ell = min(ell, __ldg(Pq + b * a.tab.pcap + room));
                }
            }
            const int idx0 = (z * N + y) * N + x;
            T sum[SM], cmp[SM];
#pragma unroll
            for (int k = 0; k < SM; k++) sum[k] = cmp[k] = (T)0;
            int i = 0;
            for (; i + kGatherU <= ell; i += kGatherU) {
                const int4 d4 = __ldg((const int4*)(Dq + i));
                const int dd[4] = {d4.x, d4.y, d4.z, d4.w};
                T gv[kGatherU][SM], dv[kGatherU];
#pragma unroll
                for (int u = 0; u < kGatherU; u++) load_g<T, SM>(gl + (size_t)(uint32_t)(idx0 + dd[u]) * SM, gv[u]);
                if (MODE == RT_MODE_FP64) {
                    const double2 w0 = __ldg((const double2*)(dq + i));
                    const double2 w1 = __ldg((const double2*)(dq + i) + 1);
                    dv[0] = (T)w0.x; dv[1] = (T)w0.y; dv[2] = (T)w1.x; dv[3] = (T)w1.y;
                } else {
                    const float4 v = __ldg((const float4*)(dq + i));
                    dv[0] = (T)v.x; dv[1] = (T)v.y; dv[2] = (T)v.z; dv[3] = (T)v.w;
                }
                acc_group<MODE, SM, kGatherU, T>(sum, cmp, gv, dv);
            }
            for (; i < ell; i++) {
                T gv[1][SM], dv[1];
                load_g<T, SM>(gl + (size_t)(uint32_t)(idx0 + __ldg(Dq + i)) * SM, gv[0]);
                dv[0] = __ldg(dq + i);
                acc_group<MODE, SM, 1, T>(sum, cmp, gv, dv);
            }
            const uint32_t j = spread10((uint32_t)x) | (spread10((uint32_t)y) << 1) | (spread10((uint32_t)z) << 2);
            double* gp = a.grad + (size_t)j * SM;
#pragma unroll
            for (int k = 0; k < SM; k++) {
                const double v = (MODE == RT_MODE_FP64) ? (double)sum[k] : __dsub_rn((double)sum[k], (double)cmp[k]);
                gp[k] = __dadd_rn(gp[k], v);
            }
            n_segs += (unsigned)ell;
            n_rays += 1;
        }
    }
    flush_counters(a.st, n_rays, n_segs, 0ull, 0ull);
}

template <int MODE, int SM>
static void gather_direction(const GatherArgs& g, int q, int grid, int sgrid, cudaStream_t s)
{
    using T = typename std::conditional<MODE == RT_MODE_FP64, double, float>::type;
    k_adj_slice<T, SM><<<sgrid, 256, 0, s>>>((const T*)g.gin, q, g.nd, g.L, (T*)g.gl);
    k_adj_gather<MODE, SM><<<grid, 256, 0, s>>>(g, q);
}

template <int MODE>
static cudaError_t go_gather(const GatherArgs& g, int grid, int sgrid, cudaStream_t s)
{
    for (int q = 0; q < g.nd; q++) {
        switch (g.S) {
        case 1: gather_direction<MODE, 1>(g, q, grid, sgrid, s); break;
        case 2: gather_direction<MODE, 2>(g, q, grid, sgrid, s); break;
        case 4: gather_direction<MODE, 4>(g, q, grid, sgrid, s); break;
        case 8: gather_direction<MODE, 8>(g, q, grid, sgrid, s); break;
        default: return cudaErrorInvalidValue;
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int MODE, int SM>
static int gather_occ()
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_adj_gather<MODE, SM>, 256, 0);
    return n;
}

static int gather_occupancy(int mode, int S)
{
    if (mode == RT_MODE_FP64)
        return S == 1 ? gather_occ<RT_MODE_FP64, 1>() : S == 2 ? gather_occ<RT_MODE_FP64, 2>()
             : S == 4 ? gather_occ<RT_MODE_FP64, 4>() : gather_occ<RT_MODE_FP64, 8>();
    return S == 1 ? gather_occ<RT_MODE_F32_KAHAN, 1>() : S == 2 ? gather_occ<RT_MODE_F32_KAHAN, 2>()
         : S == 4 ? gather_occ<RT_MODE_F32_KAHAN, 4>() : gather_occ<RT_MODE_F32_KAHAN, 8>();
}

// True when the call's shape admits the leaf gather (the sources are checked
// on the device): a full cube of equal-level leaves under its O(1) index, one
// source per leaf, the default step cap and a species count gathered as one
// vector.
bool gather_applies(const rt_octree* t, const TraceArgs& a)
{
    return a.t.uniform_level >= 0 && a.n_src == t->dev.n && t->dev.step_cap >= t->default_cap &&
           (a.S == 1 || a.S == 2 || a.S == 4 || a.S == 8);
}

static size_t round256(size_t v) { return (v + 255) / 256 * 256; }

// Enqueues the source check, the tables and the gather on `s`.  The scatter
// launched after it must carry gate = &st->gather_off.
int launch_adjoint_gather(rt_octree* t, const TraceArgs& a, int mode, cudaStream_t s)
{
    const int N = 1 << a.t.uniform_level;
    const int lcap = (3 * N + 3 + 15) / 16 * 16;
    const int pcap = (N + 1 + 3) / 4 * 4;
    const size_t tsz = mode == RT_MODE_FP64 ? 8 : 4;
    const size_t q_bytes = round256((size_t)a.nd * 8);
    const size_t len_bytes = round256((size_t)a.nd * 4);
    const size_t d_bytes = round256((size_t)a.nd * lcap * 4);
    const size_t ds_bytes = round256((size_t)a.nd * lcap * tsz);
    const size_t p_bytes = round256((size_t)a.nd * 3 * pcap * 4);
    const size_t need = q_bytes + len_bytes + d_bytes + ds_bytes + p_bytes + (size_t)a.n_src * a.S * tsz;
    if (t->adj_tab_bytes < need) {
        if (t->adj_tab) {
            cudaStreamSynchronize(s);
            cudaFree(t->adj_tab);
            t->adj_tab = nullptr;
            t->adj_tab_bytes = 0;
        }
        if (cudaMalloc(&t->adj_tab, need) != cudaSuccess) {
            t->adj_tab = nullptr;
            return cuda_error("rt_trace_columns_adjoint: gather scratch allocation");
        }
        t->adj_tab_bytes = need;
    }
    char* p = (char*)t->adj_tab;
    GatherArgs g;
    memset(&g, 0, sizeof g);
    g.queue = (unsigned long long*)p;
    p += q_bytes;
    g.tab.len = (int*)p;
    p += len_bytes;
    g.tab.D = (int*)p;
    p += d_bytes;
    g.tab.ds = p;
    p += ds_bytes;
    g.tab.P = (int*)p;
    p += p_bytes;
    g.gl = p;
    g.tab.lcap = lcap;
    g.tab.pcap = pcap;
    g.gin = a.gin;
    g.grad = (double*)a.out;
    g.dirs = a.dirs;
    g.st = a.st;
    g.n = a.n_src;
    g.nd = a.nd;
    g.S = a.S;
    g.L = a.t.uniform_level;
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = sm_count_of(dev);
    if (cudaMemsetAsync(&a.st->gather_off, 0, sizeof(int), s) != cudaSuccess)
        return cuda_error("rt_trace_columns_adjoint: gather flag reset");
    const int cgrid = (int)std::min<long long>((a.n_src + 255) / 256, (long long)sms * 8);
    k_adj_check<<<std::max(cgrid, 1), 256, 0, s>>>(a.src, a.n_src, a.t.uniform_level, a.st);
    if (mode == RT_MODE_FP64)
        k_adj_table<RT_MODE_FP64><<<a.nd, 32, 0, s>>>(a.t, a.dirs, a.nd, a.src, g.tab, a.st);
    else
        k_adj_table<RT_MODE_F32_KAHAN><<<a.nd, 32, 0, s>>>(a.t, a.dirs, a.nd, a.src, g.tab, a.st);
    if (cudaGetLastError() != cudaSuccess) return cuda_error("rt_trace_columns_adjoint: table launch");
    if (cudaMemsetAsync(g.queue, 0, sizeof(unsigned long long) * a.nd, s) != cudaSuccess)
        return cuda_error("rt_trace_columns_adjoint: queue reset");
    const int fit = std::max(1, gather_occupancy(mode, a.S));
    const int sgrid = (int)std::min<long long>((a.n_src + 255) / 256, (long long)sms * 16);
    const cudaError_t e = mode == RT_MODE_FP64 ? go_gather<RT_MODE_FP64>(g, sms * fit, sgrid, s)
                                               : go_gather<RT_MODE_F32_KAHAN>(g, sms * fit, sgrid, s);
    if (e != cudaSuccess) return cuda_error("rt_trace_columns_adjoint: gather launch");
    return RT_OK;
}

}  // namespace rt
