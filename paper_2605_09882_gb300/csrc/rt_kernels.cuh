// Persistent trace kernels: a warp pops 32 * batch consecutive rays from
// a global counter (one atomic per pop, no waiting), each lane walks one ray.
// Ray r of the padded space maps direction-major: q = r / n_src_pad,
// s = r % n_src_pad, so a warp walks 32 neighbouring sources (Morton order)
// along one direction and the warps resident at any time sweep one compact
// region of the cloud, which keeps the leaves they gather in L2.
#pragma once

#include "rt_device.cuh"

// Resident 256-thread blocks per SM the register budget is sized for: both
// F32-Kahan walks run best at 64 registers (4 blocks); the FP64 walks keep
// the compiler's choice.
#ifndef RT_MIN_BLOCKS_GRID
#define RT_MIN_BLOCKS_GRID 4
#endif
#ifndef RT_MIN_BLOCKS_TREE
#define RT_MIN_BLOCKS_TREE 4
#endif
#ifndef RT_MIN_BLOCKS
#define RT_MIN_BLOCKS 1
#endif

namespace rt {

// ----------------------------------------------------------------- visitors

// A visitor sees each segment in two halves: pre(j) as soon as the leaf is
// known (the density gather is issued there) and acc(ds) once the segment
// length is known; seg(j, ds) does both at once.

// EX: the densities are known to be FP32 with exactly SM species, so the
// gather needs no per-segment dtype or count test.
// One Kahan step for two species at once, in the packed two-lane FP32
// instructions: y = n*ds + c, t = s + y, c = y - (t - s), s = t, where c is
// the compensation with its sign flipped and d2 holds ds in both lanes.  Each
// lane rounds to nearest on its own, and RN(y - u) = -RN(u - y), so the sums
// are bit for bit those of the scalar form y = n*ds - c', c' = (t - s) - y.
__device__ __forceinline__ void kahan2(float& s0, float& s1, float& c0, float& c1, float n0, float n1,
                                       unsigned long long d2)
{
    asm("{\n\t.reg .b64 s, c, x, y, t, u;\n\t"
        "mov.b64 s, {%0, %1};\n\t"
        "mov.b64 c, {%2, %3};\n\t"
        "mov.b64 x, {%4, %5};\n\t"
        "fma.rn.f32x2 y, x, %6, c;\n\t"
        "add.rn.f32x2 t, s, y;\n\t"
        "sub.rn.f32x2 u, t, s;\n\t"
        "sub.rn.f32x2 c, y, u;\n\t"
        "mov.b64 {%0, %1}, t;\n\t"
        "mov.b64 {%2, %3}, c;\n\t"
        "}"
        : "+f"(s0), "+f"(s1), "+f"(c0), "+f"(c1)
        : "f"(n0), "f"(n1), "l"(d2));
}

template <int SM, bool EX = false>
struct FwdKahan {  // FP32 columns with Kahan compensation
    float sum[SM], ncmp[SM], n[SM];  // ncmp: the compensation, negated
    const void* dens;
    int f64, S;
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int k = 0; k < SM; k++) sum[k] = ncmp[k] = 0.f;
    }
    __device__ __forceinline__ void pre(uint32_t j)
    {
        if (EX) load_dens<SM, float>(dens, 0, SM, j, n);
        else load_dens<SM, float>(dens, f64, S, j, n);
    }
    template <class F>
    __device__ __forceinline__ void acc(F dsin)
    {
        const float ds = (float)dsin;
        unsigned long long d2 = 0ull;
        if (SM > 1) asm("mov.b64 %0, {%1, %1};" : "=l"(d2) : "f"(ds));
#pragma unroll
        for (int k = 0; k + 1 < SM; k += 2) kahan2(sum[k], sum[k + 1], ncmp[k], ncmp[k + 1], n[k], n[k + 1], d2);
        if (SM & 1) {
            const float y = __fmaf_rn(n[SM - 1], ds, ncmp[SM - 1]);
            const float tt = __fadd_rn(sum[SM - 1], y);
            ncmp[SM - 1] = __fsub_rn(y, __fsub_rn(tt, sum[SM - 1]));
            sum[SM - 1] = tt;
        }
    }
    template <class F>
    __device__ __forceinline__ void seg(uint32_t j, F ds) { pre(j); acc(ds); }
};

template <int SM, bool EX = false>
struct FwdF64 {  // FP64 columns, plain summation in path order
    double col[SM], n[SM];
    const void* dens;
    int f64, S;
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int k = 0; k < SM; k++) col[k] = 0.0;
    }
    __device__ __forceinline__ void pre(uint32_t j)
    {
        if (EX) load_dens<SM, double>(dens, 0, SM, j, n);
        else load_dens<SM, double>(dens, f64, S, j, n);
    }
    template <class F>
    __device__ __forceinline__ void acc(F dsin)
    {
        const double ds = (double)dsin;
#pragma unroll
        for (int k = 0; k < SM; k++) col[k] = __dadd_rn(col[k], __dmul_rn(n[k], ds));
    }
    template <class F>
    __device__ __forceinline__ void seg(uint32_t j, F ds) { pre(j); acc(ds); }
};

struct PathHash {
    uint64_t h;
    __device__ __forceinline__ void init() { h = 0xcbf29ce484222325ull; }
    __device__ __forceinline__ void pre(uint32_t j) { h = (h ^ (uint64_t)j) * 0x100000001b3ull; }
    template <class F>
    __device__ __forceinline__ void acc(F) {}
    template <class F>
    __device__ __forceinline__ void seg(uint32_t j, F) { pre(j); }
};

template <int SM>
struct AdjScatter {  // grad[j,k] += g[k] * ds
    double g[SM];
    double* grad;
    uint32_t jj;
    int S;
    __device__ __forceinline__ void pre(uint32_t j) { jj = j; }
    template <class F>
    __device__ __forceinline__ void acc(F dsin)
    {
        const double ds = (double)dsin;
        double* p = grad + (size_t)jj * S;
#pragma unroll
        for (int k = 0; k < SM; k++)
            if (k < S) atomicAdd(p + k, __dmul_rn(g[k], ds));
    }
    template <class F>
    __device__ __forceinline__ void seg(uint32_t j, F ds) { pre(j); acc(ds); }
};

template <class T>
struct PathRecord {  // (leaf, ds) of segment k at base + 32 k, never at or past lim
    uint32_t* leaf;
    T* ds;
    long long pos, lim;
    __device__ __forceinline__ void pre(uint32_t j)
    {
        if (pos < lim) leaf[pos] = j;
    }
    template <class F>
    __device__ __forceinline__ void acc(F d)
    {
        if (pos < lim) ds[pos] = (T)d;
        pos += 32;
    }
    template <class F>
    __device__ __forceinline__ void seg(uint32_t j, F d) { pre(j); acc(d); }
};

// ------------------------------------------------------------ common loop

__device__ __forceinline__ void flush_counters(DevStats* st, unsigned long long rays,
                                               unsigned long long segs, unsigned long long efb,
                                               unsigned long long lfb)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rays += __shfl_down_sync(RT_FULL, rays, o);
        segs += __shfl_down_sync(RT_FULL, segs, o);
        efb += __shfl_down_sync(RT_FULL, efb, o);
        lfb += __shfl_down_sync(RT_FULL, lfb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (rays) atomicAdd(&st->rays, rays);
        if (segs) atomicAdd(&st->segments, segs);
        if (efb) atomicAdd(&st->exit_fb, efb);
        if (lfb) atomicAdd(&st->lookup_fb, lfb);
    }
}

// KIND 0: forward columns; 1: path fingerprints; 2: adjoint scatter;
// 3: path recording; 4: fused per-source epilogue of the columns.

// The epilogue of one ray from its combined column N: exp(-gamma a N) summed
// per source (A_V,eff), (1 - exp(-tau)) / tau with tau = coef N summed per
// source (beta), or exp(-a N) stored per ray (attenuation).
__device__ __forceinline__ void ray_epilogue(const TraceArgs& a, long long s, long long ray, double N)
{
    double* out = (double*)a.out;
    if (a.epi_kind == RT_EPI_AV_EFF) {
        atomicAdd(out + s, exp(-a.epi_gamma * a.epi_a * N));
    } else if (a.epi_kind == RT_EPI_BETA) {
        const double tau = (a.epi_coef ? __ldg(a.epi_coef + s) : a.epi_a) * N;
        atomicAdd(out + s, tau == 0.0 ? 1.0 : -expm1(-tau) / tau);
    } else {
        out[ray] = exp(-a.epi_a * N);
    }
}
// Forward columns of one ray, stored as [ray][S].
template <int MODE, bool UNIFORM, int SM, bool EX>
__device__ __forceinline__ void forward_ray(const TraceArgs& a, const DirConst* d, const double* src,
                                            long long cap, long long ray, WalkCounters& wc)
{
    if (MODE == RT_MODE_FP64) {
        FwdF64<SM, EX> v;
        v.dens = a.dens; v.f64 = a.dens_f64; v.S = a.S;
        v.init();
        const int st = walk<MODE, UNIFORM>(a.t, d, src, cap, v, wc);
        if (st != RT_OK) { report_fault(a.st, st, ray); v.init(); }
        double* o = (double*)a.out + (size_t)ray * a.S;
#pragma unroll
        for (int k = 0; k < SM; k++)
            if (k < a.S) o[k] = v.col[k];
    } else {
        FwdKahan<SM, EX> v;
        v.dens = a.dens; v.f64 = a.dens_f64; v.S = a.S;
        v.init();
        const int st = walk<MODE, UNIFORM>(a.t, d, src, cap, v, wc);
        if (st != RT_OK) { report_fault(a.st, st, ray); v.init(); }
        float* o = (float*)a.out + (size_t)ray * a.S;
        if (SM == 4 && a.S == 4) {
            *(float4*)o = make_float4(v.sum[0], v.sum[1], v.sum[2], v.sum[3]);
        } else {
#pragma unroll
            for (int k = 0; k < SM; k++)
                if (k < a.S) o[k] = v.sum[k];
        }
    }
}

template <int KIND, int MODE, bool UNIFORM, int SM>
__global__ void __launch_bounds__(256, (MODE == RT_MODE_F32_KAHAN) ? (UNIFORM ? RT_MIN_BLOCKS_GRID : RT_MIN_BLOCKS_TREE)
                                                                : RT_MIN_BLOCKS)
k_trace(const TraceArgs a)
{
    if (KIND == 2 && a.gate && *(volatile const int*)a.gate == 0) return;  // the leaf gather ran instead
    if (MODE == RT_MODE_F32_KAHAN && !UNIFORM) fill_spread_table();
    const int lane = threadIdx.x & 31;
    const unsigned long long total = (unsigned long long)(a.layout ? a.n_src : a.n_src_pad) * (unsigned long long)a.nd;
    const long long cap = a.t.step_cap;
    unsigned long long n_rays = 0, n_segs = 0, n_efb = 0, n_lfb = 0;
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
            if (a.layout == 0 && a.dgroup <= 1) {
                q = (int)(g0 / (unsigned long long)a.n_src_pad);
                s = (long long)(g0 - (unsigned long long)q * a.n_src_pad) + lane;
                if (s >= a.n_src) continue;
            } else if (a.layout == 0) {
                // direction groups: the 32-source block b takes the dgroup
                // directions of its group in consecutive 32-ray groups, so
                // the output rows they fill complete whole sectors at once
                const unsigned long long nb = (unsigned long long)a.n_src_pad >> 5, D = (unsigned)a.dgroup;
                const unsigned long long g = g0 >> 5, gg = g / (D * nb), r = g - gg * D * nb, b = r / D;
                q = (int)(gg * D + (r - b * D));
                s = (long long)(b << 5) + lane;
                if (s >= a.n_src) continue;
            } else {
                const unsigned long long r = g0 + lane;
                if (r >= total) continue;
                s = (long long)(r / (unsigned long long)a.nd);
                q = (int)(r - (unsigned long long)s * a.nd);
            }
            const DirConst* d = a.dirs + q;
            const long long ray = s * a.nd + q;
            const double* src = a.src + 3 * s;
            WalkCounters wc = {0u, 0u, 0u};
            if (KIND == 0) {
                if (!a.dens_f64 && a.S == SM) forward_ray<MODE, UNIFORM, SM, true>(a, d, src, cap, ray, wc);
                else forward_ray<MODE, UNIFORM, SM, false>(a, d, src, cap, ray, wc);
            } else if (KIND == 1) {
                PathHash v;
                v.init();
                const int st = walk<MODE, UNIFORM>(a.t, d, src, cap, v, wc);
                if (st != RT_OK) { report_fault(a.st, st, ray); v.h = 0; wc.nseg = 0; }
                if (a.nseg) a.nseg[ray] = wc.nseg;
                if (a.hash) a.hash[ray] = v.h;
            } else if (KIND == 4) {
                double N = 0.0;
                if (MODE == RT_MODE_FP64) {
                    FwdF64<SM> v;
                    v.dens = a.dens; v.f64 = a.dens_f64; v.S = a.S;
                    v.init();
                    const int st = walk<MODE, UNIFORM>(a.t, d, src, cap, v, wc);
                    if (st != RT_OK) { report_fault(a.st, st, ray); v.init(); }
#pragma unroll
                    for (int k = 0; k < SM; k++)
                        if (k < a.S) N = __dadd_rn(N, __dmul_rn(a.epi_w[k], v.col[k]));
                } else {
                    FwdKahan<SM> v;
                    v.dens = a.dens; v.f64 = a.dens_f64; v.S = a.S;
                    v.init();
                    const int st = walk<MODE, UNIFORM>(a.t, d, src, cap, v, wc);
                    if (st != RT_OK) { report_fault(a.st, st, ray); v.init(); }
#pragma unroll
                    for (int k = 0; k < SM; k++)
                        if (k < a.S) N = __dadd_rn(N, __dmul_rn(a.epi_w[k], (double)v.sum[k]));
                }
                ray_epilogue(a, s, ray, N);
            } else if (KIND == 3) {
                const long long pos = a.rec_off[g0 >> 5] + lane, lim = a.rec_off[(g0 >> 5) + 1];
                if (MODE == RT_MODE_FP64) {
                    PathRecord<double> v = {a.rec_leaf, (double*)a.rec_ds, pos, lim};
                    const int st = walk<MODE, UNIFORM>(a.t, d, src, cap, v, wc);
                    if (st != RT_OK) report_fault(a.st, st, ray);
                } else {
                    PathRecord<float> v = {a.rec_leaf, (float*)a.rec_ds, pos, lim};
                    const int st = walk<MODE, UNIFORM>(a.t, d, src, cap, v, wc);
                    if (st != RT_OK) report_fault(a.st, st, ray);
                }
            } else {
                AdjScatter<SM> v;
                v.grad = (double*)a.out;
                v.S = a.S;
#pragma unroll
                for (int k = 0; k < SM; k++) {
                    v.g[k] = 0.0;
                    if (k < a.S)
                        v.g[k] = (MODE == RT_MODE_FP64)
                                     ? __ldg((const double*)a.gin + (size_t)ray * a.S + k)
                                     : (double)__ldg((const float*)a.gin + (size_t)ray * a.S + k);
                }
                const int st = walk<MODE, UNIFORM>(a.t, d, src, cap, v, wc);
                if (st != RT_OK) report_fault(a.st, st, ray);
            }
            n_rays++;
            n_segs += wc.nseg;
            n_efb += wc.exit_fb;
            n_lfb += wc.lookup_fb;
        }
    }
    flush_counters(a.st, n_rays, n_segs, n_efb, n_lfb);
}

// Forward columns with two rays per lane (walk_grid_pair): F32-Kahan on a
// uniform cube with FP32 densities of exactly SM species.  A warp pops one
// unit, a 64-source block and one group of dgroup directions, in the order of
// k_trace's direction groups; lane i walks sources 64u + i and 64u + 32 + i
// together for each direction of the group, and one at a time where the two
// do not qualify.
#ifndef RT_MIN_BLOCKS_PAIR
#define RT_MIN_BLOCKS_PAIR 3  // 80 registers: two rays' state without spilling the loop
#endif
template <int SM>
__device__ __forceinline__ void store_cols(const TraceArgs& a, long long ray, const FwdKahan<SM, true>& v)
{
    float* o = (float*)a.out + (size_t)ray * SM;
    if (SM == 4) {
        *(float4*)o = make_float4(v.sum[0], v.sum[1], v.sum[2], v.sum[3]);
    } else {
#pragma unroll
        for (int k = 0; k < SM; k++) o[k] = v.sum[k];
    }
}

template <int SM>
__global__ void __launch_bounds__(256, RT_MIN_BLOCKS_PAIR) k_trace_pair(const TraceArgs a)
{
    const int lane = threadIdx.x & 31;
    const int D = a.dgroup > 1 ? a.dgroup : 1;
    const unsigned long long nb2 = (unsigned long long)a.n_src_pad >> 6;
    const unsigned long long units = nb2 * (unsigned long long)(a.nd / D);
    const long long cap = a.t.step_cap;
    unsigned long long n_rays = 0, n_segs = 0, n_efb = 0, n_lfb = 0;
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(&a.st->queue, 1ull);
        u = __shfl_sync(RT_FULL, u, 0);
        if (u >= units) break;
        const unsigned long long gg = u / nb2, bp = u - gg * nb2;
        const long long s0 = (long long)(bp << 6) + lane, s1 = s0 + 32;
        if (s0 >= a.n_src) continue;
        const bool two = s1 < a.n_src;
        for (int dd = 0; dd < D; dd++) {
            const int q = (int)gg * D + dd;
            const DirConst* d = a.dirs + q;
            const long long ray0 = s0 * a.nd + q, ray1 = s1 * a.nd + q;
            WalkCounters w0 = {0u, 0u, 0u}, w1 = {0u, 0u, 0u};
            FwdKahan<SM, true> v0, v1;
            v0.dens = v1.dens = a.dens;
            v0.f64 = v1.f64 = 0;
            v0.S = v1.S = SM;
            v0.init();
            v1.init();
            int st1 = RT_OK;
            const int st0 = two ? walk_grid_pair(a.t, d, a.src + 3 * s0, a.src + 3 * s1, cap, v0, v1, w0, w1, st1)
                                : kNoPair;
            if (st0 == kNoPair) {
                forward_ray<RT_MODE_F32_KAHAN, true, SM, true>(a, d, a.src + 3 * s0, cap, ray0, w0);
                if (two) forward_ray<RT_MODE_F32_KAHAN, true, SM, true>(a, d, a.src + 3 * s1, cap, ray1, w1);
            } else {
                if (st0 != RT_OK) {
                    report_fault(a.st, st0, ray0);
                    v0.init();
                }
                if (st1 != RT_OK) {
                    report_fault(a.st, st1, ray1);
                    v1.init();
                }
                store_cols<SM>(a, ray0, v0);
                store_cols<SM>(a, ray1, v1);
            }
            n_rays += two ? 2 : 1;
            n_segs += w0.nseg + w1.nseg;
            n_efb += w0.exit_fb + w1.exit_fb;
            n_lfb += w0.lookup_fb + w1.lookup_fb;
        }
    }
    flush_counters(a.st, n_rays, n_segs, n_efb, n_lfb);
}

}  // namespace rt
