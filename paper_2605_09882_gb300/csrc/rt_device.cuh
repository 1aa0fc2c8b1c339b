// Device side of the tracer: Morton helpers, the coarse-table leaf lookup and
// the ray walk (DDA + Morton lookup + slab exit, Sec. 2.2.1-2.2.2 of
// arXiv 2605.09882), in two arithmetic forms:
//   FP64   every exit time, segment and column in IEEE FP64, no contraction;
//   F32K   exit decisions made in FP32 with a certified error bound and redone
//          in FP64 only for near-ties, segment lengths from double-float
//          times, columns in FP32 with Kahan compensation.
// Both forms visit exactly the leaves of the FP64 definition.
#pragma once

#include <math.h>

#include "rt_internal.h"

namespace rt {

#define RT_FULL 0xffffffffu

// ------------------------------------------------------------ Morton codes

__device__ __forceinline__ uint64_t spread21(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint32_t compact21(uint64_t x)
{
    x &= 0x1249249249249249ull;
    x = (x | (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x | (x >> 4)) & 0x100f00f00f00f00full;
    x = (x | (x >> 8)) & 0x001f0000ff0000ffull;
    x = (x | (x >> 16)) & 0x001f00000000ffffull;
    x = (x | (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}

__device__ __forceinline__ uint64_t interleave3(uint32_t x, uint32_t y, uint32_t z)
{
    return spread21(x) | (spread21(y) << 1) | (spread21(z) << 2);
}

// 10-bit spread for the O(1) index of a uniform grid (level <= 10).
__device__ __forceinline__ uint32_t spread10(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

constexpr uint32_t kDilX = 0x09249249u;  // bits 3b of a 30-bit Morton index

// ------------------------------------------------------------- utilities

__device__ __forceinline__ float sel3(const float v[3], int b)
{
    return b == 0 ? v[0] : (b == 1 ? v[1] : v[2]);
}
__device__ __forceinline__ double sel3(const double v[3], int b)
{
    return b == 0 ? v[0] : (b == 1 ? v[1] : v[2]);
}
__device__ __forceinline__ int sel3(const int v[3], int b)
{
    return b == 0 ? v[0] : (b == 1 ? v[1] : v[2]);
}
__device__ __forceinline__ uint32_t sel3(const uint32_t v[3], int b)
{
    return b == 0 ? v[0] : (b == 1 ? v[1] : v[2]);
}

// bit of DirConst::flags telling whether |inv_a| == |inv_b| bitwise
__device__ __forceinline__ bool inv_equal(int flags, int a, int b)
{
    return (flags >> (5 + a + b)) & 1;
}

__device__ __forceinline__ void report_fault(DevStats* st, int code, long long ray)
{
    if (atomicCAS(&st->status, 0, code) == 0) st->fault_ray = ray;
}

struct WalkCounters {
    uint32_t nseg;
    uint32_t exit_fb;
    uint32_t lookup_fb;
};

// ------------------------------------------------------------ leaf lookup

// Leaf containing the depth-21 point (cx, cy, cz): coarse Morton table at
// level T, then an O(1) index for a single-level coarse cell or a binary
// search of the sorted keys inside a mixed one.  Returns -1 if no leaf
// contains the point.  key/level receive the leaf's key and level.
__device__ __forceinline__ long long lookup_leaf(const DevTree& t, uint32_t cx, uint32_t cy,
                                                 uint32_t cz, uint64_t& key, int& level)
{
    const uint64_t M = interleave3(cx, cy, cz);
    const int csh = 3 * (kDepth - t.T);
    const uint64_t cell = M >> csh;
    const uint64_t e = __ldg(t.table + cell);
    const int code = (int)(e & 63u);
    long long j = (long long)(e >> 6);
    if (code <= kDepth) {
        if (code > t.T) {
            const uint64_t local = (M & ((1ull << csh) - 1ull)) >> (3 * (kDepth - code));
            j += (long long)local;
        }
    } else if (code == kCodeHole) {
        return -1;
    } else {
        const uint64_t ncell = 1ull << (3 * t.T);
        long long hi = (cell + 1 < ncell) ? (long long)(__ldg(t.table + cell + 1) >> 6) : t.n;
        long long lo = j;  // keys[lo] == cell base <= M
        while (hi - lo > 1) {
            const long long mid = (lo + hi) >> 1;
            if (__ldg(t.keys + mid) <= M) lo = mid;
            else hi = mid;
        }
        j = lo;
    }
    key = __ldg(t.keys + j);
    level = __ldg(t.levels + j);
    if (M - key >= (1ull << (3 * (kDepth - level)))) return -1;
    return j;
}

__device__ __forceinline__ void leaf_box(uint64_t key, int level, uint32_t lo[3], uint32_t& size)
{
    lo[0] = compact21(key);
    lo[1] = compact21(key >> 1);
    lo[2] = compact21(key >> 2);
    size = 1u << (kDepth - level);
}

// ---------------------------------------------------- source on the lattice

// Source coordinate b truncated to the 2^-53 lattice: q = floor(x * 2^53).
// Returns false for a non-finite value or one outside [0, 1).
__device__ __forceinline__ bool fixed_source(double x, long long& q)
{
    if (!(x >= 0.0 && x < 1.0)) return false;
    q = __double2ll_rz(__dmul_rn(x, 0x1p53));
    return true;
}

// ======================================================== FP64 walk (MODE 0)

// Walks one ray in FP64, the operation order of the plain definition:
//   t_b = (F_b - Q_b) * inv_b, t_out = min_b t_b, E = {b : t_b == t_out},
//   ds = t_out - t_in, stepped axes move to the neighbour cell, the others
//   take floor((Q_b + t_out m_b) 2^21) clamped into the current leaf.
// V::seg(j, ds) receives every segment.
template <bool UNIFORM, class V>
__device__ __forceinline__ int walk_fp64(const DevTree& t, const DirConst& d,
                                         const double* __restrict__ src, long long cap, V& vis,
                                         WalkCounters& wc)
{
    double Q[3];
    uint32_t c[3];
#pragma unroll
    for (int b = 0; b < 3; b++) {
        long long q;
        if (!fixed_source(src[b], q)) return RT_ERR_SOURCE_OUTSIDE;
        Q[b] = __dmul_rn(__ll2double_rn(q), 0x1p-53);
        c[b] = (uint32_t)(q >> 32);
        if (c[b] >= t.ext[b]) return RT_ERR_SOURCE_OUTSIDE;
    }
    uint32_t lo[3], size;
    uint32_t ci[3], dil = 0;  // uniform grid: level-L cell index and its Morton index
    long long j;
    const int ush = kDepth - t.uniform_level;
    if (UNIFORM) {
#pragma unroll
        for (int b = 0; b < 3; b++) ci[b] = c[b] >> ush;
        dil = spread10(ci[0]) | (spread10(ci[1]) << 1) | (spread10(ci[2]) << 2);
        j = dil;
        size = 1u << ush;
    } else {
        uint64_t key;
        int level;
        j = lookup_leaf(t, c[0], c[1], c[2], key, level);
        if (j < 0) return RT_ERR_LOOKUP_MISS;
        leaf_box(key, level, lo, size);
    }
    double t_in = 0.0;
    for (long long step = 0;; ++step) {
        if (step >= cap) return RT_ERR_STEP_LIMIT;
        if (UNIFORM) {
#pragma unroll
            for (int b = 0; b < 3; b++) lo[b] = ci[b] << ush;
        }
        double tb[3];
        double t_out = __longlong_as_double(0x7ff0000000000000ll);
#pragma unroll
        for (int b = 0; b < 3; b++) {
            tb[b] = __longlong_as_double(0x7ff0000000000000ll);
            if (d.flags & (1 << b)) {
                const uint32_t F = (d.flags & (8 << b)) ? lo[b] + size : lo[b];
                const double Fd = __dmul_rn(__uint2double_rn(F), 0x1p-21);
                tb[b] = __dmul_rn(__dsub_rn(Fd, Q[b]), d.inv[b]);
                t_out = fmin(t_out, tb[b]);
            }
        }
        const double ds = __dsub_rn(t_out, t_in);
        vis.seg((uint32_t)j, ds);
        wc.nseg++;
        t_in = t_out;
        bool leaving = false;
        unsigned E = 0;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            if ((d.flags & (1 << b)) && tb[b] == t_out) {
                E |= 1u << b;
                if (d.flags & (8 << b)) {
                    if (lo[b] + size >= t.ext[b]) leaving = true;
                } else {
                    if (lo[b] == 0) leaving = true;
                }
            }
        }
        if (leaving) break;
        if (UNIFORM) {
            // a non-stepped axis stays in its slab, which the neighbour shares
#pragma unroll
            for (int b = 0; b < 3; b++) {
                if (E & (1u << b)) {
                    const uint32_t mb = kDilX << b;
                    uint32_t db = dil & mb;
                    if (d.flags & (8 << b)) { ci[b]++; db = ((db | ~mb) + (1u << b)) & mb; }
                    else { ci[b]--; db = (db - (1u << b)) & mb; }
                    dil = (dil & ~mb) | db;
                }
            }
            j = dil;
        } else {
#pragma unroll
            for (int b = 0; b < 3; b++) {
                if (E & (1u << b)) {
                    c[b] = (d.flags & (8 << b)) ? lo[b] + size : lo[b] - 1;
                } else {
                    const double P = __dadd_rn(Q[b], __dmul_rn(t_out, d.m[b]));
                    double f = floor(__dmul_rn(P, 0x1p21));
                    f = fmax(f, (double)lo[b]);
                    f = fmin(f, (double)(lo[b] + size - 1));
                    c[b] = (uint32_t)f;
                }
            }
            uint64_t key;
            int level;
            j = lookup_leaf(t, c[0], c[1], c[2], key, level);
            if (j < 0) return RT_ERR_LOOKUP_MISS;
            leaf_box(key, level, lo, size);
        }
    }
    return RT_OK;
}

// ================================================= F32-Kahan walk (MODE 1)

// Error bound of the FP32 exit time tp = fl(fl(A - ph) * ih) against the FP64
// time of the definition: |tp - t| <= |tp| * kER + |ih| * kEA (depth-21
// units).  The derivation gives 3.1 * 2^-24 and 1.01 * 2^-25; these are larger.
constexpr float kER = 0x1p-21f;
constexpr float kEA = 0x1p-23f;

// Walks one ray with FP32 exit tests.  Depth-21 units: a source coordinate is
// qi + qf 2^-32 (qi integer, qf a 32-bit fraction), a face-minus-source
// distance is D 2^-32 with D = (F - qi) 2^32 - qf an exact integer, and the
// FP64 exit time of the definition is fl(D 2^-53 inv) box lengths.
template <bool UNIFORM, class V>
__device__ __forceinline__ int walk_f32k(const DevTree& t, const DirConst& d,
                                         const double* __restrict__ src, long long cap, V& vis,
                                         WalkCounters& wc)
{
    int qi[3];
    uint32_t qf[3];
    float ph[3], pl[3];
    uint32_t c[3];
#pragma unroll
    for (int b = 0; b < 3; b++) {
        long long q;
        if (!fixed_source(src[b], q)) return RT_ERR_SOURCE_OUTSIDE;
        qi[b] = (int)(q >> 32);
        qf[b] = (uint32_t)(q & 0xffffffffll);
        if ((uint32_t)qi[b] >= t.ext[b]) return RT_ERR_SOURCE_OUTSIDE;
        // qf 2^-32 = ph + pl exactly (ph: 24 bits, pl: the remainder)
        const float fh = __uint2float_rn(qf[b]);
        const long long back = (long long)__float2ull_rz(fh);
        ph[b] = fh * 0x1p-32f;
        pl[b] = __ll2float_rn((long long)qf[b] - back) * 0x1p-32f;
        c[b] = (uint32_t)qi[b];
    }
    uint32_t lo[3], size;
    uint32_t ci[3], dil = 0;
    long long j;
    const int ush = kDepth - t.uniform_level;
    if (UNIFORM) {
#pragma unroll
        for (int b = 0; b < 3; b++) ci[b] = c[b] >> ush;
        dil = spread10(ci[0]) | (spread10(ci[1]) << 1) | (spread10(ci[2]) << 2);
        j = dil;
        size = 1u << ush;
    } else {
        uint64_t key;
        int level;
        j = lookup_leaf(t, c[0], c[1], c[2], key, level);
        if (j < 0) return RT_ERR_LOOKUP_MISS;
        leaf_box(key, level, lo, size);
    }
    float tih = 0.f, til = 0.f;  // t_in as a double-float (depth-21 units)
    for (long long step = 0;; ++step) {
        if (step >= cap) return RT_ERR_STEP_LIMIT;
        if (UNIFORM) {
#pragma unroll
            for (int b = 0; b < 3; b++) lo[b] = ci[b] << ush;
        }
        // FP32 exit time of every moving axis
        int A[3];
        float tp[3];
        int bs = 0;
        float tmin = __int_as_float(0x7f800000);
#pragma unroll
        for (int b = 0; b < 3; b++) {
            A[b] = 0;
            tp[b] = __int_as_float(0x7f800000);
            if (d.flags & (1 << b)) {
                const uint32_t F = (d.flags & (8 << b)) ? lo[b] + size : lo[b];
                A[b] = (int)F - qi[b];
                const float x = __fsub_rn(__int2float_rn(A[b]), ph[b]);
                tp[b] = __fmul_rn(x, d.ih[b]);
                if (tp[b] < tmin) { tmin = tp[b]; bs = b; }
            }
        }
        // certified decision; exact ties between axes of equal |inv| and equal
        // |D| are recognised in integers, other near-ties go to FP64
        unsigned E = 1u << bs;
        bool amb = false;
        {
            const int As = sel3(A, bs);
            const long long Ds = ((long long)As << 32) - (long long)sel3(qf, bs);
            const float errs = fabsf(tmin) * kER + fabsf(sel3(d.ih, bs)) * kEA;
#pragma unroll
            for (int b = 0; b < 3; b++) {
                if (b != bs && (d.flags & (1 << b))) {
                    const float errb = fabsf(tp[b]) * kER + fabsf(d.ih[b]) * kEA;
                    if (__fsub_rn(tp[b], tmin) <= errs + errb) {
                        const long long Db = ((long long)A[b] << 32) - (long long)qf[b];
                        if (inv_equal(d.flags, b, bs) && llabs(Db) == llabs(Ds)) E |= 1u << b;
                        else amb = true;
                    }
                }
            }
        }
        if (amb) {
            wc.exit_fb++;
            double tb[3];
            double mn = __longlong_as_double(0x7ff0000000000000ll);
#pragma unroll
            for (int b = 0; b < 3; b++) {
                tb[b] = __longlong_as_double(0x7ff0000000000000ll);
                if (d.flags & (1 << b)) {
                    const long long D = ((long long)A[b] << 32) - (long long)qf[b];
                    tb[b] = __dmul_rn(__dmul_rn(__ll2double_rn(D), 0x1p-53), d.inv[b]);
                    mn = fmin(mn, tb[b]);
                }
            }
            E = 0;
#pragma unroll
            for (int b = 0; b < 3; b++)
                if ((d.flags & (1 << b)) && tb[b] == mn) E |= 1u << b;
            bs = __ffs(E) - 1;
        }
        // segment length from double-float exit times: t = (A - ph - pl) * (ih + il)
        const int Ae = sel3(A, bs);
        const float phe = sel3(ph, bs), ple = sel3(pl, bs);
        const float ihe = sel3(d.ih, bs), ile = sel3(d.il, bs);
        const float Af = __int2float_rn(Ae);
        const float s = __fsub_rn(Af, phe);
        const float bb = __fsub_rn(s, Af);
        const float e1 = __fadd_rn(__fsub_rn(Af, __fsub_rn(s, bb)), __fsub_rn(-phe, bb));
        const float rl = __fsub_rn(e1, ple);
        const float th = __fmul_rn(s, ihe);
        const float tl = __fadd_rn(__fmaf_rn(s, ihe, -th), __fmaf_rn(s, ile, __fmul_rn(rl, ihe)));
        const float ds = __fmul_rn(__fadd_rn(__fsub_rn(th, tih), __fsub_rn(tl, til)), 0x1p-21f);
        tih = th;
        til = tl;
        vis.seg((uint32_t)j, ds);
        wc.nseg++;
        // step the exit axes; leave at the domain edge
        bool leaving = false;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            if (E & (1u << b)) {
                if (d.flags & (8 << b)) {
                    if (lo[b] + size >= t.ext[b]) leaving = true;
                } else {
                    if (lo[b] == 0) leaving = true;
                }
            }
        }
        if (leaving) break;
        if (UNIFORM) {
#pragma unroll
            for (int b = 0; b < 3; b++) {
                if (E & (1u << b)) {
                    const uint32_t mb = kDilX << b;
                    uint32_t db = dil & mb;
                    if (d.flags & (8 << b)) { ci[b]++; db = ((db | ~mb) + (1u << b)) & mb; }
                    else { ci[b]--; db = (db - (1u << b)) & mb; }
                    dil = (dil & ~mb) | db;
                }
            }
            j = dil;
            continue;
        }
        // general octree: position of the non-stepped axes at t_out as a
        // certified integer interval [clo, chi] (depth-21 cells)
        uint32_t chi[3];
        bool wide = false;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const uint32_t lob = lo[b], hib = lo[b] + size - 1;
            if (E & (1u << b)) {
                c[b] = (d.flags & (8 << b)) ? lo[b] + size : lo[b] - 1;
                chi[b] = c[b];
            } else if (!(d.flags & (1 << b))) {
                c[b] = min(max((uint32_t)qi[b], lob), hib);
                chi[b] = c[b];
            } else {
                const float mw = __fmul_rn(th, d.m32[b]);
                const float w = __fadd_rn(mw, ph[b]);
                const float del = (fabsf(mw) + fabsf(w)) * 0x1p-21f +
                                  fabsf(d.m32[b]) * fabsf(ihe) * 0x1p-22f + 0x1p-22f;
                const long long l0 = (long long)qi[b] + (long long)floorf(__fsub_rd(w, del));
                const long long l1 = (long long)qi[b] + (long long)floorf(__fadd_ru(w, del));
                c[b] = (uint32_t)min(max(l0, (long long)lob), (long long)hib);
                chi[b] = (uint32_t)min(max(l1, (long long)lob), (long long)hib);
                if (chi[b] != c[b]) wide = true;
            }
        }
        uint64_t key;
        int level;
        j = lookup_leaf(t, c[0], c[1], c[2], key, level);
        if (j >= 0 && wide) {
            uint32_t nlo[3], nsize;
            leaf_box(key, level, nlo, nsize);
#pragma unroll
            for (int b = 0; b < 3; b++)
                if (chi[b] >= nlo[b] + nsize) j = -2;  // the interval crosses a leaf face
        }
        if (j == -2 || (j < 0 && wide)) {
            // FP64 position of the definition: P = Q + t_out m, floor(P 2^21)
            wc.lookup_fb++;
            const long long De = ((long long)Ae << 32) - (long long)sel3(qf, bs);
            const double te = __dmul_rn(__dmul_rn(__ll2double_rn(De), 0x1p-53), sel3(d.inv, bs));
#pragma unroll
            for (int b = 0; b < 3; b++) {
                if (!(E & (1u << b)) && (d.flags & (1 << b))) {
                    const long long qb = ((long long)qi[b] << 32) | (long long)qf[b];
                    const double Qb = __dmul_rn(__ll2double_rn(qb), 0x1p-53);
                    const double P = __dadd_rn(Qb, __dmul_rn(te, d.m[b]));
                    double f = floor(__dmul_rn(P, 0x1p21));
                    f = fmax(f, (double)lo[b]);
                    f = fmin(f, (double)(lo[b] + size - 1));
                    c[b] = (uint32_t)f;
                }
            }
            j = lookup_leaf(t, c[0], c[1], c[2], key, level);
        }
        if (j < 0) return RT_ERR_LOOKUP_MISS;
        leaf_box(key, level, lo, size);
    }
    return RT_OK;
}

// ------------------------------------ F32-Kahan walk on a uniform grid

// Double-float exit time t = (A - ph - pl) * (ih + il) (depth-21 units) of one
// axis: th = fl(fl(A - ph) * ih) is the FP32 time the certified bound is stated
// for, th + tl carries about 44 bits.
__device__ __forceinline__ void exit_time(float Af, float ph, float pl, float ih, float il, float& th,
                                          float& tl)
{
    const float s = __fsub_rn(Af, ph);
    const float bb = __fsub_rn(s, Af);
    const float e1 = __fadd_rn(__fsub_rn(Af, __fsub_rn(s, bb)), __fsub_rn(-ph, bb));
    const float rl = __fsub_rn(e1, pl);
    th = __fmul_rn(s, ih);
    tl = __fadd_rn(__fmaf_rn(s, ih, -th), __fmaf_rn(s, il, __fmul_rn(rl, ih)));
}

// Exit set when the two smallest FP32 times are within the certified margin:
// axes that tie exactly (bitwise-equal |inv| and equal |D|) are recognised in
// integers, anything else is decided by the FP64 times of the definition.
template <int VM>
__device__ __forceinline__ unsigned resolve_exit(const float th[3], const float Af[3], const uint32_t qf[3],
                                                 const float ih[3], int flags,
                                                 const DirConst* __restrict__ dp, int bs, WalkCounters& wc)
{
    unsigned E = 1u << bs;
    bool amb = false;
    const float tmin = sel3(th, bs);
    const long long Ds = ((long long)__float2int_rn(sel3(Af, bs)) << 32) - (long long)sel3(qf, bs);
    const float errs = fabsf(tmin) * kER + fabsf(sel3(ih, bs)) * kEA;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        if ((VM & (1 << b)) && b != bs) {
            const float errb = fabsf(th[b]) * kER + fabsf(ih[b]) * kEA;
            if (__fsub_rn(th[b], tmin) <= errs + errb) {
                const long long Db = ((long long)__float2int_rn(Af[b]) << 32) - (long long)qf[b];
                if (inv_equal(flags, b, bs) && llabs(Db) == llabs(Ds)) E |= 1u << b;
                else amb = true;
            }
        }
    }
    if (amb) {
        wc.exit_fb++;
        double tb[3];
        double mn = __longlong_as_double(0x7ff0000000000000ll);
#pragma unroll
        for (int b = 0; b < 3; b++) {
            tb[b] = mn;
            if (VM & (1 << b)) {
                const long long D = ((long long)__float2int_rn(Af[b]) << 32) - (long long)qf[b];
                tb[b] = __dmul_rn(__dmul_rn(__ll2double_rn(D), 0x1p-53), __ldg(&dp->inv[b]));
            }
        }
#pragma unroll
        for (int b = 0; b < 3; b++) mn = fmin(mn, tb[b]);
        E = 0;
#pragma unroll
        for (int b = 0; b < 3; b++)
            if ((VM & (1 << b)) && tb[b] == mn) E |= 1u << b;
    }
    return E;
}

// Walk of one ray through a full cube of equal-level leaves (level L <= 10),
// F32-Kahan arithmetic, for a direction whose moving axes are the bits of VM.
// The leaf index is the level-L Morton index, kept per axis in dilated form;
// the per-axis far-face distance A (exact integer and exact float) and the
// double-float exit time change only on the axes that step.
template <int VM, class V>
__device__ __forceinline__ int walk_f32k_grid(const DevTree& t, const DirConst* __restrict__ dp,
                                              const double* __restrict__ src, long long cap, V& vis,
                                              WalkCounters& wc)
{
    constexpr int nvm = ((VM >> 0) & 1) + ((VM >> 1) & 1) + ((VM >> 2) & 1);
    const int sh = kDepth - t.uniform_level;
    const int N1 = (1 << t.uniform_level) - 1;
    const int size = 1 << sh;
    const int flags = __ldg(&dp->flags);
    float ih[3], il[3];
    uint32_t qf[3];
    float ph[3], pl[3];
    int c[3];
    float Af[3], th[3], tl[3];
    uint32_t dl[3];
    float cE = 0.f;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        long long q;
        if (!fixed_source(src[b], q)) return RT_ERR_SOURCE_OUTSIDE;
        const int qi = (int)(q >> 32);
        qf[b] = (uint32_t)(q & 0xffffffffll);
        if ((uint32_t)qi >= t.ext[b]) return RT_ERR_SOURCE_OUTSIDE;
        const float fh = __uint2float_rn(qf[b]);
        const long long back = (long long)__float2ull_rz(fh);
        ph[b] = fh * 0x1p-32f;
        pl[b] = __ll2float_rn((long long)qf[b] - back) * 0x1p-32f;
        c[b] = qi >> sh;
        dl[b] = spread10((uint32_t)c[b]) << b;
        Af[b] = 0.f;
        th[b] = tl[b] = ih[b] = il[b] = 0.f;
        if (VM & (1 << b)) {
            ih[b] = __ldg(&dp->ih[b]);
            il[b] = __ldg(&dp->il[b]);
            const int pos = (flags >> (3 + b)) & 1;
            Af[b] = __int2float_rn(((c[b] + pos) << sh) - qi);
            exit_time(Af[b], ph[b], pl[b], ih[b], il[b], th[b], tl[b]);
            cE = fmaxf(cE, fabsf(ih[b]) * kEA);
        }
    }
    uint32_t j = dl[0] | dl[1] | dl[2];
    float tih = 0.f, til = 0.f;
    for (long long step = 0;; ++step) {
        if (step >= cap) return RT_ERR_STEP_LIMIT;
        vis.pre(j);
        float tmin = __int_as_float(0x7f800000), t2 = tmin;
        int bs = 0;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            if (VM & (1 << b)) {
                if (th[b] < tmin) { t2 = tmin; tmin = th[b]; bs = b; }
                else t2 = fminf(t2, th[b]);
            }
        }
        unsigned E = 1u << bs;
        if (nvm > 1 && !(__fsub_rn(t2, tmin) > (fabsf(t2) + fabsf(tmin)) * kER + 2.f * cE)) {
            E = resolve_exit<VM>(th, Af, qf, ih, flags, dp, bs, wc);
            bs = __ffs(E) - 1;
        }
        const float ths = sel3(th, bs), tls = sel3(tl, bs);
        const float ds = __fmul_rn(__fadd_rn(__fsub_rn(ths, tih), __fsub_rn(tls, til)), 0x1p-21f);
        tih = ths;
        til = tls;
        vis.acc(ds);
        wc.nseg++;
        bool leaving = false;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            if ((VM & (1 << b)) && (E & (1u << b))) {
                const int pos = (flags >> (3 + b)) & 1;
                if (c[b] == (pos ? N1 : 0)) leaving = true;
                c[b] += pos ? 1 : -1;
                Af[b] = __fadd_rn(Af[b], pos ? (float)size : -(float)size);
                exit_time(Af[b], ph[b], pl[b], ih[b], il[b], th[b], tl[b]);
                const uint32_t mb = kDilX << b;
                dl[b] = pos ? (((dl[b] | ~mb) + (1u << b)) & mb) : ((dl[b] - (1u << b)) & mb);
            }
        }
        if (leaving) break;
        j = dl[0] | dl[1] | dl[2];
    }
    return RT_OK;
}

// Walk of one ray (direction *dp, in global memory) in either arithmetic form.
template <int MODE, bool UNIFORM, class V>
__device__ __forceinline__ int walk(const DevTree& t, const DirConst* __restrict__ dp,
                                    const double* __restrict__ src, long long cap, V& vis,
                                    WalkCounters& wc)
{
    if (MODE == RT_MODE_FP64) {
        const DirConst d = *dp;
        return walk_fp64<UNIFORM>(t, d, src, cap, vis, wc);
    }
    if (UNIFORM) {
        switch (__ldg(&dp->flags) & 7) {
        case 1: return walk_f32k_grid<1>(t, dp, src, cap, vis, wc);
        case 2: return walk_f32k_grid<2>(t, dp, src, cap, vis, wc);
        case 3: return walk_f32k_grid<3>(t, dp, src, cap, vis, wc);
        case 4: return walk_f32k_grid<4>(t, dp, src, cap, vis, wc);
        case 5: return walk_f32k_grid<5>(t, dp, src, cap, vis, wc);
        case 6: return walk_f32k_grid<6>(t, dp, src, cap, vis, wc);
        default: return walk_f32k_grid<7>(t, dp, src, cap, vis, wc);
        }
    }
    const DirConst d = *dp;
    return walk_f32k<UNIFORM>(t, d, src, cap, vis, wc);
}

// ------------------------------------------------------------- densities

// Loads S densities of leaf j into n[0..SM) (zeros past S), widening or
// narrowing to T.
template <int SM, class T>
__device__ __forceinline__ void load_dens(const void* __restrict__ dens, int f64, int S, uint32_t j,
                                          T n[SM])
{
    if (!f64) {
        const float* p = (const float*)dens;
        if (S == SM) {
            if (SM == 1) {
                n[0] = (T)__ldg(p + j);
            } else if (SM == 2) {
                const float2 v = __ldg((const float2*)p + j);
                n[0] = (T)v.x; n[1] = (T)v.y;
            } else {
#pragma unroll
                for (int h = 0; h < SM / 4; h++) {
                    const float4 v = __ldg((const float4*)p + (size_t)j * (SM / 4) + h);
                    n[4 * h] = (T)v.x; n[4 * h + 1] = (T)v.y;
                    n[4 * h + 2] = (T)v.z; n[4 * h + 3] = (T)v.w;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < SM; k++) n[k] = (k < S) ? (T)__ldg(p + (size_t)j * S + k) : (T)0;
        }
    } else {
        const double* p = (const double*)dens;
        if (S == SM && SM >= 2) {
#pragma unroll
            for (int h = 0; h < SM / 2; h++) {
                const double2 v = __ldg((const double2*)p + (size_t)j * (SM / 2) + h);
                n[2 * h] = (T)v.x; n[2 * h + 1] = (T)v.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < SM; k++) n[k] = (k < S) ? (T)__ldg(p + (size_t)j * S + k) : (T)0;
        }
    }
}

}  // namespace rt
