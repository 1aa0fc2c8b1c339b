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

// spread10 of every 10-bit value, per block in shared memory, for the leaf
// lookup of the F32-Kahan tree walk (one load per axis instead of the nine
// instructions of the shifts and masks).  Every kernel that runs that walk
// fills it first; the lookup masks what it reads to the table's range, so an
// unfilled table could give a wrong leaf but no out-of-range access.
__shared__ uint32_t s_spread10[1024];

__device__ __forceinline__ void fill_spread_table()
{
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) s_spread10[i] = spread10((uint32_t)i);
    __syncthreads();
}

// The bits of a 30-bit Morton index that belong to the two axes other than b.
__device__ __forceinline__ constexpr uint32_t dil_holes(int b) { return ~(kDilX << b) & 0x3fffffffu; }

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
//
// Taken from the bits of x with integer operations (the FP64 pipe is narrow
// and every ray needs this for each axis): x = m 2^(e - 1075) for a biased
// exponent e >= 1 (m with its implicit bit), so x 2^53 = m 2^(e - 1022) and,
// as x < 1 means e <= 1022, q = m >> (1022 - e).  A subnormal x gives q = 0.
// Equal to trunc(x * 2^53) in FP64, where the product is exact.
__device__ __forceinline__ bool fixed_source(double x, long long& q)
{
    const long long bits = __double_as_longlong(x);
    // [0, 1): sign clear and below the bits of 1.0 (NaN and infinity are
    // above); -0.0 is the one negative-signed value inside
    if (bits < 0 || bits >= 0x3FF0000000000000ll) {
        q = 0;
        return bits == (long long)0x8000000000000000ull;
    }
    const int e = (int)(bits >> 52);
    const long long m = (bits & 0x000FFFFFFFFFFFFFll) | ((long long)(e != 0) << 52);
    const int sh = 1022 - e;
    q = sh >= 53 ? 0ll : (m >> sh);
    return true;
}

// ------------------------------------------------ resumable walks (chunks)

// Walk state at the top of the step loop: the leaf about to be entered, its
// box and the time the ray entered it.  It determines the rest of the walk, so
// a walk stopped there and resumed later visits exactly the leaves and
// segment lengths of an uninterrupted one.  status: 0 not started, 1 stopped
// at a leaf outside the chunk being traced, 2 finished.
struct RayState {
    uint32_t j;          // leaf about to be entered
    uint32_t lo[3];      // its lower corner (depth-21 lattice)
    uint32_t nseg;       // segments so far
    uint8_t level;       // its level
    uint8_t status;
    uint16_t pad;
    double t;            // FP64 walk: entry time t_in
    float th, tl;        // F32-Kahan walk: entry time (double-float, depth-21 units)
    uint64_t hash;       // path fingerprint so far (kept by the caller)
};

constexpr int kSuspended = -1;  // internal: the walk stopped at a leaf outside the chunk

// Plain walks: no state, never stop early (s is never read).
struct NoResume {
    static constexpr bool enabled = false;
    RayState* s;
    __device__ __forceinline__ bool inside(long long) const { return true; }
};

// Walks that trace only the leaves of one contiguous leaf range [j0, j1) (a
// Morton-range chunk of the linear octree) and stop, saving their state, when
// the next leaf lies outside it.
struct ChunkResume {
    static constexpr bool enabled = true;
    RayState* s;
    long long j0, j1;
    __device__ __forceinline__ bool inside(long long j) const { return j >= j0 && j < j1; }
};

// ======================================================== FP64 walk (MODE 0)

// Walks one ray in FP64, the operation order of the plain definition:
//   t_b = (F_b - Q_b) * inv_b, t_out = min_b t_b, E = {b : t_b == t_out},
//   ds = t_out - t_in, stepped axes move to the neighbour cell, the others
//   take floor((Q_b + t_out m_b) 2^21) clamped into the current leaf (formed
//   only when the neighbour is finer than the current leaf; see below).
// V::seg(j, ds) receives every segment.
template <bool UNIFORM, class V, class R = NoResume>
__device__ __forceinline__ int walk_fp64(const DevTree& t, const DirConst& d,
                                         const double* __restrict__ src, long long cap, V& vis,
                                         WalkCounters& wc, R* rs = nullptr)
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
    } else if (R::enabled && rs->s->status == 1) {
        j = rs->s->j;
#pragma unroll
        for (int b = 0; b < 3; b++) lo[b] = rs->s->lo[b];
        size = 1u << (kDepth - rs->s->level);
    } else {
        uint64_t key;
        int level;
        j = lookup_leaf(t, c[0], c[1], c[2], key, level);
        if (j < 0) return RT_ERR_LOOKUP_MISS;
        leaf_box(key, level, lo, size);
    }
    double t_in = (R::enabled && rs->s->status == 1) ? rs->s->t : 0.0;
    for (long long step = R::enabled ? (long long)rs->s->nseg : 0;; ++step) {
        if (step >= cap) return RT_ERR_STEP_LIMIT;
        if (R::enabled && !rs->inside(j)) {
            rs->s->j = (uint32_t)j;
#pragma unroll
            for (int b = 0; b < 3; b++) rs->s->lo[b] = lo[b];
            rs->s->level = (uint8_t)(kDepth - (31 - __clz(size)));
            rs->s->t = t_in;
            rs->s->nseg = (uint32_t)step;
            return kSuspended;
        }
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
            // The exit axes step; the others first take the leaf's lower
            // corner.  Unless the leaf found there is finer than the current
            // one it holds the whole face-adjacent cell of the current size
            // (octree cells are aligned), hence the exit point: only a finer
            // neighbour needs the position of the definition.
#pragma unroll
            for (int b = 0; b < 3; b++)
                c[b] = (E & (1u << b)) ? ((d.flags & (8 << b)) ? lo[b] + size : lo[b] - 1) : lo[b];
            uint64_t key;
            int level;
            j = lookup_leaf(t, c[0], c[1], c[2], key, level);
            if (E != 7u && j >= 0 && (1u << (kDepth - level)) < size) {
#pragma unroll
                for (int b = 0; b < 3; b++) {
                    if (!(E & (1u << b))) {
                        const double P = __dadd_rn(Q[b], __dmul_rn(t_out, d.m[b]));
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
    }
    return RT_OK;
}

// FP64 walk on a full cube of equal-level leaves, moving axes VM (compile
// time), in the mirrored frame of the F32-Kahan grid walk (a moving axis with
// m_b < 0 is reflected, so every moving axis advances by one cell).  The exit
// time of the definition, fl(fl(F_b - Q_b) inv_b), is formed as
// fl(D_b (|inv_b| 2^-53)) with D_b = |F_b - Q_b| 2^53 an exact integer held
// in a double: F_b - Q_b is exact on the 2^-53 lattice and the scaling by
// 2^-53 is exact, so both round the same real product and give the same
// double (up to the sign of a zero time).  D_b grows by the leaf size on each
// step of its axis.  Exit times are non-negative, so their minimum and ties
// are taken on the bit patterns as integers; ds = t_out - t_in is in FP64.
// Only the axes that step recompute their time (one FP64 add and multiply
// each), one axis at a time.
//
// LOCK (VM 3 or 7): bitwise-equal |inv_x| = |inv_y| and equal D_x = D_y at the
// source, so x and y have the same exit time for the whole walk and y steps
// whenever x does, without a time of its own.
template <int VM, bool LOCK, class V>
__device__ __forceinline__ int walk_fp64_grid(const DevTree& t, const DirConst* __restrict__ dp,
                                              const double* __restrict__ src, long long cap, V& vis,
                                              WalkCounters& wc)
{
    constexpr int VT = LOCK ? (VM & 5) : VM;  // the axes with a time of their own
    const int sh = kDepth - t.uniform_level;
    const int N1 = (1 << t.uniform_level) - 1;
    const double dsz = (double)(1ll << (sh + 32));  // leaf size on the 2^-53 lattice, exact
    const int flags = __ldg(&dp->flags);
    const long long kInf = 0x7ff0000000000000ll;
    double D[3], inv53[3];
    long long tb[3];  // exit times as bit patterns
    int cm[3];        // mirrored cell coordinate
    uint32_t dl[3], xm = 0u;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        long long q;
        if (!fixed_source(src[b], q)) return RT_ERR_SOURCE_OUTSIDE;
        const uint32_t cb = (uint32_t)(q >> 32);
        if (cb >= t.ext[b]) return RT_ERR_SOURCE_OUTSIDE;
        const int c = (int)(cb >> sh);
        const bool neg = (VM & (1 << b)) && !((flags >> (3 + b)) & 1);
        cm[b] = neg ? (c ^ N1) : c;
        dl[b] = (spread10((uint32_t)cm[b]) << b) | dil_holes(b);
        if (neg) xm |= spread10((uint32_t)N1) << b;
        D[b] = inv53[b] = 0.0;
        tb[b] = kInf;
        if (VT & (1 << b)) {
            const long long F53 = (long long)(neg ? c : c + 1) << (sh + 32);
            D[b] = __ll2double_rn(neg ? q - F53 : F53 - q);
            inv53[b] = __dmul_rn(fabs(__ldg(&dp->inv[b])), 0x1p-53);
            tb[b] = __double_as_longlong(__dmul_rn(D[b], inv53[b]));
        }
    }
    uint32_t j = (dl[0] & dl[1] & dl[2]) ^ xm;
    double t_in = 0.0;
    const uint32_t lim = wc.nseg + (uint32_t)min(cap, (long long)0x7fffffff);  // cap >= 1
    for (;;) {
        vis.pre(j);
        long long to = kInf;
#pragma unroll
        for (int b = 0; b < 3; b++)
            if (VT & (1 << b)) to = min(to, tb[b]);
        const double t_out = __longlong_as_double(to);
        vis.acc(__dsub_rn(t_out, t_in));
        wc.nseg++;
        t_in = t_out;
        unsigned E = 0u;
#pragma unroll
        for (int b = 0; b < 3; b++)
            if ((VT & (1 << b)) && tb[b] == to) E |= 1u << b;
        bool leaving = false;
        do {
            const int s = __ffs(E) - 1;
            E &= E - 1u;
            const double Ds = __dadd_rn(sel3(D, s), dsz);
            const long long ts = __double_as_longlong(__dmul_rn(Ds, sel3(inv53, s)));
#pragma unroll
            for (int b = 0; b < 3; b++) {
                if ((VM & (1 << b)) && (b == s || (LOCK && b == 1 && s == 0))) {
                    leaving |= cm[b] == N1;
                    cm[b]++;
                    dl[b] = (dl[b] + (1u << b)) | dil_holes(b);
                    if (VT & (1 << b)) {
                        D[b] = Ds;
                        tb[b] = ts;
                    }
                }
            }
        } while (E);
        if (leaving || wc.nseg >= lim) {  // the cap ends a ray that still goes on
            if (leaving) break;
            return RT_ERR_STEP_LIMIT;
        }
        j = (dl[0] & dl[1] & dl[2]) ^ xm;
    }
    return RT_OK;
}

// True when the x and y exit times of an FP64 grid walk stay equal: both axes
// move, |inv_x| = |inv_y| bitwise, and the source's mirrored distances to its
// leaf's far x and y faces are equal on the 2^-53 lattice.
__device__ __forceinline__ bool xy_locked_fp64(const DevTree& t, int flags, const double* __restrict__ src)
{
    if ((flags & 3) != 3 || !inv_equal(flags, 0, 1)) return false;
    long long q[2];
    if (!fixed_source(src[0], q[0]) || !fixed_source(src[1], q[1])) return false;
    const int sh = kDepth - t.uniform_level;
    long long Dm[2];
#pragma unroll
    for (int b = 0; b < 2; b++) {
        const long long c = q[b] >> (sh + 32);
        Dm[b] = ((flags >> (3 + b)) & 1) ? ((c + 1) << (sh + 32)) - q[b] : q[b] - (c << (sh + 32));
    }
    return Dm[0] == Dm[1];
}

// ================================================= F32-Kahan walk (MODE 1)

// Error bound of the FP32 exit time tp = fl(fl(A - ph) * ih) against the FP64
// time of the definition: |tp - t| <= |tp| * kER + |ih| * kEA (depth-21
// units).  The derivation gives 3.1 * 2^-24 and 1.01 * 2^-25; these are larger.
constexpr float kER = 0x1p-21f;
constexpr float kEA = 0x1p-23f;

// In depth-21 units a source coordinate is qi + qf 2^-32 (qi integer, qf a
// 32-bit fraction) and a face-minus-source distance is D 2^-32 with
// D = (F - qi) 2^32 - qf an exact integer; the FP64 exit time of the
// definition is fl(D 2^-53 inv) box lengths.  QZ marks a source whose
// fractions are all zero (every leaf centre down to level 20): then ph = pl =
// 0 and A = F - qi is the whole distance.

// (h1 - h0) + (l1 - l0) for the double-float times h + l: both differences
// in one packed two-lane FP32 subtraction (each lane rounds to nearest, as
// the two scalar subtractions would).
__device__ __forceinline__ float diff_sum(float h1, float l1, float h0, float l0)
{
    float dh, dl;
    asm("{\n\t.reg .b64 a, b;\n\t"
        "mov.b64 a, {%2, %3};\n\t"
        "mov.b64 b, {%4, %5};\n\t"
        "sub.rn.f32x2 a, a, b;\n\t"
        "mov.b64 {%0, %1}, a;\n\t"
        "}"
        : "=f"(dh), "=f"(dl)
        : "f"(h1), "f"(l1), "f"(h0), "f"(l0));
    return __fadd_rn(dh, dl);
}

// ------------------------------------ F32-Kahan walk on a uniform grid

// Double-float exit time t = (A - ph - pl) * (ih + il) (depth-21 units) of one
// axis: th = fl(fl(A - ph) * ih) is the FP32 time the certified bound is stated
// for, th + tl carries about 44 bits.
template <bool QZ>
__device__ __forceinline__ void exit_time(float Af, float ph, float pl, float ih, float il, float& th,
                                          float& tl)
{
    if (QZ) {
        th = __fmul_rn(Af, ih);
        tl = __fmaf_rn(Af, il, __fmaf_rn(Af, ih, -th));
        return;
    }
    const float s = __fsub_rn(Af, ph);
    const float bb = __fsub_rn(s, Af);
    const float e1 = __fadd_rn(__fsub_rn(Af, __fsub_rn(s, bb)), __fsub_rn(-ph, bb));
    const float rl = __fsub_rn(e1, pl);
    th = __fmul_rn(s, ih);
    tl = __fadd_rn(__fmaf_rn(s, ih, -th), __fmaf_rn(s, il, __fmul_rn(rl, ih)));
}

// Integer value of an integer-valued float |v| < 2^22 without a conversion
// instruction.
__device__ __forceinline__ int small_float_to_int(float v)
{
    return __float_as_int(__fadd_rn(v, 12582912.0f)) - 0x4B400000;
}

// The smallest, second and third smallest FP32 exit times over the moving
// axes VM, with the axes of the first two (ties: lower axis first).
template <int VM>
__device__ __forceinline__ void order_exits(const float th[3], float& t1, int& i1, float& t2, int& i2,
                                            float& t3)
{
    const float inf = __int_as_float(0x7f800000);
    if (VM == 7) {
        const bool s = th[1] < th[0];
        const float lo = s ? th[1] : th[0], hi = s ? th[0] : th[1];
        const int il = s ? 1 : 0, ih = s ? 0 : 1;
        if (th[2] < lo) { t1 = th[2]; i1 = 2; t2 = lo; i2 = il; t3 = hi; }
        else if (th[2] < hi) { t1 = lo; i1 = il; t2 = th[2]; i2 = 2; t3 = hi; }
        else { t1 = lo; i1 = il; t2 = hi; i2 = ih; t3 = th[2]; }
    } else if (VM == 3 || VM == 5 || VM == 6) {
        const int a = (VM == 6) ? 1 : 0, b = (VM == 3) ? 1 : 2;
        const bool s = th[b] < th[a];
        t1 = s ? th[b] : th[a]; i1 = s ? b : a;
        t2 = s ? th[a] : th[b]; i2 = s ? a : b;
        t3 = inf;
    } else {
        const int a = (VM == 1) ? 0 : (VM == 2 ? 1 : 2);
        t1 = th[a]; i1 = a; t2 = t3 = inf; i2 = a;
    }
}

// D of axis b from its far-face distance A: (A 2^32) - qf.  MIR marks the
// mirrored frame of the uniform-grid walk, where a negative axis carries
// A' = -A, so that D' = -D = (A' 2^32) + qf.
template <bool MIR>
__device__ __forceinline__ long long face_distance(float A, uint32_t qf, int flags, int b)
{
    const long long hi = (long long)small_float_to_int(A) << 32;
    if (MIR && !((flags >> (3 + b)) & 1)) return hi + (long long)qf;
    return hi - (long long)qf;
}

// Exit set when the two smallest FP32 times are within the certified margin:
// axes that tie exactly (bitwise-equal |inv| and equal |D|) are recognised in
// integers, anything else is decided by the FP64 times of the definition
// (|D| 2^-53 |inv|, the same value for either sign convention).
template <int VM, bool MIR>
__device__ __forceinline__ unsigned resolve_exit(const float th[3], const float Af[3], const uint32_t qf[3],
                                                 const float ih[3], int flags,
                                                 const DirConst* __restrict__ dp, int bs, WalkCounters& wc)
{
    unsigned E = 1u << bs;
    bool amb = false;
    const float tmin = sel3(th, bs);
    const long long Ds = face_distance<MIR>(sel3(Af, bs), sel3(qf, bs), flags, bs);
    const float errs = fabsf(tmin) * kER + fabsf(sel3(ih, bs)) * kEA;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        if ((VM & (1 << b)) && b != bs) {
            const float errb = fabsf(th[b]) * kER + fabsf(ih[b]) * kEA;
            if (__fsub_rn(th[b], tmin) <= errs + errb) {
                const long long Db = face_distance<MIR>(Af[b], qf[b], flags, b);
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
                const long long D = face_distance<MIR>(Af[b], qf[b], flags, b);
                const double inv = __ldg(&dp->inv[b]);
                tb[b] = __dmul_rn(__dmul_rn(__ll2double_rn(D), 0x1p-53), MIR ? fabs(inv) : inv);
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

// Exit set of one step: the smallest exit time decides unless the second is
// within the certified margin; then an exact tie of two equal-|inv| axes of a
// QZ source is recognised from equal |A|, and anything else is resolved.
template <int VM, bool QZ, bool MIR>
__device__ __forceinline__ unsigned exit_set(const float th[3], const float Af[3], const uint32_t qf[3],
                                             const float ih[3], int flags, float cE,
                                             const DirConst* __restrict__ dp, int& bs, WalkCounters& wc)
{
    constexpr int nvm = ((VM >> 0) & 1) + ((VM >> 1) & 1) + ((VM >> 2) & 1);
    float t1, t2, t3;
    int i1, i2;
    order_exits<VM>(th, t1, i1, t2, i2, t3);
    bs = i1;
    unsigned E = 1u << i1;
    if (nvm > 1 && !(__fsub_rn(t2, t1) > (fabsf(t2) + fabsf(t1)) * kER + 2.f * cE)) {
        bool done = false;
        if (QZ && t2 == t1 && inv_equal(flags, i1, i2) && fabsf(sel3(Af, i1)) == fabsf(sel3(Af, i2)) &&
            (nvm < 3 || __fsub_rn(t3, t1) > (fabsf(t3) + fabsf(t1)) * kER + 2.f * cE)) {
            E |= 1u << i2;
            bs = min(i1, i2);
            done = true;
        }
        if (!done) {
            E = resolve_exit<VM, MIR>(th, Af, qf, ih, flags, dp, i1, wc);
            bs = __ffs(E) - 1;
        }
    }
    return E;
}

// Source coordinates on the 2^-53 lattice: qi + qf 2^-32 (depth-21 units) and
// the exact split qf 2^-32 = ph + pl.
__device__ __forceinline__ int source_fixed(const double* __restrict__ src, const DevTree& t, int qi[3],
                                            uint32_t qf[3], float ph[3], float pl[3])
{
#pragma unroll
    for (int b = 0; b < 3; b++) {
        long long q;
        if (!fixed_source(src[b], q)) return RT_ERR_SOURCE_OUTSIDE;
        qi[b] = (int)(q >> 32);
        qf[b] = (uint32_t)(q & 0xffffffffll);
        if ((uint32_t)qi[b] >= t.ext[b]) return RT_ERR_SOURCE_OUTSIDE;
        // fh = qf rounded to a float; qf - fh is below 2^7 in magnitude, so
        // both are taken without 64-bit conversions: fh is an integer of at
        // most 33 bits, read back from its exponent and significand
        const float fh = __uint2float_rn(qf[b]);
        const uint32_t fb = __float_as_uint(fh);
        const int fe = (int)(fb >> 23) - 150;  // fh = (significand) 2^fe
        const uint64_t fm = (uint64_t)((fb & 0x7fffffu) | 0x800000u);
        const long long back = (long long)(fe >= 0 ? fm << fe : fm >> min(-fe, 24));  // fh = 0: 0
        ph[b] = fh * 0x1p-32f;
        pl[b] = __int2float_rn((int)((long long)qf[b] - back)) * 0x1p-32f;
    }
    return RT_OK;
}

// Exit axis b of the grid walk steps one cell: the domain-exit test, its
// far-face distance and exit time, and its dilated index.  Under LOCK, y moves
// with x, whose distance has already grown (x steps first).
template <int b, bool QZ, bool LOCK>
__device__ __forceinline__ void grid_step(float Af[3], const float Alim[3], const float ph[3], const float pl[3],
                                          const float ih[3], const float il[3], float th[3], float tl[3],
                                          uint32_t dl[3], float fsize, bool& leaving)
{
    if (LOCK && b == 1) {
        leaving |= Af[0] == Alim[1];
    } else {
        leaving |= Af[b] == Alim[b];
        Af[b] = __fadd_rn(Af[b], fsize);
        exit_time<QZ>(Af[b], ph[b], pl[b], ih[b], il[b], th[b], tl[b]);
    }
    dl[b] = (dl[b] + (1u << b)) | dil_holes(b);
}

// Walk of one ray through a full cube of equal-level leaves (level L <= 10),
// F32-Kahan arithmetic, for a direction whose moving axes are the bits of VM.
//
// The walk runs in a mirrored frame: a moving axis with m_b < 0 is reflected
// (cell c -> N1 - c = c ^ N1, distance A -> -A, inv -> -inv), so every moving
// axis advances by +1 cell and every exit time is |A - frac| |inv|, bitwise
// the value of the unreflected form because rounding is sign-symmetric.  Per
// axis the walk keeps the far-face distance A (an exact float) and the
// double-float exit time, changed only when the axis steps, and the mirrored
// cell index in dilated Morton form with the other axes' bit positions set to
// one, so that a step is one add and one OR and the leaf index is the AND of
// the three fields, reflected back by one XOR.  The ray leaves the cube when
// an exit axis steps out of a leaf whose far face is the domain boundary.
//
// LOCK (VM 3 or 7, QZ sources, bitwise-equal |inv_x| = |inv_y| and equal |A_x|,
// |A_y| at the source): x and y keep equal |A| and equal exit times for the
// whole walk (both grow by the leaf size whenever they step, together), so
// their exits always tie exactly and the choice is {x, y} against {z}.
template <int VM, bool QZ, bool LOCK, class V>
__device__ __forceinline__ int walk_f32k_grid(const DevTree& t, const DirConst* __restrict__ dp,
                                              const double* __restrict__ src, long long cap, V& vis,
                                              WalkCounters& wc)
{
    const int sh = kDepth - t.uniform_level;
    const int N1 = (1 << t.uniform_level) - 1;
    const float fsize = (float)(1 << sh);
    const int flags = __ldg(&dp->flags);
    float ih[3], il[3], ph[3], pl[3];
    int qi[3];
    uint32_t qf[3], dl[3];
    uint32_t xm = 0u;
    float Af[3], Alim[3], th[3], tl[3];
    float cE = 0.f;
    const int st = source_fixed(src, t, qi, qf, ph, pl);
    if (st != RT_OK) return st;
    if (QZ) {  // the fractions are zero: let the compiler drop them
#pragma unroll
        for (int b = 0; b < 3; b++) {
            qf[b] = 0u;
            ph[b] = pl[b] = 0.f;
        }
    }
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const int c = qi[b] >> sh;
        const bool neg = (VM & (1 << b)) && !((flags >> (3 + b)) & 1);
        dl[b] = (spread10((uint32_t)(neg ? (c ^ N1) : c)) << b) | dil_holes(b);
        if (neg) xm |= spread10((uint32_t)N1) << b;
        Af[b] = Alim[b] = th[b] = tl[b] = ih[b] = il[b] = 0.f;
        if (VM & (1 << b)) {
            // times in box lengths: ih and il scaled by 2^-21 (exact)
            ih[b] = fabsf(__ldg(&dp->ih[b])) * 0x1p-21f;
            il[b] = (neg ? -__ldg(&dp->il[b]) : __ldg(&dp->il[b])) * 0x1p-21f;
            if (neg) {
                ph[b] = -ph[b];
                pl[b] = -pl[b];
            }
            Af[b] = __int2float_rn(neg ? qi[b] - (c << sh) : ((c + 1) << sh) - qi[b]);
            Alim[b] = __int2float_rn(neg ? qi[b] : (1 << kDepth) - qi[b]);
            exit_time<QZ>(Af[b], ph[b], pl[b], ih[b], il[b], th[b], tl[b]);
            cE = fmaxf(cE, ih[b] * kEA);
        }
    }
    if (LOCK) Alim[1] = __fadd_rn(Alim[1], fsize);  // y is tested on A_x after x has stepped
    uint32_t j = (dl[0] & dl[1] & dl[2]) ^ xm;
    float tih = 0.f, til = 0.f;
    const uint32_t lim = wc.nseg + (uint32_t)min(cap, (long long)0x7fffffff);  // cap >= 1
    for (;;) {
        vis.pre(j);
        int bs;
        unsigned E;
        if (LOCK) {
            if (VM == 3) {
                E = 3u;
                bs = 0;
            } else if (__fsub_rn(th[2], th[0]) > (th[2] + th[0]) * kER + 2.f * cE) {
                E = 3u;
                bs = 0;
            } else if (__fsub_rn(th[0], th[2]) > (th[2] + th[0]) * kER + 2.f * cE) {
                E = 4u;
                bs = 2;
            } else {
                float thl[3] = {th[0], th[0], th[2]}, Afl[3] = {Af[0], Af[0], Af[2]};
                E = resolve_exit<VM, true>(thl, Afl, qf, ih, flags, dp, th[2] < th[0] ? 2 : 0, wc);
                bs = __ffs(E) - 1;
            }
        } else {
            E = exit_set<VM, QZ, true>(th, Af, qf, ih, flags, cE, dp, bs, wc);
        }
        const float ths = sel3(th, bs), tls = sel3(tl, bs);
        const float ds = diff_sum(ths, tls, tih, til);
        tih = ths;
        til = tls;
        wc.nseg++;
        bool leaving = false;
        // A warp whose lanes all take the same locked step (every lane of a
        // leaf-centre beam does) runs only that step's body.
        const unsigned am = (LOCK && VM == 7) ? __activemask() : 0u;
        if (LOCK && VM == 7 && __all_sync(am, E == 4u)) {
            grid_step<2, QZ, LOCK>(Af, Alim, ph, pl, ih, il, th, tl, dl, fsize, leaving);
        } else if (LOCK && VM == 7 && __all_sync(am, E == 3u)) {
            grid_step<0, QZ, LOCK>(Af, Alim, ph, pl, ih, il, th, tl, dl, fsize, leaving);
            grid_step<1, QZ, LOCK>(Af, Alim, ph, pl, ih, il, th, tl, dl, fsize, leaving);
        } else {
            if ((VM & 1) && (E & 1u)) grid_step<0, QZ, LOCK>(Af, Alim, ph, pl, ih, il, th, tl, dl, fsize, leaving);
            if ((VM & 2) && (E & 2u)) grid_step<1, QZ, LOCK>(Af, Alim, ph, pl, ih, il, th, tl, dl, fsize, leaving);
            if ((VM & 4) && (E & 4u)) grid_step<2, QZ, LOCK>(Af, Alim, ph, pl, ih, il, th, tl, dl, fsize, leaving);
        }
        // accumulated after the step, which needs no densities, so that the
        // step runs while the leaf's densities are still on their way
        vis.acc(ds);
        if (leaving || wc.nseg >= lim) {  // the cap ends a ray that still goes on
            if (leaving) break;
            return RT_ERR_STEP_LIMIT;
        }
        j = (dl[0] & dl[1] & dl[2]) ^ xm;
    }
    return RT_OK;
}

// ------------------------------------ two rays per lane on a uniform grid

// Two rays of one direction from sources on the depth-21 lattice (zero 32-bit
// fractions) whose distances to their cells' far faces are equal on every
// moving axis -- every two leaf centres of a uniform cube -- have the same
// exit times, exit choices and segment lengths, step for step: each path is
// the other translated by whole cells.  One lane walks both and takes each
// exit decision once; the leaf indices, the domain-exit tests, the densities
// and the sums are per ray.  Each ray's leaves, segment lengths and sums are
// bit for bit those of walk_f32k_grid.  kNoPair (nothing done): the sources
// do not qualify.
constexpr int kNoPair = -3;

template <int b, bool LOCK>
__device__ __forceinline__ void pair_step(float Af[3], const float Alim0[3], const float Alim1[3],
                                          const float ih[3], const float il[3], float th[3], float tl[3],
                                          uint32_t dl0[3], uint32_t dl1[3], float fsize, bool& lv0, bool& lv1)
{
    if (LOCK && b == 1) {  // y tracks x (stepped just before)
        lv0 |= Af[0] == Alim0[1];
        lv1 |= Af[0] == Alim1[1];
    } else {
        lv0 |= Af[b] == Alim0[b];
        lv1 |= Af[b] == Alim1[b];
        Af[b] = __fadd_rn(Af[b], fsize);
        exit_time<true>(Af[b], 0.f, 0.f, ih[b], il[b], th[b], tl[b]);
    }
    dl0[b] = (dl0[b] + (1u << b)) | dil_holes(b);
    dl1[b] = (dl1[b] + (1u << b)) | dil_holes(b);
}

template <int VM, bool LOCK, class V>
__device__ __forceinline__ int walk_f32k_grid_pair(const DevTree& t, const DirConst* __restrict__ dp,
                                                   const double* __restrict__ src0,
                                                   const double* __restrict__ src1, long long cap, V& v0,
                                                   V& v1, WalkCounters& w0, WalkCounters& w1, int& st1)
{
    const int sh = kDepth - t.uniform_level;
    const int N1 = (1 << t.uniform_level) - 1;
    const float fsize = (float)(1 << sh);
    const int flags = __ldg(&dp->flags);
    int q0[3], q1[3];
    uint32_t qf[3], qf1[3];
    float ph[3], pl[3];
    if (source_fixed(src0, t, q0, qf, ph, pl) != RT_OK || source_fixed(src1, t, q1, qf1, ph, pl) != RT_OK)
        return kNoPair;
    if ((qf[0] | qf[1] | qf[2] | qf1[0] | qf1[1] | qf1[2]) != 0u) return kNoPair;
    uint32_t dl0[3], dl1[3], xm = 0u;
    float Af[3], Alim0[3], Alim1[3], th[3], tl[3], ih[3], il[3];
    float cE = 0.f;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const int c0 = q0[b] >> sh, c1 = q1[b] >> sh;
        const bool neg = (VM & (1 << b)) && !((flags >> (3 + b)) & 1);
        dl0[b] = (spread10((uint32_t)(neg ? (c0 ^ N1) : c0)) << b) | dil_holes(b);
        dl1[b] = (spread10((uint32_t)(neg ? (c1 ^ N1) : c1)) << b) | dil_holes(b);
        if (neg) xm |= spread10((uint32_t)N1) << b;
        Af[b] = Alim0[b] = Alim1[b] = th[b] = tl[b] = ih[b] = il[b] = 0.f;
        if (VM & (1 << b)) {
            const int A0 = neg ? q0[b] - (c0 << sh) : ((c0 + 1) << sh) - q0[b];
            const int A1 = neg ? q1[b] - (c1 << sh) : ((c1 + 1) << sh) - q1[b];
            if (A0 != A1) return kNoPair;
            ih[b] = fabsf(__ldg(&dp->ih[b])) * 0x1p-21f;
            il[b] = (neg ? -__ldg(&dp->il[b]) : __ldg(&dp->il[b])) * 0x1p-21f;
            Af[b] = __int2float_rn(A0);
            Alim0[b] = __int2float_rn(neg ? q0[b] : (1 << kDepth) - q0[b]);
            Alim1[b] = __int2float_rn(neg ? q1[b] : (1 << kDepth) - q1[b]);
            exit_time<true>(Af[b], 0.f, 0.f, ih[b], il[b], th[b], tl[b]);
            cE = fmaxf(cE, ih[b] * kEA);
        }
    }
    if (LOCK) {
        Alim0[1] = __fadd_rn(Alim0[1], fsize);
        Alim1[1] = __fadd_rn(Alim1[1], fsize);
    }
    uint32_t j0 = (dl0[0] & dl0[1] & dl0[2]) ^ xm, j1 = (dl1[0] & dl1[1] & dl1[2]) ^ xm;
    float tih = 0.f, til = 0.f;
    const uint32_t capn = (uint32_t)min(cap, (long long)0x7fffffff);  // cap >= 1
    const uint32_t lim0 = w0.nseg + capn, lim1 = w1.nseg + capn;
    WalkCounters ws = {0u, 0u, 0u};  // exit fall-backs of the shared decisions so far
    bool a0 = true, a1 = true;
    int st0 = RT_OK;
    st1 = RT_OK;
    for (;;) {
        if (a0) v0.pre(j0);
        if (a1) v1.pre(j1);
        int bs;
        unsigned E;
        if (LOCK) {
            if (VM == 3) {
                E = 3u;
                bs = 0;
            } else if (__fsub_rn(th[2], th[0]) > (th[2] + th[0]) * kER + 2.f * cE) {
                E = 3u;
                bs = 0;
            } else if (__fsub_rn(th[0], th[2]) > (th[2] + th[0]) * kER + 2.f * cE) {
                E = 4u;
                bs = 2;
            } else {
                float thl[3] = {th[0], th[0], th[2]}, Afl[3] = {Af[0], Af[0], Af[2]};
                E = resolve_exit<VM, true>(thl, Afl, qf, ih, flags, dp, th[2] < th[0] ? 2 : 0, ws);
                bs = __ffs(E) - 1;
            }
        } else {
            E = exit_set<VM, true, true>(th, Af, qf, ih, flags, cE, dp, bs, ws);
        }
        const float ths = sel3(th, bs), tls = sel3(tl, bs);
        const float ds = diff_sum(ths, tls, tih, til);
        tih = ths;
        til = tls;
        bool lv0 = false, lv1 = false;
        const unsigned am = (LOCK && VM == 7) ? __activemask() : 0u;
        if (LOCK && VM == 7 && __all_sync(am, E == 4u)) {
            pair_step<2, LOCK>(Af, Alim0, Alim1, ih, il, th, tl, dl0, dl1, fsize, lv0, lv1);
        } else if (LOCK && VM == 7 && __all_sync(am, E == 3u)) {
            pair_step<0, LOCK>(Af, Alim0, Alim1, ih, il, th, tl, dl0, dl1, fsize, lv0, lv1);
            pair_step<1, LOCK>(Af, Alim0, Alim1, ih, il, th, tl, dl0, dl1, fsize, lv0, lv1);
        } else {
            if ((VM & 1) && (E & 1u)) pair_step<0, LOCK>(Af, Alim0, Alim1, ih, il, th, tl, dl0, dl1, fsize, lv0, lv1);
            if ((VM & 2) && (E & 2u)) pair_step<1, LOCK>(Af, Alim0, Alim1, ih, il, th, tl, dl0, dl1, fsize, lv0, lv1);
            if ((VM & 4) && (E & 4u)) pair_step<2, LOCK>(Af, Alim0, Alim1, ih, il, th, tl, dl0, dl1, fsize, lv0, lv1);
        }
        // each ray is accumulated after the step, as in walk_f32k_grid
        if (a0) {
            v0.acc(ds);
            w0.nseg++;
            if (lv0 || w0.nseg >= lim0) {  // the cap ends a ray that still goes on
                a0 = false;
                st0 = lv0 ? RT_OK : RT_ERR_STEP_LIMIT;
                w0.exit_fb += ws.exit_fb;
            }
        }
        if (a1) {
            v1.acc(ds);
            w1.nseg++;
            if (lv1 || w1.nseg >= lim1) {
                a1 = false;
                st1 = lv1 ? RT_OK : RT_ERR_STEP_LIMIT;
                w1.exit_fb += ws.exit_fb;
            }
        }
        if (!(a0 || a1)) break;
        j0 = (dl0[0] & dl0[1] & dl0[2]) ^ xm;
        j1 = (dl1[0] & dl1[1] & dl1[2]) ^ xm;
    }
    return st0;
}

// True when the x and y exits of a QZ source on a uniform grid stay locked:
// both axes move, |inv_x| = |inv_y| bitwise, and the source is as far from
// its leaf's far x face as from its far y face.
__device__ __forceinline__ bool xy_locked(const DevTree& t, int flags, const double* __restrict__ src)
{
    if ((flags & 3) != 3 || !inv_equal(flags, 0, 1)) return false;
    long long qx, qy;
    if (!fixed_source(src[0], qx) || !fixed_source(src[1], qy)) return false;
    const int sh = kDepth - t.uniform_level;
    const int size = 1 << sh;
    const int rx = (int)(qx >> 32) & (size - 1), ry = (int)(qy >> 32) & (size - 1);
    const int ax = ((flags >> 3) & 1) ? size - rx : rx;
    const int ay = ((flags >> 4) & 1) ? size - ry : ry;
    return ax == ay;
}

// walk_f32k_grid_pair for the direction's moving axes, with the x/y lock when
// the first source has it (the second, at the same offsets, then has it too).
template <class V>
__device__ __forceinline__ int walk_grid_pair(const DevTree& t, const DirConst* __restrict__ dp,
                                              const double* __restrict__ src0, const double* __restrict__ src1,
                                              long long cap, V& v0, V& v1, WalkCounters& w0, WalkCounters& w1,
                                              int& st1)
{
    const int flags = __ldg(&dp->flags);
    const int vm = flags & 7;
    if ((vm == 3 || vm == 7) && xy_locked(t, flags, src0)) {
        if (vm == 3) return walk_f32k_grid_pair<3, true>(t, dp, src0, src1, cap, v0, v1, w0, w1, st1);
        return walk_f32k_grid_pair<7, true>(t, dp, src0, src1, cap, v0, v1, w0, w1, st1);
    }
    switch (vm) {
    case 1: return walk_f32k_grid_pair<1, false>(t, dp, src0, src1, cap, v0, v1, w0, w1, st1);
    case 2: return walk_f32k_grid_pair<2, false>(t, dp, src0, src1, cap, v0, v1, w0, w1, st1);
    case 3: return walk_f32k_grid_pair<3, false>(t, dp, src0, src1, cap, v0, v1, w0, w1, st1);
    case 4: return walk_f32k_grid_pair<4, false>(t, dp, src0, src1, cap, v0, v1, w0, w1, st1);
    case 5: return walk_f32k_grid_pair<5, false>(t, dp, src0, src1, cap, v0, v1, w0, w1, st1);
    case 6: return walk_f32k_grid_pair<6, false>(t, dp, src0, src1, cap, v0, v1, w0, w1, st1);
    default: return walk_f32k_grid_pair<7, false>(t, dp, src0, src1, cap, v0, v1, w0, w1, st1);
    }
}

// ------------------------------------ F32-Kahan walk on a general octree

// A float of the direction table, loaded where it is used (a volatile load,
// so it is not hoisted into a register held across the walk).
__device__ __forceinline__ float dir_const(const float* p)
{
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// floor(v) for |v| < 2^22 without a conversion instruction: v + 1.5 * 2^23
// rounded down lies in [2^23, 2^24), where floats are the integers.
__device__ __forceinline__ int floor_small(float v)
{
    return __float_as_int(__fadd_rd(v, 12582912.0f)) - 0x4B400000;
}

// Leaf containing the depth-21 point c, and its level.  The coarse table gives
// the leaf directly for a coarse cell inside one leaf or of one level (no key
// or level is read then); a mixed cell is searched by key.  -1: no leaf.
__device__ __forceinline__ long long find_leaf(const DevTree& t, const uint32_t c[3], int& level)
{
    const int s = kDepth - t.T;
    const uint32_t cell = (s_spread10[(c[0] >> s) & 1023u] | (s_spread10[(c[1] >> s) & 1023u] << 1) |
                           (s_spread10[(c[2] >> s) & 1023u] << 2)) &
                          ((1u << (3 * t.T)) - 1u);
    const uint64_t e = __ldg(t.table + cell);
    const int code = (int)(e & 63u);
    const long long first = (long long)(e >> 6);
    if (code <= t.T) {
        level = code;
        return first;
    }
    if (code <= kDepth) {
        const int sl = kDepth - code, nb = code - t.T;  // nb: bits per axis of the index within the cell
        const uint32_t mask = (1u << nb) - 1u;
        level = code;
        if (nb == 1)  // one level below the table: the octant
            return first + (long long)(((c[0] >> sl) & 1u) | (((c[1] >> sl) & 1u) << 1) | (((c[2] >> sl) & 1u) << 2));
        if (nb <= 10)  // the 30-bit interleave suffices
            return first + (long long)((s_spread10[(c[0] >> sl) & mask] | (s_spread10[(c[1] >> sl) & mask] << 1) |
                                        (s_spread10[(c[2] >> sl) & mask] << 2)) &
                                       ((1u << (3 * nb)) - 1u));
        const uint64_t local = spread21((c[0] >> sl) & mask) | (spread21((c[1] >> sl) & mask) << 1) |
                               (spread21((c[2] >> sl) & mask) << 2);
        return first + (long long)local;
    }
    if (code == kCodeHole) return -1;
    const uint64_t M = interleave3(c[0], c[1], c[2]);
    const uint64_t ncell = 1ull << (3 * t.T);
    long long hi = ((uint64_t)cell + 1 < ncell) ? (long long)(__ldg(t.table + cell + 1) >> 6) : t.n;
    long long lo = first;  // keys[lo] == cell base <= M
    while (hi - lo > 1) {
        const long long mid = (lo + hi) >> 1;
        if (__ldg(t.keys + mid) <= M) lo = mid;
        else hi = mid;
    }
    const uint64_t key = __ldg(t.keys + lo);
    level = __ldg(t.levels + lo);
    if (M - key >= (1ull << (3 * (kDepth - level)))) return -1;
    return lo;
}

// Walk of one ray through a general octree, F32-Kahan arithmetic, moving axes
// VM (compile time).  Exit decisions as in walk_f32k_grid.  The next leaf is
// looked up at the lower corner of the current leaf on the non-stepped axes;
// only when that neighbour is finer, at the FP32 position of the non-stepped
// axes when its certified interval lies inside the leaf found, else at the
// FP64 position.
template <int VM, bool QZ, class V, class R = NoResume>
__device__ __forceinline__ int walk_f32k_tree(const DevTree& t, const DirConst* __restrict__ dp,
                                              const double* __restrict__ src, long long cap, V& vis,
                                              WalkCounters& wc, R* rs = nullptr)
{
    // The direction's constants (ih, il, m32) are read from the direction
    // table where they are used: one broadcast load per warp, kept out of the
    // per-ray registers.
    const int flags = __ldg(&dp->flags);
    float ph[3], pl[3], qif[3];  // qif: 2^23 + qi, exact
    int qi[3];
    uint32_t qf[3], c[3];
    float cE = 0.f;
    const int st = source_fixed(src, t, qi, qf, ph, pl);
    if (st != RT_OK) return st;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        qif[b] = __int_as_float(0x4B000000 | qi[b]);
        c[b] = (uint32_t)qi[b];
        if (VM & (1 << b)) cE = fmaxf(cE, fabsf(dir_const(&dp->ih[b])) * kEA);
    }
    int level;
    long long j;
    uint32_t size, lo[3];
    float tih = 0.f, til = 0.f;
    if (R::enabled && rs->s->status == 1) {
        j = rs->s->j;
        level = rs->s->level;
        size = 1u << (kDepth - level);
#pragma unroll
        for (int b = 0; b < 3; b++) lo[b] = rs->s->lo[b];
        tih = rs->s->th;
        til = rs->s->tl;
    } else {
        j = find_leaf(t, c, level);
        if (j < 0) return RT_ERR_LOOKUP_MISS;
        size = 1u << (kDepth - level);
#pragma unroll
        for (int b = 0; b < 3; b++) lo[b] = c[b] & ~(size - 1u);
    }
    // cap >= 1; a resumed walk counts from the ray's start (wc.nseg holds it)
    const uint32_t lim = (R::enabled ? 0u : wc.nseg) + (uint32_t)min(cap, (long long)0x7fffffff);
    for (;;) {
        if (R::enabled && !rs->inside(j)) {
            rs->s->j = (uint32_t)j;
#pragma unroll
            for (int b = 0; b < 3; b++) rs->s->lo[b] = lo[b];
            rs->s->level = (uint8_t)(kDepth - (31 - __clz(size)));
            rs->s->th = tih;
            rs->s->tl = til;
            rs->s->nseg = wc.nseg;
            return kSuspended;
        }
        vis.pre((uint32_t)j);
        float Af[3], th[3], tl[3], ih[3];
#pragma unroll
        for (int b = 0; b < 3; b++) {
            Af[b] = th[b] = tl[b] = ih[b] = 0.f;
            if (VM & (1 << b)) {
                ih[b] = dir_const(&dp->ih[b]);
                const uint32_t F = ((flags >> (3 + b)) & 1) ? lo[b] + size : lo[b];
                // (2^23 + F) - (2^23 + qi) = F - qi: integers below 2^24, exact
                Af[b] = __fsub_rn(__int_as_float(0x4B000000 | (int)F), qif[b]);
                if (QZ) {
                    th[b] = __fmul_rn(Af[b], ih[b]);
                } else {
                    th[b] = __fmul_rn(__fsub_rn(Af[b], ph[b]), ih[b]);
                }
            }
        }
        int bs;
        const unsigned E = exit_set<VM, QZ, false>(th, Af, qf, ih, flags, cE, dp, bs, wc);
        float the, tle;
        exit_time<QZ>(sel3(Af, bs), sel3(ph, bs), sel3(pl, bs), sel3(ih, bs), dir_const(&dp->il[bs]), the, tle);
        const float ds = __fmul_rn(__fadd_rn(__fsub_rn(the, tih), __fsub_rn(tle, til)), 0x1p-21f);
        tih = the;
        til = tle;
        vis.acc(ds);
        wc.nseg++;
        // Step the exit axes; a moving axis that does not step first takes the
        // leaf's lower corner.  The leaf found there is the neighbour of the
        // definition unless it is finer than the current leaf: a leaf at least
        // as large covers the whole face-adjacent cell of the current size
        // (octree cells are aligned), so any exit point on the face lands in it.
        bool leaving = false;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const int pos = (flags >> (3 + b)) & 1;
            if ((VM & (1 << b)) && (E & (1u << b))) {
                if (pos ? (lo[b] + size >= t.ext[b]) : (lo[b] == 0)) leaving = true;
                c[b] = pos ? lo[b] + size : lo[b] - 1;
            } else if (!(VM & (1 << b))) {
                c[b] = (uint32_t)qi[b];  // a fixed coordinate stays inside every leaf on the path
            } else {
                c[b] = lo[b];
            }
        }
        if (leaving) break;
        const uint32_t size0 = size;  // the current leaf's size
        j = find_leaf(t, c, level);
        size = 1u << (kDepth - level);
        if ((VM & ~E) != 0u && j >= 0 && size < size0) {
            // a finer neighbour: position the moving non-exit axes on a
            // certified interval around the exit point
            const float ihe = sel3(ih, bs);
            bool wide = false;
            uint32_t chi[3];
#pragma unroll
            for (int b = 0; b < 3; b++) {
                chi[b] = c[b];
                if ((VM & (1 << b)) && !(E & (1u << b))) {
                    const uint32_t hib = lo[b] + size0 - 1;
                    const float m32 = dir_const(&dp->m32[b]);
                    const float mw = __fmul_rn(the, m32);
                    const float w = QZ ? mw : __fadd_rn(mw, ph[b]);
                    const float del = (fabsf(mw) + fabsf(w)) * 0x1p-21f + fabsf(m32) * fabsf(ihe) * 0x1p-22f +
                                      0x1p-22f;
                    // |w| + del < 2^22: floor by adding 1.5 * 2^23 rounded down
                    const int l0 = qi[b] + floor_small(__fsub_rd(w, del));
                    const int l1 = qi[b] + floor_small(__fadd_ru(w, del));
                    c[b] = (uint32_t)min(max(l0, (int)lo[b]), (int)hib);
                    chi[b] = (uint32_t)min(max(l1, (int)lo[b]), (int)hib);
                    wide |= chi[b] != c[b];
                }
            }
            j = find_leaf(t, c, level);
            size = 1u << (kDepth - level);
            if (wide && j >= 0) {
#pragma unroll
                for (int b = 0; b < 3; b++)
                    if (chi[b] >= (c[b] & ~(size - 1u)) + size) j = -2;
            }
            if (j == -2 || (j < 0 && wide)) {
                // FP64 position of the definition: floor((Q + t_out m) 2^21)
                wc.lookup_fb++;
                const long long De = ((long long)small_float_to_int(sel3(Af, bs)) << 32) - (long long)sel3(qf, bs);
                const double te = __dmul_rn(__dmul_rn(__ll2double_rn(De), 0x1p-53), __ldg(&dp->inv[bs]));
#pragma unroll
                for (int b = 0; b < 3; b++) {
                    if ((VM & (1 << b)) && !(E & (1u << b))) {
                        const long long qb = ((long long)qi[b] << 32) | (long long)qf[b];
                        const double Qb = __dmul_rn(__ll2double_rn(qb), 0x1p-53);
                        const double P = __dadd_rn(Qb, __dmul_rn(te, __ldg(&dp->m[b])));
                        double f = floor(__dmul_rn(P, 0x1p21));
                        f = fmax(f, (double)lo[b]);
                        f = fmin(f, (double)(lo[b] + size0 - 1));
                        c[b] = (uint32_t)f;
                    }
                }
                j = find_leaf(t, c, level);
                size = 1u << (kDepth - level);
            }
        }
        if (j < 0) return RT_ERR_LOOKUP_MISS;
        if (wc.nseg >= lim) return RT_ERR_STEP_LIMIT;  // the cap ends a ray that still goes on
#pragma unroll
        for (int b = 0; b < 3; b++) lo[b] = c[b] & ~(size - 1u);
    }
    return RT_OK;
}

// True when every coordinate of the source has a zero 32-bit fraction on the
// depth-21 lattice (every leaf centre down to level 20 does).
__device__ __forceinline__ bool source_on_lattice(const double* __restrict__ src)
{
    bool z = true;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        long long q;
        if (fixed_source(src[b], q)) z = z && ((q & 0xffffffffll) == 0);
    }
    return z;
}

template <bool QZ, class V>
__device__ __forceinline__ int walk_grid_vm(int vm, const DevTree& t, const DirConst* __restrict__ dp,
                                            const double* __restrict__ src, long long cap, V& vis,
                                            WalkCounters& wc)
{
    if (QZ && (vm == 3 || vm == 7) && xy_locked(t, __ldg(&dp->flags), src)) {
        if (vm == 3) return walk_f32k_grid<3, true, true>(t, dp, src, cap, vis, wc);
        return walk_f32k_grid<7, true, true>(t, dp, src, cap, vis, wc);
    }
    switch (vm) {
    case 1: return walk_f32k_grid<1, QZ, false>(t, dp, src, cap, vis, wc);
    case 2: return walk_f32k_grid<2, QZ, false>(t, dp, src, cap, vis, wc);
    case 3: return walk_f32k_grid<3, QZ, false>(t, dp, src, cap, vis, wc);
    case 4: return walk_f32k_grid<4, QZ, false>(t, dp, src, cap, vis, wc);
    case 5: return walk_f32k_grid<5, QZ, false>(t, dp, src, cap, vis, wc);
    case 6: return walk_f32k_grid<6, QZ, false>(t, dp, src, cap, vis, wc);
    default: return walk_f32k_grid<7, QZ, false>(t, dp, src, cap, vis, wc);
    }
}

template <bool QZ, class V>
__device__ __forceinline__ int walk_tree_vm(int vm, const DevTree& t, const DirConst* __restrict__ dp,
                                            const double* __restrict__ src, long long cap, V& vis,
                                            WalkCounters& wc)
{
    switch (vm) {
    case 1: return walk_f32k_tree<1, QZ>(t, dp, src, cap, vis, wc);
    case 2: return walk_f32k_tree<2, QZ>(t, dp, src, cap, vis, wc);
    case 3: return walk_f32k_tree<3, QZ>(t, dp, src, cap, vis, wc);
    case 4: return walk_f32k_tree<4, QZ>(t, dp, src, cap, vis, wc);
    case 5: return walk_f32k_tree<5, QZ>(t, dp, src, cap, vis, wc);
    case 6: return walk_f32k_tree<6, QZ>(t, dp, src, cap, vis, wc);
    default: return walk_f32k_tree<7, QZ>(t, dp, src, cap, vis, wc);
    }
}

template <bool QZ, class V, class R>
__device__ __forceinline__ int walk_tree_vm_r(int vm, const DevTree& t, const DirConst* __restrict__ dp,
                                              const double* __restrict__ src, long long cap, V& vis,
                                              WalkCounters& wc, R* rs)
{
    switch (vm) {
    case 1: return walk_f32k_tree<1, QZ>(t, dp, src, cap, vis, wc, rs);
    case 2: return walk_f32k_tree<2, QZ>(t, dp, src, cap, vis, wc, rs);
    case 3: return walk_f32k_tree<3, QZ>(t, dp, src, cap, vis, wc, rs);
    case 4: return walk_f32k_tree<4, QZ>(t, dp, src, cap, vis, wc, rs);
    case 5: return walk_f32k_tree<5, QZ>(t, dp, src, cap, vis, wc, rs);
    case 6: return walk_f32k_tree<6, QZ>(t, dp, src, cap, vis, wc, rs);
    default: return walk_f32k_tree<7, QZ>(t, dp, src, cap, vis, wc, rs);
    }
}

// General-octree walk of one ray that traces only the leaves of rs's chunk:
// it starts (status 0) or resumes (status 1) from rs->s and returns
// kSuspended, with the state saved, at the first leaf outside the chunk.
// wc.nseg must hold the ray's segment count so far.
template <int MODE, class V>
__device__ __forceinline__ int walk_chunk(const DevTree& t, const DirConst* __restrict__ dp,
                                          const double* __restrict__ src, long long cap, V& vis,
                                          WalkCounters& wc, ChunkResume* rs)
{
    if (MODE == RT_MODE_FP64) {
        const DirConst d = *dp;
        return walk_fp64<false>(t, d, src, cap, vis, wc, rs);
    }
    const int vm = __ldg(&dp->flags) & 7;
    return source_on_lattice(src) ? walk_tree_vm_r<true>(vm, t, dp, src, cap, vis, wc, rs)
                                  : walk_tree_vm_r<false>(vm, t, dp, src, cap, vis, wc, rs);
}

// Walk of one ray (direction *dp, in global memory) in either arithmetic form.
template <int MODE, bool UNIFORM, class V>
__device__ __forceinline__ int walk(const DevTree& t, const DirConst* __restrict__ dp,
                                    const double* __restrict__ src, long long cap, V& vis,
                                    WalkCounters& wc)
{
    if (MODE == RT_MODE_FP64) {
        if (UNIFORM) {
            const int fl = __ldg(&dp->flags);
            if (((fl & 7) == 3 || (fl & 7) == 7) && xy_locked_fp64(t, fl, src)) {
                if ((fl & 7) == 3) return walk_fp64_grid<3, true>(t, dp, src, cap, vis, wc);
                return walk_fp64_grid<7, true>(t, dp, src, cap, vis, wc);
            }
            switch (fl & 7) {
            case 1: return walk_fp64_grid<1, false>(t, dp, src, cap, vis, wc);
            case 2: return walk_fp64_grid<2, false>(t, dp, src, cap, vis, wc);
            case 3: return walk_fp64_grid<3, false>(t, dp, src, cap, vis, wc);
            case 4: return walk_fp64_grid<4, false>(t, dp, src, cap, vis, wc);
            case 5: return walk_fp64_grid<5, false>(t, dp, src, cap, vis, wc);
            case 6: return walk_fp64_grid<6, false>(t, dp, src, cap, vis, wc);
            default: return walk_fp64_grid<7, false>(t, dp, src, cap, vis, wc);
            }
        }
        const DirConst d = *dp;
        return walk_fp64<UNIFORM>(t, d, src, cap, vis, wc);
    }
    const int vm = __ldg(&dp->flags) & 7;
    const bool qz = source_on_lattice(src);
    if (UNIFORM)
        return qz ? walk_grid_vm<true>(vm, t, dp, src, cap, vis, wc) : walk_grid_vm<false>(vm, t, dp, src, cap, vis, wc);
    return qz ? walk_tree_vm<true>(vm, t, dp, src, cap, vis, wc) : walk_tree_vm<false>(vm, t, dp, src, cap, vis, wc);
}

// ------------------------------------------------------------- densities

// Exact float -> double in integer operations: sign, exponent rebiased by
// 1023 - 127 and the mantissa shifted up 29 bits; a subnormal is first scaled
// by 2^24 in FP32 (exact) and rebiased 24 less; zeros, infinities and NaNs
// keep their class.  No instruction of the FP64 pipe is issued.
__device__ __forceinline__ double widen_f32(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t a = u & 0x7fffffffu;
    const bool sub = a < 0x00800000u;
    const uint32_t un = sub ? __float_as_uint(__fmul_rn(__uint_as_float(a), 0x1p24f)) : a;
    uint32_t hi = (un >> 3) + (sub ? 0x38000000u - (24u << 20) : 0x38000000u);
    hi = (a >= 0x7f800000u) ? ((a >> 3) | 0x7ff00000u) : hi;
    hi = (a == 0u) ? 0u : hi;
    return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)(un << 29));
}
template <class T>
__device__ __forceinline__ T from_f32(float f) { return (T)f; }
template <>
__device__ __forceinline__ double from_f32<double>(float f) { return widen_f32(f); }

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
                n[0] = from_f32<T>(__ldg(p + j));
            } else if (SM == 2) {
                const float2 v = __ldg((const float2*)p + j);
                n[0] = from_f32<T>(v.x); n[1] = from_f32<T>(v.y);
            } else {
#pragma unroll
                for (int h = 0; h < SM / 4; h++) {
                    const float4 v = __ldg((const float4*)p + (size_t)j * (SM / 4) + h);
                    n[4 * h] = from_f32<T>(v.x); n[4 * h + 1] = from_f32<T>(v.y);
                    n[4 * h + 2] = from_f32<T>(v.z); n[4 * h + 3] = from_f32<T>(v.w);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < SM; k++) n[k] = (k < S) ? from_f32<T>(__ldg(p + (size_t)j * S + k)) : (T)0;
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
