/*
 * Plain FP64 CPU oracle for direction-dependent column densities
 * (RAYTHEIA, arXiv 2605.09882).  TEST INFRASTRUCTURE ONLY: the tests, the
 * package smoke check and the benchmark's CPU-baseline leg call it; the
 * product path never does.  It shares no code with the CUDA library.
 *
 * What it computes (Sec. 2.2, Eq. for I(p,q)): for every source p and
 * HEALPix direction q, I(p,q,k) = sum over intersected leaves j of
 * n_k[j] * r_cell,j, where r_cell,j = t_out - t_in is the slab-method chord
 * of the ray R = Q + m t through leaf j (Sec. 2.2.2, Eqs. for t_i, t_in < t_out
 * and r_cell).  The leaves are found by the DDA walk of Sec. 2.2.1: advance to
 * the next cell boundary, encode the advanced position as a Morton code and
 * find the leaf by a lookup in the sorted key array.
 *
 * Readings where the paper is silent (each one fixes bits both sides share):
 *  - depth D = 21 lattice, key = interleave(x, y, z) with x in bit 3b;
 *  - sources are truncated to the 2^-53 lattice before tracing, so every
 *    face-minus-source difference F - Q is exact in FP64;
 *  - t_b = (F_b - Q_b) * inv_b with inv_b = 1 / m_b evaluated once per ray;
 *  - t_in is the previous t_out (0 at the source), so ds = t_out - t_in;
 *  - every axis whose t_b equals t_out exactly is stepped at once;
 *  - an axis that is not stepped takes floor((Q_b + t_out m_b) 2^21), clamped
 *    into the current leaf's extent on that axis;
 *  - the walk ends when a stepped axis leaves the domain extent.
 * All arithmetic is IEEE FP64 round-to-nearest with no contraction
 * (build with -ffp-contract=off).
 *
 * Parity status of each function against the paper: pinned by the tests in
 * tests/test_oracle_*.py (closed forms, invariants, brute force); the paper
 * itself prints no column or path values, so no test compares against a
 * printed number.
 */
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_D 21

/* OR_MUTANT selects a planted mistake (tests only, to show that the pins
 * catch it); 0 is the oracle proper. */
#ifndef OR_MUTANT
#define OR_MUTANT 0
#endif

enum {
    OR_OK = 0,
    OR_ERR_ARG = 1,
    OR_ERR_UNSORTED = 2,
    OR_ERR_MISALIGNED = 3,
    OR_ERR_OVERLAP_OR_GAP = 4,
    OR_ERR_SOURCE_OUTSIDE = 5,
    OR_ERR_STEP_LIMIT = 6,
    OR_ERR_NONFINITE = 7,
    OR_ERR_MISS = 10
};

/* ---------------------------------------------------------------- Morton */

/* Morton code of a depth-21 integer point: bit b of x goes to bit 3b,
 * of y to 3b + 1, of z to 3b + 2 (Sec. 2.2.1, "Morton Codes"). */
uint64_t or_morton_encode(uint32_t x, uint32_t y, uint32_t z)
{
    uint64_t key = 0;
    for (int b = 0; b < OR_D; b++) {
#if OR_MUTANT == 1 /* x and y bits transposed */
        key |= (uint64_t)((y >> b) & 1u) << (3 * b);
        key |= (uint64_t)((x >> b) & 1u) << (3 * b + 1);
#else
        key |= (uint64_t)((x >> b) & 1u) << (3 * b);
        key |= (uint64_t)((y >> b) & 1u) << (3 * b + 1);
#endif
        key |= (uint64_t)((z >> b) & 1u) << (3 * b + 2);
    }
    return key;
}

void or_morton_decode(uint64_t key, uint32_t xyz[3])
{
    xyz[0] = xyz[1] = xyz[2] = 0;
    for (int b = 0; b < OR_D; b++) {
        xyz[0] |= (uint32_t)((key >> (3 * b)) & 1u) << b;
        xyz[1] |= (uint32_t)((key >> (3 * b + 1)) & 1u) << b;
        xyz[2] |= (uint32_t)((key >> (3 * b + 2)) & 1u) << b;
    }
}

void or_morton_encode_many(const uint32_t* xyz, int64_t n, uint64_t* keys)
{
    for (int64_t i = 0; i < n; i++)
        keys[i] = or_morton_encode(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]);
}

void or_morton_decode_many(const uint64_t* keys, int64_t n, uint32_t* xyz)
{
    for (int64_t i = 0; i < n; i++) or_morton_decode(keys[i], xyz + 3 * i);
}

/* --------------------------------------------------------------- HEALPix */

/* cos and sin of (pi/2) * r / den for 0 <= r < den, evaluated in the first
 * octant so that the mirror symmetry about pi/4 holds bitwise. */
static void quarter_cos_sin(int64_t r, int64_t den, double* c, double* s)
{
    if (2 * r == den) {
        *c = sqrt(0.5);
        *s = *c;
    } else if (2 * r < den) {
        double a = (M_PI / 2.0) * (double)r / (double)den;
        *c = cos(a);
        *s = sin(a);
    } else {
        double a = (M_PI / 2.0) * (double)(den - r) / (double)den;
        *c = sin(a);
        *s = cos(a);
    }
}

/* Unit vector with z = zn / zd, azimuth (pi/2) * num / den. */
static void pixel_vector(int64_t zn, int64_t zd, int64_t num, int64_t den, double* v)
{
    int64_t quadrant = num / den;
    int64_t r = num % den;
    double c, s, cphi, sphi;
    quarter_cos_sin(r, den, &c, &s);
    switch (quadrant) {
    case 0: cphi = c; sphi = s; break;
    case 1: cphi = -s; sphi = c; break;
    case 2: cphi = -c; sphi = -s; break;
    default: cphi = s; sphi = -c; break;
    }
    double z = (double)zn / (double)zd;
    double st = sqrt((double)(zd * zd - zn * zn)) / (double)zd;
    v[0] = st * cphi;
    v[1] = st * sphi;
    v[2] = z;
    for (int b = 0; b < 3; b++)
        if (v[b] == 0.0) v[b] = 0.0; /* no negative zeros */
}

/* HEALPix pixel centres, RING order (Gorski et al. 2005), 12 nside^2 rows.
 * The paper uses N_rays = 12 * 4^l (Sec. 2, "HEALPix rays").
 * Rings i = 1 .. 4 nside - 1 from north to south; in each ring the azimuth
 * ascends from its smallest value in [0, 2 pi).
 *   polar cap (i < nside):   z = 1 - i^2 / (3 nside^2), phi = (pi / 2i)(j - 1/2), j = 1..4i
 *   equator (nside <= i <= 3 nside): z = 4/3 - 2i / (3 nside),
 *                            phi = (pi / 2 nside)(j - 1 + [(i - nside) even] / 2), j = 1..4 nside
 *   south cap: mirror of the north cap (z -> -z). */
int or_healpix(int nside, double* dirs)
{
    if (nside < 1 || nside > 1024) return OR_ERR_ARG;
    int64_t N = nside, p = 0;
    for (int64_t i = 1; i <= 4 * N - 1; i++) {
        if (i < N || i > 3 * N) {
            int64_t ii = (i < N) ? i : 4 * N - i;
            int64_t zd = 3 * N * N;
            int64_t zn = zd - ii * ii;
            if (i > 3 * N) zn = -zn;
            for (int64_t j = 1; j <= 4 * ii; j++, p++)
                /* (pi / 2i)(j - 1/2) = (pi/2) * (2j - 1) / (2 ii) */
                pixel_vector(zn, zd, 2 * j - 1, 2 * ii, dirs + 3 * p);
        } else {
            int64_t zd = 3 * N;
            int64_t zn = 4 * N - 2 * i;
#if OR_MUTANT == 2 /* half-pixel azimuth offset on the wrong rings */
            int64_t half = ((i - N) % 2 == 1) ? 1 : 0;
#else
            int64_t half = ((i - N) % 2 == 0) ? 1 : 0;
#endif
            for (int64_t j = 1; j <= 4 * N; j++, p++)
                /* (pi / 2N)(j - 1 + half/2) = (pi/2) * (2(j - 1) + half) / (2N) */
                pixel_vector(zn, zd, 2 * (j - 1) + half, 2 * N, dirs + 3 * p);
        }
    }
    return (p == 12 * N * N) ? OR_OK : OR_ERR_ARG;
}

/* --------------------------------------------------------------- octree */

typedef struct {
    const uint64_t* keys;
    const uint8_t* levels;
    int64_t n;
    uint32_t ext[3];
} or_tree;

static uint64_t leaf_span(uint8_t level) { return 1ull << (3 * (OR_D - level)); }

/* Checks that the leaves are a valid leaf-only linear octree tiling the
 * domain box [0, ext)^3 (depth-21 cells).  Precedence of the reported fault:
 * ARG > MISALIGNED > UNSORTED > OVERLAP_OR_GAP. */
int or_validate(const uint64_t* keys, const uint8_t* levels, int64_t n, const int32_t* extent)
{
    uint32_t ext[3];
    if (!keys || !levels || n <= 0 || n >= (1ll << 32)) return OR_ERR_ARG;
    for (int b = 0; b < 3; b++) {
        int32_t e = extent ? extent[b] : (1 << OR_D);
        if (e <= 0 || e > (1 << OR_D)) return OR_ERR_ARG;
        ext[b] = (uint32_t)e;
    }
    for (int64_t j = 0; j < n; j++)
        if (levels[j] > OR_D) return OR_ERR_ARG;
    for (int64_t j = 0; j < n; j++)
        if ((keys[j] >> 63) || (keys[j] & (leaf_span(levels[j]) - 1))) return OR_ERR_MISALIGNED;
    for (int64_t j = 0; j + 1 < n; j++)
        if (keys[j + 1] <= keys[j]) return OR_ERR_UNSORTED;
    for (int64_t j = 0; j + 1 < n; j++)
        if (keys[j + 1] - keys[j] < leaf_span(levels[j])) return OR_ERR_OVERLAP_OR_GAP;
    uint64_t vol = 0;
    for (int64_t j = 0; j < n; j++) {
        uint32_t c[3];
        or_morton_decode(keys[j], c);
        uint32_t size = 1u << (OR_D - levels[j]);
        for (int b = 0; b < 3; b++)
            if ((uint64_t)c[b] + size > ext[b]) return OR_ERR_OVERLAP_OR_GAP;
        vol += leaf_span(levels[j]);
    }
    if (vol != (uint64_t)ext[0] * ext[1] * ext[2]) return OR_ERR_OVERLAP_OR_GAP;
    return OR_OK;
}

/* Leaf containing depth-21 point c: the last key <= Morton(c), checked for
 * containment; -1 if none (cannot happen in a validated tree). */
static int64_t locate(const or_tree* t, const uint32_t c[3])
{
    uint64_t M = or_morton_encode(c[0], c[1], c[2]);
    int64_t lo = 0, hi = t->n; /* first index with key > M */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (t->keys[mid] <= M) lo = mid + 1;
        else hi = mid;
    }
    int64_t j = lo - 1;
    if (j < 0) return -1;
    if (M - t->keys[j] >= leaf_span(t->levels[j])) return -1;
    return j;
}

/* ----------------------------------------------------------------- walk */

typedef void (*visit_fn)(void* ctx, int64_t leaf, double ds);

/* The maximum number of segments a ray can have through cells of level
 * <= lmax: each step advances at least one axis past a face of the level-lmax
 * lattice. */
static int64_t step_cap(const or_tree* t)
{
    int lmax = 0;
    for (int64_t j = 0; j < t->n; j++)
        if (t->levels[j] > lmax) lmax = t->levels[j];
    return 3 * (1ll << lmax) + 3;
}

/* Walks the ray from src along m; calls visit for every segment.  Returns an
 * OR_ status; *nseg and *hash receive the segment count and the FNV-1a style
 * hash of the visited leaf indices. */
static int walk(const or_tree* t, const double src[3], const double m[3], int64_t cap,
                visit_fn visit, void* ctx, uint64_t* nseg, uint64_t* hash)
{
    double Q[3], inv[3];
    uint32_t c[3];
    uint64_t h = 0xcbf29ce484222325ull, count = 0;
    for (int b = 0; b < 3; b++) {
        if (!(src[b] >= 0.0 && src[b] < 1.0)) return OR_ERR_SOURCE_OUTSIDE;
        double q = floor(src[b] * 0x1p53); /* truncate to the 2^-53 lattice */
        Q[b] = q * 0x1p-53;
        c[b] = (uint32_t)floor(Q[b] * 0x1p21);
        if (c[b] >= t->ext[b]) return OR_ERR_SOURCE_OUTSIDE;
        inv[b] = (m[b] != 0.0) ? 1.0 / m[b] : 0.0;
    }
    int64_t j = locate(t, c);
    if (j < 0) return OR_ERR_MISS;
    double t_in = 0.0;
    for (int64_t step = 0;; step++) {
        if (step >= cap) return OR_ERR_STEP_LIMIT;
        uint32_t lo[3];
        or_morton_decode(t->keys[j], lo);
        uint32_t size = 1u << (OR_D - t->levels[j]);
        /* slab exits: the far face on every axis the ray moves along */
        double tb[3], t_out = INFINITY;
        for (int b = 0; b < 3; b++) {
            tb[b] = INFINITY;
            if (m[b] != 0.0) {
#if OR_MUTANT == 3 /* near face instead of far face */
                double F = (double)(m[b] > 0.0 ? lo[b] : lo[b] + size) * 0x1p-21;
#else
                double F = (double)(m[b] > 0.0 ? lo[b] + size : lo[b]) * 0x1p-21;
#endif
                tb[b] = (F - Q[b]) * inv[b];
                if (tb[b] < t_out) t_out = tb[b];
            }
        }
        double ds = t_out - t_in;
#if OR_MUTANT == 4 /* the source's own leaf dropped */
        if (visit && step > 0) visit(ctx, j, ds);
#else
        if (visit) visit(ctx, j, ds);
#endif
        h = (h ^ (uint64_t)j) * 0x100000001b3ull;
        count++;
#if OR_MUTANT != 5 /* t_in never advanced: ds = t_out */
        t_in = t_out;
#endif
        /* step every axis whose exit equals t_out; leave at the domain edge */
        int leaving = 0;
        uint32_t nc[3];
        for (int b = 0; b < 3; b++) {
#if OR_MUTANT == 6 /* only the first tied axis is stepped */
            int first_tie = 1;
            for (int a = 0; a < b; a++)
                if (m[a] != 0.0 && tb[a] == t_out) first_tie = 0;
            if (m[b] != 0.0 && tb[b] == t_out && first_tie) {
#else
            if (m[b] != 0.0 && tb[b] == t_out) {
#endif
                if (m[b] > 0.0) {
                    if ((uint64_t)lo[b] + size >= t->ext[b]) leaving = 1;
                    nc[b] = lo[b] + size;
                } else {
                    if (lo[b] == 0) leaving = 1;
                    nc[b] = lo[b] - 1;
                }
            } else {
                double P = Q[b] + t_out * m[b];
                double f = floor(P * 0x1p21);
                if (f < (double)lo[b]) f = (double)lo[b];
                if (f > (double)(lo[b] + size - 1)) f = (double)(lo[b] + size - 1);
                nc[b] = (uint32_t)f;
            }
        }
        if (leaving) break;
        j = locate(t, nc);
        if (j < 0) return OR_ERR_MISS;
    }
    if (nseg) *nseg = count;
    if (hash) *hash = h;
    return OR_OK;
}

/* ------------------------------------------------------------ threading */

typedef struct {
    const or_tree* tree;
    const double* dens; /* [n][S] */
    int S;
    const double* src;
    int64_t s0, s1;
    const double* dirs;
    int nd;
    int64_t cap;
    double* cols;     /* [n_src][nd][S] or NULL */
    uint64_t* hash;   /* [n_src][nd] or NULL */
    uint64_t* nseg;   /* [n_src][nd] or NULL */
    const double* g;  /* adjoint seed [n_src][nd][S] or NULL */
    double* grad;     /* private [n][S] buffer for the adjoint */
    int status;
} job_t;

typedef struct {
    const double* dens;
    int S;
    double* col;      /* forward: [S] */
    const double* g;  /* adjoint: [S] */
    double* grad;     /* adjoint: [n][S] */
    int bad;          /* forward: a crossed leaf's density is not a number density */
} seg_ctx;

static void visit_forward(void* vctx, int64_t j, double ds)
{
    seg_ctx* x = (seg_ctx*)vctx;
    for (int k = 0; k < x->S; k++) {
        const double d = x->dens[j * x->S + k];
        /* the integrated quantities are number densities: finite and >= 0 */
        if (!(d >= 0.0 && d <= DBL_MAX)) x->bad = 1;
        x->col[k] += d * ds;
    }
}

static void visit_adjoint(void* vctx, int64_t j, double ds)
{
    seg_ctx* x = (seg_ctx*)vctx;
#if OR_MUTANT == 7 /* adjoint drops the ds factor */
    (void)ds;
    for (int k = 0; k < x->S; k++) x->grad[j * x->S + k] += x->g[k];
#else
    for (int k = 0; k < x->S; k++) x->grad[j * x->S + k] += x->g[k] * ds;
#endif
}

static void* run_job(void* arg)
{
    job_t* jb = (job_t*)arg;
    double col[64];
    for (int64_t s = jb->s0; s < jb->s1; s++) {
        for (int q = 0; q < jb->nd; q++) {
            int64_t r = s * jb->nd + q;
            seg_ctx x;
            x.dens = jb->dens;
            x.S = jb->S;
            x.col = col;
            x.g = jb->g ? jb->g + r * jb->S : NULL;
            x.grad = jb->grad;
            x.bad = 0;
            for (int k = 0; k < jb->S; k++) col[k] = 0.0;
            visit_fn v = jb->g ? visit_adjoint : (jb->cols ? visit_forward : NULL);
            uint64_t ns = 0, h = 0;
            int st = walk(jb->tree, jb->src + 3 * s, jb->dirs + 3 * q, jb->cap, v, &x, &ns, &h);
            if (st == OR_OK && x.bad) st = OR_ERR_NONFINITE;
            if (st != OR_OK && jb->status == OR_OK) jb->status = st;
            if (st != OR_OK) { ns = 0; h = 0; for (int k = 0; k < jb->S; k++) col[k] = 0.0; }
            if (jb->cols)
                for (int k = 0; k < jb->S; k++) jb->cols[r * jb->S + k] = col[k];
            if (jb->hash) jb->hash[r] = h;
            if (jb->nseg) jb->nseg[r] = ns;
        }
    }
    return NULL;
}

/* The trace entry points trust the tree: call or_validate first. */
static int setup_tree(or_tree* t, const uint64_t* keys, const uint8_t* levels, int64_t n,
                      const int32_t* extent)
{
    if (!keys || !levels || n <= 0) return OR_ERR_ARG;
    t->keys = keys;
    t->levels = levels;
    t->n = n;
    for (int b = 0; b < 3; b++) {
        int32_t e = extent ? extent[b] : (1 << OR_D);
        if (e <= 0 || e > (1 << OR_D)) return OR_ERR_ARG;
        t->ext[b] = (uint32_t)e;
    }
    return OR_OK;
}

static int run_threads(job_t* base, int64_t n_src, int nthreads, int64_t n_leaves)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n_src < nthreads) nthreads = n_src > 0 ? (int)n_src : 1;
    job_t* jobs = (job_t*)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    int status = OR_OK;
    for (int i = 0; i < nthreads; i++) {
        jobs[i] = *base;
        jobs[i].s0 = n_src * i / nthreads;
        jobs[i].s1 = n_src * (i + 1) / nthreads;
        jobs[i].status = OR_OK;
        if (base->g) jobs[i].grad = (double*)calloc((size_t)(n_leaves * base->S), sizeof(double));
        pthread_create(&th[i], NULL, run_job, &jobs[i]);
    }
    for (int i = 0; i < nthreads; i++) {
        pthread_join(th[i], NULL);
        if (jobs[i].status != OR_OK && status == OR_OK) status = jobs[i].status;
    }
    if (base->g) { /* deterministic reduction in thread order */
        for (int i = 0; i < nthreads; i++) {
            for (int64_t e = 0; e < n_leaves * base->S; e++) base->grad[e] += jobs[i].grad[e];
            free(jobs[i].grad);
        }
    }
    free(jobs);
    free(th);
    return status;
}

/* Columns I(p,q,k) (Sec. 2.2, Alg. 1's accumulation) for every source and
 * direction; also the per-ray segment count and path hash.  Any output
 * pointer may be NULL.  dens is FP64 [n][S]: number densities, so a ray that
 * crosses a leaf whose density is NaN, infinite or negative has no column
 * (zeroed) and the call returns OR_ERR_NONFINITE. */
int or_trace(const uint64_t* keys, const uint8_t* levels, int64_t n, const int32_t* extent,
             const double* dens, int S, const double* src, int64_t n_src,
             const double* dirs, int nd, double* cols, uint64_t* hash, uint64_t* nseg,
             int nthreads)
{
    or_tree t;
    int st = setup_tree(&t, keys, levels, n, extent);
    if (st != OR_OK) return st;
    if (S < 1 || S > 64 || nd < 1 || n_src < 0) return OR_ERR_ARG;
    job_t jb;
    memset(&jb, 0, sizeof jb);
    jb.tree = &t; jb.dens = dens; jb.S = S; jb.src = src; jb.dirs = dirs; jb.nd = nd;
    jb.cap = step_cap(&t); jb.cols = cols; jb.hash = hash; jb.nseg = nseg;
    if (cols && !dens) return OR_ERR_ARG;
    return run_threads(&jb, n_src, nthreads, n);
}

/* Gradient of sum_{s,q,k} g[s,q,k] I(s,q,k) with respect to dens:
 * grad[j,k] += sum over rays crossing j of g[s,q,k] * ds (the transpose of
 * the forward map; not in the paper).  grad is ACCUMULATED into. */
int or_adjoint(const uint64_t* keys, const uint8_t* levels, int64_t n, const int32_t* extent,
               int S, const double* src, int64_t n_src, const double* dirs, int nd,
               const double* g, double* grad, int nthreads)
{
    or_tree t;
    int st = setup_tree(&t, keys, levels, n, extent);
    if (st != OR_OK) return st;
    if (S < 1 || S > 64 || nd < 1 || n_src < 0 || !g || !grad) return OR_ERR_ARG;
    job_t jb;
    memset(&jb, 0, sizeof jb);
    jb.tree = &t; jb.S = S; jb.src = src; jb.dirs = dirs; jb.nd = nd;
    jb.cap = step_cap(&t); jb.g = g; jb.grad = grad;
    return run_threads(&jb, n_src, nthreads, n);
}

typedef struct {
    int64_t* leaf;
    double* ds;
    int64_t cap, count;
} path_ctx;

static void visit_path(void* vctx, int64_t j, double ds)
{
    path_ctx* p = (path_ctx*)vctx;
    if (p->count < p->cap) {
        p->leaf[p->count] = j;
        p->ds[p->count] = ds;
    }
    p->count++;
}

/* The full (leaf, ds) sequence of one ray.  Returns the segment count (which
 * may exceed max_out; only the first max_out are stored) or -status. */
int64_t or_trace_path(const uint64_t* keys, const uint8_t* levels, int64_t n, const int32_t* extent,
                      const double* src, const double* dir, int64_t* leaf, double* ds,
                      int64_t max_out)
{
    or_tree t;
    int st = setup_tree(&t, keys, levels, n, extent);
    if (st != OR_OK) return -st;
    path_ctx p = {leaf, ds, max_out, 0};
    st = walk(&t, src, dir, step_cap(&t), visit_path, &p, NULL, NULL);
    if (st != OR_OK) return -st;
    return p.count;
}
