/*
 * rt_api.h - C ABI of the GB300 column-density tracer.
 *
 * The library computes, for every source point p and every HEALPix direction
 * q, the per-species column densities I(p,q,k) = sum_j n_k[j] * r_cell,j
 * (arXiv 2605.09882, Sec. 2.2, equation for I(p,q)) by reverse ray tracing
 * through a leaf-only linear octree: a DDA walk from cell boundary to cell
 * boundary, a Morton-code lookup of the next leaf in the sorted key array
 * (Sec. 2.2.1) and the slab method for each chord r_cell = t_out - t_in
 * (Sec. 2.2.2).  The adjoint (the transpose of that linear map) is an
 * addition of this library; the paper has no gradient.
 *
 * Conventions shared by every entry point:
 *  - Domain: the unit cube [0,1)^3, or the box [0, extent_b * 2^-21) when an
 *    extent is given.  Integer positions use the depth-21 lattice.
 *  - Octree: n_leaves keys (uint64) sorted strictly ascending and levels
 *    (uint8, 0..21).  Leaf j covers the Morton interval
 *    [key_j, key_j + 8^(21 - level_j)); key = interleave(x, y, z) of its
 *    depth-21 integer corner with x in bit 3b, y in bit 3b+1, z in bit 3b+2.
 *    The leaves must tile the domain box exactly.
 *  - Densities: [n_leaves][n_species] row-major, species fastest, RT_F32 or
 *    RT_F64.
 *  - Sources: float64 [n_src][3].  Each coordinate is truncated to the 2^-53
 *    lattice (a move below 1.2e-16 box lengths) so that every face-minus-
 *    source difference is exact in FP64.
 *  - Directions: the 12 * nside^2 HEALPix pixel centres in RING order
 *    (nside a power of two, 1..1024), as returned by rt_healpix_dirs.
 *  - Output columns: [n_src][12 * nside^2][n_species], species fastest, in
 *    units of (density) x (box length).
 *  - Pointers named d_* are device memory owned by the caller; h_* are host
 *    memory owned by the caller.  Nothing is freed or retained by a call except
 *    where stated.
 *  - Streams: every device operation is enqueued on `stream` (a cudaStream_t;
 *    NULL = legacy default stream) and returns before it completes.  Argument
 *    errors are returned synchronously.  Faults found by a kernel (a source
 *    outside the domain, a step cap reached, a failed lookup) are recorded in
 *    the octree's status word, read by rt_get_stats.
 *  - Threads: calls that share one rt_octree must be ordered on one stream;
 *    the handle holds the work-queue counter and the statistics.
 */
#ifndef RT_API_H
#define RT_API_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes returned by every int-valued entry point. */
enum rt_status {
    RT_OK = 0,
    RT_ERR_ARG = 1,             /* bad argument (null pointer, size, level > 21, bad nside, ...) */
    RT_ERR_UNSORTED = 2,        /* keys not strictly ascending */
    RT_ERR_MISALIGNED = 3,      /* key not a multiple of 8^(21 - level), or bit 63 set */
    RT_ERR_OVERLAP_OR_GAP = 4,  /* leaves overlap, leave the domain box, or leave a gap */
    RT_ERR_SOURCE_OUTSIDE = 5,  /* a source coordinate is not finite or outside the domain */
    RT_ERR_STEP_LIMIT = 6,      /* a ray reached the step cap (never for a valid octree) */
    RT_ERR_NONFINITE = 7,       /* a density is NaN, infinite or negative */
    RT_ERR_CUDA = 8,            /* a CUDA runtime call failed; see rt_last_error */
    RT_ERR_OOM = 9,             /* device allocation failed */
    RT_ERR_LOOKUP_MISS = 10     /* a walked position matched no leaf (never for a valid octree) */
};

enum rt_dtype { RT_F32 = 0, RT_F64 = 1 };

/* Arithmetic of the walk and of the columns.
 *  RT_MODE_FP64: every exit time, segment and column in IEEE FP64 without
 *    contraction; columns are bitwise those of the plain FP64 definition.
 *  RT_MODE_F32_KAHAN: exit-axis and next-leaf decisions certified equal to the
 *    FP64 ones (FP32 with an error bound, FP64 only for near-ties), segment
 *    lengths from double-float times, columns in FP32 with Kahan compensation.
 *  Visited-leaf sequences are identical in both modes. */
enum rt_mode { RT_MODE_FP64 = 0, RT_MODE_F32_KAHAN = 1 };

typedef struct rt_octree rt_octree; /* opaque */

/* Statistics and device status accumulated by the calls on one octree. */
typedef struct rt_stats {
    uint64_t rays;            /* rays traced */
    uint64_t segments;        /* (ray, leaf) pairs visited, ties counted once */
    uint64_t exit_fallbacks;  /* F32-Kahan steps whose exit axis needed FP64 */
    uint64_t lookup_fallbacks;/* F32-Kahan steps whose next leaf needed FP64 */
    int32_t status;           /* first device fault (rt_status), RT_OK if none */
    int32_t gathered;         /* 1 if an adjoint call took the leaf gather */
    int64_t fault_ray;        /* ray index (s * n_dirs + q) of that fault (for RT_ERR_NONFINITE
                                 the leaf index), -1 if none */
} rt_stats;

/* Builds the lookup structures of a leaf-only linear octree (Sec. 2.2.1:
 * leaves stored as compact arrays of Morton code and refinement level).
 *   d_keys, d_levels: device arrays of n_leaves entries, BORROWED: they must
 *     stay allocated and unchanged until rt_destroy_octree.
 *   n_leaves: 1 .. 2^32 - 1.
 *   h_extent: host int32[3], domain size in depth-21 cells per axis
 *     (1 .. 2^21), or NULL for the full cube (2^21 each).
 *   stream: the stream the checks and the table build are enqueued on.
 *   out: receives the handle on RT_OK, NULL otherwise.
 * Checks the octree on the device (sorted, aligned, tiling the box; fault
 * precedence ARG > MISALIGNED > UNSORTED > OVERLAP_OR_GAP), builds a coarse
 * Morton table over the top levels and synchronizes `stream` once to read the
 * validation result.  The handle owns the table and a small scratch block. */
int rt_build_octree(const uint64_t* d_keys, const uint8_t* d_levels, int64_t n_leaves,
                    const int32_t* h_extent, void* stream, rt_octree** out);

/* Frees a handle and what it owns (not the borrowed keys and levels).
 * Synchronizes the device first.  NULL is ignored. */
void rt_destroy_octree(rt_octree* tree);

/* HEALPix pixel centres in RING order (the paper's N_rays = 12 * 4^l
 * directions, Sec. 2), Gorski et al. 2005 ring equations, evaluated on the
 * host.  h_out: host float64 [12 * nside^2][3].  Host-only; needs no GPU. */
int rt_healpix_dirs(int nside, double* h_out);

/* Forward trace (Sec. 2.2, I(p,q) = sum_k f_k r_cell,k, for every source and
 * direction).
 *   d_src: float64 [n_src][3] inside the domain box.
 *   d_dens: [n_leaves][n_species] of dens_dtype; n_species 1..8.  The
 *     densities are checked on the device first (one read of the array): a
 *     NaN, infinite or negative value sets RT_ERR_NONFINITE in the status
 *     word, with the index of its leaf as the fault position; the columns are
 *     still computed from the values as given.  rt_trace_epilogue,
 *     rt_trace_columns_chunked and rt_trace_columns_host (which then returns
 *     the code) check the same way; a batch does not.
 *   mode: rt_mode.  d_out: [n_src][12 nside^2][n_species], float32 for
 *     RT_MODE_F32_KAHAN, float64 for RT_MODE_FP64; fully written (rays from a
 *     source outside the domain get zeros and set RT_ERR_SOURCE_OUTSIDE).
 * The first call for a given nside on a device uploads its direction table
 * (an allocation); make that call outside CUDA graph capture. */
int rt_trace_columns(const rt_octree* tree, const double* d_src, int64_t n_src, int nside,
                     const void* d_dens, int n_species, int dens_dtype, int mode,
                     void* d_out, void* stream);

/* Forward trace (Sec. 2.2) end to end from HOST buffers: copies the octree,
 * densities and sources to the device, indexes the octree (as
 * rt_build_octree), traces, and copies the columns back; returns when h_out
 * is written.
 *   h_keys, h_levels, n_leaves, h_extent: as rt_build_octree, in host memory.
 *   h_src: host float64 [n_src][3].  h_dens: host [n_leaves][n_species] of
 *     dens_dtype.  h_out: host [n_src][12 nside^2][n_species], float32 for
 *     RT_MODE_F32_KAHAN, float64 for RT_MODE_FP64.
 *   chunk_src: sources per pipeline chunk (0: about n_src / 8); rounded up to
 *     a multiple of 32 and to at most 1024 chunks.  Chunk c's source copy,
 *     trace and column copy run on separate streams, so copies overlap the
 *     traces of neighbouring chunks; page-locked host buffers (cudaHostAlloc
 *     or cudaHostRegister) let the copies run as DMA.
 *   h_stats: optional; receives the trace's statistics.
 *   stream: the stream the traces run on (two more are created inside).
 * Device buffers (the octree, densities, all sources and two column
 * chunks), the two copy streams and the events are kept per device between
 * calls and grow on demand; rt_trace_columns_host_release frees them.  Calls
 * are serialized by a process-wide lock.  Returns RT_ERR_OOM if the buffers
 * do not fit, the code of the first faulting ray if a ray faulted (its
 * columns are zero), and the rt_build_octree codes for a malformed octree. */
int rt_trace_columns_host(const uint64_t* h_keys, const uint8_t* h_levels, int64_t n_leaves,
                          const int32_t* h_extent, const double* h_src, int64_t n_src, int nside,
                          const void* h_dens, int n_species, int dens_dtype, int mode, void* h_out,
                          int64_t chunk_src, rt_stats* h_stats, void* stream);

/* Frees the device buffers, streams and events rt_trace_columns_host keeps,
 * on every device it used (waiting for their copies first). */
void rt_trace_columns_host_release(void);

/* Per-source quantities computed inside the trace, so that the columns are
 * never written (the paper's 3D-PDR coupling, Sec. 2.4, and its accuracy
 * test, Sec. 3).  Each ray's combined column is N = sum_k weights[k] I_k, a
 * linear combination of its species columns (as in the optical depth's
 * [n_j g_i / g_j - n_i] integrand).
 *   RT_EPI_AV_EFF:      out[p] = -(1/gamma) ln( (1/N_rays) sum_q exp(-gamma a N_pq) )
 *                       (A_V,eff; a = A_V0 x box length in the columns' unit)
 *   RT_EPI_BETA:        out[p] = (1/N_rays) sum_q (1 - exp(-tau_pq)) / tau_pq,
 *                       tau_pq = c_p N_pq, c_p = d_coef[p] (or a if d_coef is NULL);
 *                       a term is 1 at tau = 0 (escape probability)
 *   RT_EPI_ATTENUATION: out[p][q] = exp(-a N_pq) (attenuation I / I_0)
 * The FP64 arithmetic of the epilogue uses the CUDA math library's exp and
 * expm1. */
enum rt_epilogue_kind { RT_EPI_AV_EFF = 1, RT_EPI_BETA = 2, RT_EPI_ATTENUATION = 3 };

typedef struct rt_epilogue {
    int kind;                 /* rt_epilogue_kind */
    int reserved;
    double weights[8];        /* species weights; entries past n_species ignored */
    double a;                 /* extinction / opacity per unit combined column */
    double gamma;             /* A_V,eff only (3.02 in the paper) */
    const double* d_coef;     /* beta only: per-source c_p [n_src] or NULL */
} rt_epilogue;

/* Traces like rt_trace_columns and writes only the epilogue:
 *   d_out: float64 [n_src] (A_V,eff, beta) or [n_src][12 nside^2]
 *   (attenuation).  Per-source sums use FP64 atomics across the directions,
 *   so their order is not fixed. */
int rt_trace_epilogue(const rt_octree* tree, const double* d_src, int64_t n_src, int nside,
                      const void* d_dens, int n_species, int dens_dtype, int mode,
                      const rt_epilogue* h_epi, double* d_out, void* stream);

/* Forward trace over a chunked contribution grid (Alg. 1: the contribution
 * grid is traversed one chunk at a time, each ray adds the partial integral
 * of the part of its path inside the chunk, and sources outside the cloud get
 * I(p, q) = 0).  The chunks are n_chunks contiguous ranges of about equal size
 * of the Morton-sorted leaf array; the densities of one chunk at a time are
 * read, so h_dens may live in HOST memory (page-locked for overlapped copies):
 * chunk k is copied into one of two device buffers while chunk k - 1 is
 * traced.  A device pointer is read in place.  Every ray keeps its walk state
 * and running column sums between chunks (about 48 + 4 n_species bytes of
 * device scratch per ray, allocated and freed by the call), stops when its
 * next leaf lies in another chunk and resumes there, and the chunks are swept
 * in order until every ray has left the domain, so paths and columns are bit
 * for bit those of rt_trace_columns (which this call reproduces with the
 * general-octree walk).
 *   dens: [n_leaves][n_species] of dens_dtype, host or device memory, 16-byte
 *     aligned.
 *   d_mask: device uint8 [n_src]; a source with mask 0 is outside the cloud
 *     and gets zero columns without tracing; NULL traces every source.
 *   n_chunks: 1 .. n_leaves.
 *   d_out: as rt_trace_columns.  d_nseg (uint32 [n_src][n_dirs]) and d_hash
 *     (uint64, as rt_trace_paths) are optional path fingerprints (zero for a
 *     masked source).
 * Synchronizes `stream` once per sweep over the chunks and at the end. */
int rt_trace_columns_chunked(const rt_octree* tree, const double* d_src, int64_t n_src, int nside,
                             const void* dens, int n_species, int dens_dtype, int mode,
                             const uint8_t* d_mask, int n_chunks, void* d_out, uint32_t* d_nseg,
                             uint64_t* d_hash, void* stream);

/* Per-ray path fingerprints: the number of segments and the hash
 * h <- (h XOR leaf) * 0x100000001b3 (h0 = 0xcbf29ce484222325) over the
 * visited leaf indices in walk order, for every ray of the walk that
 * rt_trace_columns does in the same mode.  d_nseg: uint32 [n_src][n_dirs];
 * d_hash: uint64 [n_src][n_dirs]; either may be NULL. */
int rt_trace_paths(const rt_octree* tree, const double* d_src, int64_t n_src, int nside,
                   int mode, uint32_t* d_nseg, uint64_t* d_hash, void* stream);

/* Adjoint of rt_trace_columns with respect to the densities (not in the
 * paper): d_grad_dens[j,k] += sum over rays (s,q) crossing leaf j of
 * d_grad_out[s,q,k] * ds(s,q,j).
 *   d_grad_out: same shape as the forward output; float32 for
 *     RT_MODE_F32_KAHAN, float64 for RT_MODE_FP64.
 *   d_grad_dens: float64 [n_leaves][n_species], ACCUMULATED into (the caller
 *     zeroes it).
 *   path_policy:
 *     0 = automatic.  On a full cube of equal-level leaves with one source per
 *       leaf, source s in leaf s, all at the same offset inside their leaf
 *       (leaf centres, for example), every ray of a direction takes the same
 *       steps and segment lengths, and each leaf's gradient is gathered by one
 *       thread from per-direction step tables: no atomics, and the same bits
 *       on every run (F32-Kahan: FP32 products with Kahan compensation, added
 *       once per leaf in FP64).  The sources are checked on the device; any
 *       other call (and this one if the check fails) recomputes the paths
 *       and scatters with FP64 atomics, whose summation order is not fixed.
 *       The first gather on a handle allocates its step tables (kept by the
 *       handle and grown when a later call needs more).
 *     1 = recompute the paths while scattering (FP64 atomics).
 *     2 = record the paths (rt_record_paths), scatter from the record and
 *       free it (synchronizes `stream`, resets the octree's statistics).  To
 *       reuse a record, call rt_record_paths once and rt_paths_adjoint /
 *       rt_paths_columns many times.
 *     3 = deterministic: the leaf gather where it applies (the call then
 *       synchronizes `stream` to learn whether the sources had its layout),
 *       otherwise a record, rt_paths_adjoint_ordered over it, and the record
 *       freed; the same bits on every run. */
int rt_trace_columns_adjoint(const rt_octree* tree, const double* d_src, int64_t n_src,
                             int nside, const void* d_grad_out, int n_species, int mode,
                             double* d_grad_dens, int path_policy, void* stream);

/* Builds the contribution grid from a uniform source grid (Sec. 2.2.1:
 * cells split recursively into eight children down to a maximum depth;
 * Sec. 2.4: a cell splits only if n_max >= n_pdr and
 * (n_max - n_min) / n_max >= rel_var, evaluated in FP64 exactly as written).
 * A leaf's value is the mean of the source cells it covers.
 *   d_nref: [8^level] refinement density (nref_dtype), the source grid of
 *     2^level cells per axis in Morton order (cell i = interleave(x, y, z)
 *     at that level); level 1..10.
 *   d_vals: [8^level][n_species] values averaged into the leaves (vals_dtype,
 *     Morton order), or NULL to average d_nref itself (n_species = 1).
 *   max_level: deepest leaf level (<= level; also the minimum cell size).
 *   d_keys, d_levels, d_leaf_vals ([capacity][n_species] of vals_dtype):
 *     outputs, caller-allocated with capacity >= 8^level; the leaves come out
 *     sorted by key, ready for rt_build_octree.
 *   h_n_leaves: receives the number of leaves (the call synchronizes).
 * Allocates and frees its own scratch (about 1.2 x 8^(level-1) cells of
 * pyramid). */
int rt_build_amr(const void* d_nref, int nref_dtype, const void* d_vals, int n_species, int vals_dtype,
                 int level, double n_pdr, double rel_var, int max_level, uint64_t* d_keys,
                 uint8_t* d_levels, void* d_leaf_vals, int64_t capacity, int64_t* h_n_leaves,
                 void* stream);

/* ---------------------------------------------------------- recorded paths
 * The (leaf, ds) sequence of every ray, recorded once so that the forward
 * columns and the adjoint can be evaluated again without walking (an
 * addition of this library).  Rays are stored 32 at a time as the walk visits
 * them: segment k of lane i of group g at slot off[g] + 32 k + i; a group
 * holds 32 x its longest path.  About 8 bytes per slot in F32-Kahan mode (a
 * uint32 leaf and a float32 ds), 12 in FP64 mode (float64 ds). */
typedef struct rt_paths rt_paths; /* opaque */

/* Walks every ray twice on `stream`: once to count the segments (then one
 * synchronization to size the record) and once to write it.  Resets the
 * octree's statistics.  RT_ERR_OOM if the record does not fit. */
int rt_record_paths(const rt_octree* tree, const double* d_src, int64_t n_src, int nside, int mode,
                    void* stream, rt_paths** out);

/* Rays, segments and device bytes of a record. */
int rt_paths_info(const rt_paths* paths, int64_t* n_rays, int64_t* n_segments, int64_t* bytes);

/* Columns from a record, in the record's mode; the same arithmetic in the
 * same order as rt_trace_columns, hence the same bits. */
int rt_paths_columns(const rt_paths* paths, const void* d_dens, int n_species, int dens_dtype,
                     void* d_out, void* stream);

/* Adjoint from a record: d_grad_dens[j,k] += sum g[s,q,k] ds (accumulated). */
int rt_paths_adjoint(const rt_paths* paths, const void* d_grad_out, int n_species,
                     double* d_grad_dens, void* stream);

/* Adjoint from a record like rt_paths_adjoint, but each leaf's terms are
 * summed by one thread in the record's order (rays as traced, segments in
 * walk order), FP64 products and sums: the same bits on every run, whatever
 * the geometry.  The first call sorts the record's slots by leaf (a stable
 * radix sort; about 8 bytes per slot plus 8 per leaf, kept by the record;
 * synchronizes `stream`); RT_ERR_ARG for a record of 2^32 or more slots. */
int rt_paths_adjoint_ordered(rt_paths* paths, const void* d_grad_out, int n_species,
                             double* d_grad_dens, void* stream);

/* Frees a record (synchronizes the device first).  NULL is ignored. */
void rt_destroy_paths(rt_paths* paths);

/* Copies the statistics of `tree` into *h_out after synchronizing `stream`. */
int rt_get_stats(const rt_octree* tree, rt_stats* h_out, void* stream);

/* Zeroes the statistics and the status word (enqueued on `stream`). */
int rt_reset_stats(rt_octree* tree, void* stream);

/* Test knob: per-ray step cap (0 restores the geometric bound 3 * 2^lmax + 3,
 * which no valid walk can reach).  A ray that reaches the cap stops and sets
 * RT_ERR_STEP_LIMIT instead of looping. */
int rt_set_step_cap(rt_octree* tree, int64_t cap);

/* Launch shape of the persistent trace kernels: threads per block (a
 * multiple of 32 in 32..256; 0 = default 256), resident blocks per SM (0 =
 * as many as fit) and 32-ray groups a warp takes per work-queue pop (1..64;
 * 0 = default 4).  Applies to later calls in this process.  The F32-Kahan
 * forward of rt_trace_columns on a full cube of equal-level leaves with FP32
 * densities of 1, 2, 4 or 8 species walks two rays per lane: its warps pop
 * one 64-source block and one direction group at a time, whatever
 * groups_per_pop says, and at most 3 of its blocks fit on an SM. */
int rt_set_launch(int threads_per_block, int blocks_per_sm, int groups_per_pop);

/* Caps the coarse-table level of later rt_build_octree calls (-1, the
 * default: no cap; 0..10).  A shallower table leaves more lookups to the
 * per-thread binary search of the sorted keys inside a coarse cell that holds
 * leaves of several levels; the results are the same. */
int rt_set_table_cap(int max_level);

/* Lookup choice: 1 (default) lets a full cube of equal-level leaves use the
 * O(1) Morton index; 0 forces the coarse table and key search even then
 * (both give identical results). */
int rt_set_lookup(rt_octree* tree, int use_uniform_index);

/* Number of leaves and the deepest level of a handle (host values). */
int rt_octree_info(const rt_octree* tree, int64_t* n_leaves, int* max_level, int* uniform_level);

/* Forward trace that allocates no device memory (the paper has no
 * counterpart; this is an interface addition).  It computes what
 * rt_trace_columns computes, on a raw octree instead of a handle, for callers
 * that cannot call cudaMalloc: an application whose own pool owns all device
 * memory, or code that must not allocate or free because cudaMalloc and
 * cudaFree can synchronize the whole device.
 *   d_keys, d_levels, n_leaves, h_extent: as for rt_build_octree; the octree
 *     is NOT validated here and must be valid (for example checked once with
 *     rt_build_octree wherever allocation is allowed).
 *   max_level: the deepest leaf level (sets the step cap; a full cube of
 *     leaves all at this level uses the O(1) Morton index, any other octree a
 *     binary search of all keys).
 *   nside: 1, 2, 4 or 8 only; the rest as for rt_trace_columns.
 *   h_stats: NULL, or host memory that receives this call's statistics and
 *     status; then the call synchronizes `stream`.
 * The launch shape (rt_set_launch) and the ray order are those of
 * rt_trace_columns's one-ray-per-lane kernel (where rt_trace_columns walks
 * two rays per lane, the columns are bitwise the same).  Each call zeroes the statistics and copies the lookup
 * entry and the direction table from host tables that are computed once per
 * nside and never change afterwards.
 * All scratch (work-queue counter, statistics, status word, direction table)
 * lives in one file-scope device array of about 74 KiB that every GPU which
 * loads the library holds until exit.  The first call on a device looks up
 * that array's address with cudaGetSymbolAddress (a runtime call that
 * allocates nothing).  Every call reuses the array and re-zeroes the
 * counters it needs, so calls that overlap on the GPU (on different streams
 * or threads) race and must be ordered by the caller. */
int rt_trace_columns_noalloc(const uint64_t* d_keys, const uint8_t* d_levels, int64_t n_leaves,
                             const int32_t* h_extent, int max_level, const double* d_src,
                             int64_t n_src, int nside, const void* d_dens, int n_species,
                             int dens_dtype, int mode, void* d_out, rt_stats* h_stats,
                             void* stream);

/* ---------------------------------------------------------------- batches
 * Many independent clouds (octrees of uneven size and depth) traced in one
 * persistent launch over a single work queue, replayed as a CUDA graph
 * (a memset node that resets the queue, then the kernel node).  An addition
 * of this library; the paper traces one cloud with MPI/OpenMP (Alg. 1). */
typedef struct rt_cloud_desc {
    const rt_octree* tree;   /* built with rt_build_octree on this device */
    const double* d_src;     /* float64 [n_src][3] */
    int64_t n_src;
    int nside;               /* power of two, 1..1024 */
    int n_species;           /* 1..8 */
    const void* d_dens;      /* [n_leaves][n_species], dens_dtype, 16-byte aligned */
    int dens_dtype;
    int reserved;
    void* d_out;             /* [n_src][12 nside^2][n_species], f32 (F32-Kahan) or f64 (FP64) */
} rt_cloud_desc;

typedef struct rt_batch rt_batch; /* opaque */

/* Uploads the descriptors of n_clouds clouds (copied; the pointers inside
 * must stay valid while the batch is used) and allocates the batch's queue
 * and statistics.  Synchronous. */
int rt_batch_create(const rt_cloud_desc* h_desc, int n_clouds, int mode, rt_batch** out);

/* Traces every ray of every cloud in one launch, enqueued on `stream` as a
 * CUDA graph; the graph is built on the first call and rebuilt only when the
 * launch shape (rt_set_launch) changes.  Outputs as rt_trace_columns. */
int rt_batch_launch(rt_batch* batch, void* stream);

/* Statistics of the batch (synchronizes `stream`) / zeroes them (enqueued). */
int rt_batch_stats(const rt_batch* batch, rt_stats* h_out, void* stream);
int rt_batch_reset_stats(rt_batch* batch, void* stream);

/* Frees the batch (synchronizes the device first).  NULL is ignored. */
void rt_batch_destroy(rt_batch* batch);

/* Picks the launch shape of `batch` by timing: threads per block in
 * {64, 128, 256} x resident blocks per SM, then 32-ray groups per queue pop,
 * each measured with CUDA events over two launches on `stream`.  The best is
 * applied with rt_set_launch and, if cache_json is not NULL, stored there
 * keyed by (GPU name, SM count, mode, clouds, rays, max species); a later
 * call with a matching key applies the cached shape without timing.
 * h_best (optional): int[3] = {threads, blocks per SM, groups per pop};
 * h_rate (optional): segments/s of the best shape. */
int rt_batch_autotune(rt_batch* batch, const char* cache_json, int* h_best, double* h_rate, void* stream);

/* The batch calls in descriptor form (the object API above underneath).
 * rt_trace_batched traces the n_clouds clouds of h_desc in one persistent
 * launch replayed as a CUDA graph, enqueued on `stream`: the batch for a
 * descriptor set is built on its first call (synchronously, an allocation)
 * and kept, so later calls with the same descriptors (compared byte for
 * byte, and the same octree builds) and mode only replay it; another
 * descriptor set replaces it (the old batch is freed after a device
 * synchronization).  Outputs as rt_trace_columns.
 * rt_autotune tunes the launch shape on a temporary batch of h_desc (timed on
 * the legacy default stream) exactly as rt_batch_autotune does, caching in
 * cache_json (may be NULL), and applies it with rt_set_launch. */
int rt_trace_batched(const rt_cloud_desc* h_desc, int n_clouds, int mode, void* stream);
int rt_autotune(const rt_cloud_desc* h_desc, int n_clouds, int mode, const char* cache_json);

/* Message of the last failed call on this host thread ("" if none). */
const char* rt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RT_API_H */
