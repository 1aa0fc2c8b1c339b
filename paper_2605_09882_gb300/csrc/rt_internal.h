// Internal types of the tracer library (host and device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rt_api.h"

namespace rt {

constexpr int kDepth = 21;          // anchor depth of the Morton lattice
constexpr int kMaxSpecies = 8;
constexpr int kBaseTableLevel = 7;  // coarse table level for every tree (8^7 = 2M entries at most)
constexpr int kMaxTableLevel = 10;  // deepest coarse table (the lookup's cell index holds 30 bits)
constexpr int kCodeHole = 62;       // coarse cell outside the domain box
constexpr int kCodeMixed = 63;      // coarse cell with leaves of several levels

// Device view of an octree handle.
struct DevTree {
    const uint64_t* keys;
    const uint8_t* levels;
    const uint64_t* table;   // [8^T] entries: (first leaf << 6) | code
    int64_t n;
    uint32_t ext[3];
    int T;                   // coarse table level
    int uniform_level;       // >= 0: full cube of leaves all at this level (O(1) index)
    int lmax;
    int64_t step_cap;
};

// Per-direction constants, computed on the host from the HEALPix table.
struct DirConst {
    double m[3];
    double inv[3];   // 1 / m_b (0 where m_b == 0)
    float m32[3];    // m_b rounded to float
    float ih[3];     // inv_b = ih + il (float-float split)
    float il[3];
    int flags;       // bit b: m_b != 0; bit 3+b: m_b > 0; bits 6,7,8: |inv| equal for (0,1),(0,2),(1,2)
    int pad;
};

// Statistics block in device memory (one per octree handle).
struct DevStats {
    unsigned long long queue;      // work-queue counter (reset before every launch)
    unsigned long long rays;
    unsigned long long segments;
    unsigned long long exit_fb;
    unsigned long long lookup_fb;
    int status;
    int gather_off;                // adjoint: nonzero when the leaf-gather form does not apply
    long long fault_ray;
    int gathered;                  // set when a leaf-gather adjoint ran
    int pad;
};

struct TraceArgs {
    DevTree t;
    const DirConst* dirs;
    int nd;
    const double* src;
    int64_t n_src;
    int64_t n_src_pad;       // n_src rounded up to a multiple of 32
    const void* dens;        // forward: densities; adjoint: unused
    int dens_f64;
    int S;
    void* out;               // forward: columns; adjoint: grad_dens (double)
    const void* gin;         // adjoint: d_grad_out
    uint32_t* nseg;          // path fingerprints (optional)
    uint64_t* hash;
    DevStats* st;
    int batch;               // 32-ray groups per queue pop
    int layout;              // ray order: 0 direction-major (sources padded to 32), 1 source-major
    int dgroup;              // layout 0: directions per group (a power of two dividing nd; <= 1: one)
    int pair;                // forward on a uniform cube: two rays per lane (k_trace_pair); n_src_pad % 64 == 0
    // path recording (KIND 3): per 32-ray group, segment k of lane i is entry
    // rec_off[g] + 32 k + i of rec_leaf / rec_ds
    const long long* rec_off;
    uint32_t* rec_leaf;
    void* rec_ds;
    // fused epilogue (KIND 4): combined column N = sum_k epi_w[k] I_k per ray
    int epi_kind;
    double epi_w[kMaxSpecies];
    double epi_a, epi_gamma;
    const double* epi_coef;
    // adjoint scatter: runs only if *gate is nonzero (the leaf-gather form did
    // not apply to this call); NULL: always runs
    const int* gate;
};

// Ray order of a trace: direction-major (32 neighbouring sources share a
// direction in a warp) unless there are too few sources to fill a warp, then
// source-major (a warp walks 32 directions of the same source).
inline int ray_layout(int64_t n_src) { return n_src < 32 ? 1 : 0; }

// Launch helpers (defined in the .cu files).
cudaError_t launch_forward(const TraceArgs& a, int mode, int block, int grid, cudaStream_t s);
cudaError_t launch_paths(const TraceArgs& a, int mode, int block, int grid, cudaStream_t s);
cudaError_t launch_adjoint(const TraceArgs& a, int mode, int block, int grid, cudaStream_t s);
cudaError_t launch_epilogue(const TraceArgs& a, int mode, int block, int grid, cudaStream_t s);
int occupancy_epi(int mode, int S, bool uniform, int block);
int occupancy_fwd(int kind, int mode, int S, bool uniform, int block);
int occupancy_pair(int S, int block);
int occupancy_adj(int mode, int S, bool uniform, int block);

}  // namespace rt

// Host-side octree handle.
struct rt_octree {
    rt::DevTree dev;
    rt::DevStats* st;        // device
    uint64_t* table;         // device, owned
    int device;
    int uniform_allowed;     // 0: use the coarse table even for a uniform grid
    int64_t default_cap;
    void* adj_tab;           // device, owned: step tables of the leaf-gather adjoint (grown on demand)
    size_t adj_tab_bytes;
    unsigned long long gen;  // build number, unique in the process (a reused address is another tree)
};
