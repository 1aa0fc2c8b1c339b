// Host-side helpers shared by the library's translation units.
#pragma once

#include <string.h>

#include <algorithm>

#include "rt_internal.h"

namespace rt {
int set_error(int code, const char* msg);
int cuda_error(const char* where);
void clear_error();
// current launch shape (threads per block, blocks per SM cap, groups per pop)
void launch_shape(int* block, int* blocks_per_sm, int* groups_per_pop);
// device direction table of nside on device dev (uploaded on first use)
const DirConst* direction_table(int dev, int nside, int* status);
int sm_count_of(int dev);
// deepest coarse-table level rt_build_octree may choose (-1: no cap)
int table_level_cap();
// enqueues the density check (RT_ERR_NONFINITE into st for a NaN, infinite or
// negative value; leaf index base + i / S as the fault position)
int check_densities(const void* dens, long long n_leaves, int S, int f64, long long base, DevStats* st,
                    cudaStream_t s);
// rt_trace_columns with the density check optional (the host-buffer call
// checks the whole array once, not per source chunk)
int trace_columns_impl(const rt_octree* t, const double* d_src, int64_t n_src, int nside, const void* d_dens,
                       int n_species, int dens_dtype, int mode, void* d_out, void* stream, bool check);
// argument checks and TraceArgs of the single-octree trace entry points
int prepare_trace(const rt_octree* t, const double* d_src, int64_t n_src, int nside, int S, int mode,
                  TraceArgs& a, const char* who);
// leaf-gather adjoint (rt_gather.cu): whether the call's shape admits it, and
// its launch (source check, step tables, gather) on stream s
bool gather_applies(const rt_octree* t, const TraceArgs& a);
int launch_adjoint_gather(rt_octree* t, const TraceArgs& a, int mode, cudaStream_t s);
}  // namespace rt
