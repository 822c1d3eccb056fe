// fq_launch.h -- host-side table of kernel launchers, one entry per
// (address width, amplitude type, Hamiltonian kind).
#pragma once

#include <cuda_runtime.h>

#include "fq_shared.h"

namespace fq {

struct KernelSet {
    size_t key_bytes, amp_bytes, spawn_bytes;
    size_t spawn_key_stride, spawn_val_stride;  // spawn buffer bytes per entry (SpawnIO)
    size_t slot_bytes;  // one merge table slot: key, sum, list entry
    void (*spawn)(const LaunchCfg&, const RunDesc*, const unsigned*, unsigned, cudaStream_t);
    void (*merge)(const LaunchCfg&, const RunDesc*, const unsigned*, unsigned, cudaStream_t);
    cudaError_t (*prepare)(size_t merge_smem);
    int (*spawn_occupancy)(int var);               // resident blocks per SM
    int (*merge_occupancy)(int ann, int var, size_t smem);
    size_t (*merge_smem)(int ann, int wpb, unsigned slots);  // dynamic shared memory of a launch
    size_t (*sort_ws_bytes)(unsigned elems);                 // one sort workspace
    void (*scratch_init)(unsigned char* scratch, unsigned slots, unsigned nwarps, cudaStream_t);
    void (*seed)(const RunDesc*, const void*, const double*, size_t, cudaStream_t);
    void (*gather_vec)(const void* keys, const void* amps, unsigned cap, const unsigned* cnt,
                       const unsigned* off, unsigned B, void* okeys, double* ovals,
                       const unsigned* segs, cudaStream_t);
    void (*lookup)(const RunDesc* d, const void* keys, size_t n, double* out, cudaStream_t);
    void (*restride)(const void* ok, const void* oa, unsigned oc, const unsigned* cnt, unsigned B,
                     void* nk, void* na, unsigned nc, cudaStream_t);
    void (*gather_spawns)(const void* keys, const void* vals, unsigned cap, unsigned Cp,
                          const unsigned* cnt, const unsigned* off, unsigned B, void* okeys,
                          double* ovals, cudaStream_t);
    void (*column)(const ModelParams&, const void* key, void* dest, double* val, unsigned cap,
                   double* diag, unsigned* m, cudaStream_t);
    void (*ref_count)(const ModelParams&, const void* refs, int n, unsigned* m, cudaStream_t);
    void (*ref_terms)(const ModelParams&, const void* refs, const double* y, int n,
                      const unsigned* off, void* tkeys, double* th, double* tv, unsigned* tseg,
                      int log2B, cudaStream_t);
    // replica overlaps: `grid` blocks of `wpb` warps, then the row
    void (*overlap)(const RunDesc* runs, const OverlapDesc* od, int grid, int wpb,
                    unsigned table, cudaStream_t);
    size_t overlap_slot_bytes;  // one slot of an overlap table: key, FP64 amplitude, list entry
    cudaError_t (*prepare_overlap)(size_t smem);
    // Gram-Schmidt of run k: dot products, coefficients, axpy (grid x wpb warps)
    void (*gs)(const RunDesc* runs, const GsDesc* gs, int k, int grid, int wpb, unsigned table,
               cudaStream_t);
    cudaError_t (*prepare_gs)(size_t smem);
    size_t gs_slot_bytes;  // one slot of the axpy table: key, value, list entry, flag
};

// kw = 64-bit words per address (1 or 2), amp = FQ_AMP_*, kind = FQ_KIND_*
const KernelSet* kernel_set(int kw, int amp, int kind);

// warps per block of the compiled kernel variants (fq_kernels.cuh, Var<V>)
inline int variant_wpb(int var) { return var == 0 ? 8 : 4; }
constexpr int kKernelVariants = 3;

void launch_shift(const RunDesc* runs, int nruns, cudaStream_t s);

}  // namespace fq
