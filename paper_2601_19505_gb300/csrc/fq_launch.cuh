// fq_launch.cuh -- launcher definitions for one (address, amplitude) pair;
// included by the fq_inst_*.cu translation units only.
#pragma once

#include "fq_kernels.cuh"
#include "fq_launch.h"

namespace fq {

template <class K, int AMP, int KIND> struct Launch {
    typedef typename AmpT<AMP>::A A;
    typedef typename AmpT<AMP>::S S;
    typedef typename AmpT<AMP>::ACC ACC;

    static constexpr size_t spawn_smem(int wpb) {
        return (size_t)wpb * SpawnSmem<K, AMP, 128, KIND>::bytes;
    }
    template <int V> static void spawn_v(const LaunchCfg& c, const RunDesc* d, const unsigned* sr,
                                         unsigned G, cudaStream_t s) {
        constexpr int W = Var<V>::WPB;
        k_spawn<K, AMP, KIND, V, 4><<<c.spawn_grid, W * 32, spawn_smem(W), s>>>(d, sr, G);
    }
    static void spawn(const LaunchCfg& c, const RunDesc* d, const unsigned* sr, unsigned G,
                      cudaStream_t s) {
        if (c.spawn_var == 1) spawn_v<1>(c, d, sr, G, s);
        else if (c.spawn_var == 2) spawn_v<2>(c, d, sr, G, s);
        else spawn_v<0>(c, d, sr, G, s);
    }
    template <int V> static void merge_v(const LaunchCfg& c, const RunDesc* d, const unsigned* sr,
                                         unsigned G, cudaStream_t s) {
        constexpr int W = Var<V>::WPB;
        if (c.ann == FQ_ANN_SORT_ARM) {
            const size_t smem = (size_t)W * merge_warp_bytes<K, AMP, FQ_ANN_SORT_ARM>(c.slots);
            k_merge<K, AMP, KIND, V, FQ_ANN_SORT_ARM><<<c.merge_grid, W * 32, smem, s>>>(
                d, sr, G, c.slots, c.sort_scratch, c.sort_elems);
        } else {
            const size_t smem = (size_t)W * merge_warp_bytes<K, AMP, FQ_ANN_HASH_ARM>(c.slots);
            k_merge<K, AMP, KIND, V, FQ_ANN_HASH_ARM><<<c.merge_grid, W * 32, smem, s>>>(
                d, sr, G, c.slots, c.scratch, c.scratch_slots);
        }
    }
    static void merge(const LaunchCfg& c, const RunDesc* d, const unsigned* sr, unsigned G,
                      cudaStream_t s) {
        if (c.merge_var == 1) merge_v<1>(c, d, sr, G, s);
        else if (c.merge_var == 2) merge_v<2>(c, d, sr, G, s);
        else merge_v<0>(c, d, sr, G, s);
    }
    template <int V> static cudaError_t prepare_v(size_t smem) {
        cudaError_t e = cudaFuncSetAttribute(k_merge<K, AMP, KIND, V, FQ_ANN_HASH_ARM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_merge<K, AMP, KIND, V, FQ_ANN_SORT_ARM>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_spawn<K, AMP, KIND, V, 4>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)spawn_smem(Var<V>::WPB));
        return e;
    }
    static cudaError_t prepare(size_t smem) {
        cudaError_t e = prepare_v<0>(smem);
        if (e == cudaSuccess) e = prepare_v<1>(smem);
        if (e == cudaSuccess) e = prepare_v<2>(smem);
        return e;
    }
    static int spawn_occupancy(int var) {
        int n = 0;
        if (var == 1)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_spawn<K, AMP, KIND, 1, 4>, 128, spawn_smem(4));
        else if (var == 2)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_spawn<K, AMP, KIND, 2, 4>, 128, spawn_smem(4));
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_spawn<K, AMP, KIND, 0, 4>, 256, spawn_smem(8));
        return n;
    }
    template <int ANN> static int merge_occupancy_a(int var, size_t smem) {
        int n = 0;
        if (var == 1)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_merge<K, AMP, KIND, 1, ANN>, 128, smem);
        else if (var == 2)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_merge<K, AMP, KIND, 2, ANN>, 128, smem);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_merge<K, AMP, KIND, 0, ANN>, 256, smem);
        return n;
    }
    static int merge_occupancy(int ann, int var, size_t smem) {
        return ann == FQ_ANN_SORT_ARM ? merge_occupancy_a<FQ_ANN_SORT_ARM>(var, smem)
                                      : merge_occupancy_a<FQ_ANN_HASH_ARM>(var, smem);
    }
    static size_t merge_smem(int ann, int wpb, unsigned slots) {
        return (size_t)wpb * (ann == FQ_ANN_SORT_ARM
                                  ? merge_warp_bytes<K, AMP, FQ_ANN_SORT_ARM>(slots)
                                  : merge_warp_bytes<K, AMP, FQ_ANN_HASH_ARM>(slots));
    }
    static void scratch_init(unsigned char* scratch, unsigned slots, unsigned nwarps,
                             cudaStream_t s) {
        k_scratch_init<K, AMP><<<1024, 256, 0, s>>>(scratch, slots, nwarps);
    }
    static void seed(const RunDesc* d, const void* keys, const double* amps, size_t n,
                     cudaStream_t s) {
        if (!n) return;
        k_seed<K, AMP><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d, (const K*)keys, amps, n);
    }
    static void gather_vec(const void* keys, const void* amps, unsigned cap, const unsigned* cnt,
                           const unsigned* off, unsigned B, void* okeys, double* ovals,
                           const unsigned* segs, cudaStream_t s) {
        k_gather<K, A><<<B < 4096 ? B : 4096, 256, 0, s>>>((const K*)keys, (const A*)amps, cap, cnt,
                                                           off, B, (K*)okeys, ovals, segs);
    }
    static void restride(const void* ok, const void* oa, unsigned oc, const unsigned* cnt,
                         unsigned B, void* nk, void* na, unsigned nc, cudaStream_t s) {
        k_restride<K, A><<<B < 8192 ? B : 8192, 128, 0, s>>>((const K*)ok, (const A*)oa, oc, cnt, B,
                                                            (K*)nk, (A*)na, nc);
    }
    static void lookup(const RunDesc* d, const void* keys, size_t n, double* out, cudaStream_t s) {
        if (!n) return;
        k_lookup<K, AMP><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d, (const K*)keys, n, out);
    }
    static void gather_spawns(const void* keys, const void* vals, unsigned cap, unsigned Cp,
                              const unsigned* cnt, const unsigned* off, unsigned B, void* okeys,
                              double* ovals, cudaStream_t s) {
        k_gather_spawns<K, S><<<B < 4096 ? B : 4096, 256, 0, s>>>(keys, vals, cap, Cp, cnt, off, B,
                                                                  (K*)okeys, ovals);
    }
    static void column(const ModelParams& mp, const void* key, void* dest, double* val,
                       unsigned cap, double* diag, unsigned* m, cudaStream_t s) {
        k_column<K, KIND><<<1, 1, 0, s>>>(mp, *(const K*)key, (K*)dest, val, cap, diag, m);
    }
    static void ref_count(const ModelParams& mp, const void* refs, int n, unsigned* m,
                          cudaStream_t s) {
        k_ref_count<K, KIND><<<(n + 63) / 64, 64, 0, s>>>(mp, (const K*)refs, n, m);
    }
    static void ref_terms(const ModelParams& mp, const void* refs, const double* y, int n,
                          const unsigned* off, void* tkeys, double* th, double* tv,
                          unsigned* tseg, int log2B, cudaStream_t s) {
        k_ref_terms<K, KIND><<<(n + 63) / 64, 64, 0, s>>>(mp, (const K*)refs, y, n, off,
                                                          (K*)tkeys, th, tv, tseg, log2B);
    }
    static void overlap(const RunDesc* d, const OverlapDesc* od, int grid, int wpb,
                        unsigned table, cudaStream_t s) {
        const size_t smem = (size_t)wpb * table * (sizeof(K) + sizeof(double) + sizeof(unsigned));
        k_overlap<K, AMP, KIND><<<grid, wpb * 32, smem, s>>>(d, od);
        k_overlap_row<<<1, 256, 0, s>>>(d, od, (unsigned)(grid * wpb));
    }
    static cudaError_t prepare_overlap(size_t smem) {
        return cudaFuncSetAttribute(k_overlap<K, AMP, KIND>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    static constexpr size_t gs_dots_slot() { return sizeof(K) + sizeof(double) + sizeof(unsigned); }
    static constexpr size_t gs_axpy_slot() { return sizeof(K) + sizeof(ACC) + sizeof(unsigned) + 1; }
    static void gs(const RunDesc* d, const GsDesc* g, int k, int grid, int wpb, unsigned table,
                   cudaStream_t s) {
        k_gs_dots<K, AMP><<<grid, wpb * 32, (size_t)wpb * table * gs_dots_slot(), s>>>(d, g, k);
        k_gs_alpha<<<1, 32, 0, s>>>(d, g, k, (unsigned)(grid * wpb));
        k_gs_axpy<K, AMP, KIND><<<grid, wpb * 32, (size_t)wpb * table * gs_axpy_slot(), s>>>(d, g, k);
    }
    static cudaError_t prepare_gs(size_t smem) {
        cudaError_t e = cudaFuncSetAttribute(k_gs_dots<K, AMP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_gs_axpy<K, AMP, KIND>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return e;
    }
    static KernelSet make() {
        KernelSet k;
        k.key_bytes = sizeof(K);
        k.amp_bytes = sizeof(A);
        k.spawn_bytes = sizeof(S);
        k.spawn_key_stride = SpawnIO<K, S>::key_bytes;
        k.spawn_val_stride = SpawnIO<K, S>::val_bytes;
        k.slot_bytes = slot_bytes<K, AMP>();
        k.spawn = spawn;
        k.merge = merge;
        k.prepare = prepare;
        k.spawn_occupancy = spawn_occupancy;
        k.scratch_init = scratch_init;
        k.merge_occupancy = merge_occupancy;
        k.merge_smem = merge_smem;
        k.sort_ws_bytes = SortWs<K, AMP>::bytes;
        k.seed = seed;
        k.gather_vec = gather_vec;
        k.gather_spawns = gather_spawns;
        k.lookup = lookup;
        k.restride = restride;
        k.column = column;
        k.ref_count = ref_count;
        k.ref_terms = ref_terms;
        k.overlap = overlap;
        k.prepare_overlap = prepare_overlap;
        k.gs = gs;
        k.prepare_gs = prepare_gs;
        k.gs_slot_bytes = gs_dots_slot() > gs_axpy_slot() ? gs_dots_slot() : gs_axpy_slot();
        k.overlap_slot_bytes = sizeof(K) + sizeof(double) + sizeof(unsigned);
        return k;
    }
};

}  // namespace fq

#define FQ_INSTANTIATE(NAME, KEY, AMP)                                    \
    namespace fq {                                                        \
    void NAME(KernelSet* out) {                                           \
        out[0] = Launch<KEY, AMP, FQ_KIND_REAL_1D>::make();               \
        out[1] = Launch<KEY, AMP, FQ_KIND_REAL_2D>::make();               \
        out[2] = Launch<KEY, AMP, FQ_KIND_MOM_1D>::make();                \
    }                                                                     \
    }
