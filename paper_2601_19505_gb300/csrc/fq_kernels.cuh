// fq_kernels.cuh -- the FCIQMC step as three kernels per step for a batch of
// independent runs (Rimu.jl paper, Eq. stochasticTransitionOperator):
//
//   k_spawn  For every occupied entry c_i of c^(n): decide an exact or a
//            stochastic column (|c_i| t_rel >= m_i, Sec. 7.1), then write the
//            column's spawns H_ji coef_i, coef_i = -dt c_i (exact) or
//            -dt (m_i / n_i) c_i for n_i = ceil|c_i| uniform picks (Eq.
//            column-compression), into the bucket owning each destination.
//   k_merge  For every bucket: sum the spawns to the bucket per address in
//            an on-chip open-addressing table (annihilation); give each entry
//            of c^(n)'s segment its diagonal term 1 + dt (S - H_ii) plus the
//            sum of its address, then the addresses only spawns reached;
//            apply vector compression Pi (Eq. vec-compression); compact the
//            survivors into c^(n+1)'s segment; accumulate ||c||_1 (exactly),
//            len and the projected-energy terms.
//   k_shift  One block per run: Eq. shift-update, a history row, the buffer
//            flip, and the diagonal-factor table of the next step.
//
// Layout: the vector of a run is hash-segmented (the paper's PDVec segments,
// Sec. 6.4, as thousands of small segments sized for one merge warp's
// on-chip table): segment b = top log2(B) bits of seg_hash(address), capacity Cv
// entries each, structure-of-arrays keys/amplitudes.  Spawn buckets use the
// same segment map with capacity Cs.  All sizes and pointers are read from
// device memory, so one captured CUDA graph replays any number of steps.
//
// GB300 executes FP64 at a small fraction of its FP32/integer rate, so the
// kernels keep FP64 work to about one multiply per spawn and one multiply
// and add per entry (FP64 amplitudes) or none (FP32 amplitudes); decisions
// whose result is exact are
// taken on integer bits (fq_device.cuh), with results identical to the FP64
// expressions they stand for.
#pragma once

#include <cuda_runtime.h>

#include "fq_device.cuh"
#include "fq_shared.h"

namespace fq {

template <int AMP> struct AmpT;
template <> struct AmpT<FQ_AMP_INT> {
    typedef long long A;    // stored amplitude
    typedef int S;          // spawn value
    typedef long long ACC;  // on-chip sum
    typedef double C;       // per-source coefficient
};
template <> struct AmpT<FQ_AMP_F64> { typedef double A, S, ACC, C; };
template <> struct AmpT<FQ_AMP_F32> { typedef float A, S, ACC, C; };

// compiled variants of the spawn and merge kernels (the autotuner picks one
// of each): warps per block and the resident blocks per SM the registers
// are capped for -- 8 x 2 (up to 128 registers a thread, 16 warps per SM),
// 4 x 5 (up to 96, 20 warps), 4 x 6 (up to 80, 24 warps)
template <int V> struct Var;
template <> struct Var<0> { static constexpr int WPB = 8, MINB = 2; };
template <> struct Var<1> { static constexpr int WPB = 4, MINB = 5; };
template <> struct Var<2> { static constexpr int WPB = 4, MINB = 6; };
constexpr int kVariants = 3;

// ---------------------------------------------------------------------------
// Where slot `pos` of bucket b lies in the spawn buffers (B buckets of Cs
// slots).  The first Cp slots of every bucket form a dense primary region of
// B Cp entries; the other Cs - Cp slots of every bucket follow it.  Spawns
// land in random buckets, so each store touches a random page of the region
// it falls in, and on GB300 such stores slow down with the size of that
// region (measured: 4.9e8 random 32-byte stores took 27 ms spread over
// 51 GB, 56 ms over 103 GB).  A primary region sized for the steady-state
// bucket fill keeps nearly every store in a small region while the
// capacity for transients stays.
__host__ __device__ __forceinline__ size_t spawn_slot(unsigned b, unsigned pos, unsigned Cp,
                                                      unsigned Cs, unsigned B) {
    return pos < Cp ? (size_t)b * Cp + pos
                    : (size_t)B * Cp + (size_t)b * (Cs - Cp) + (pos - Cp);
}

// ---------------------------------------------------------------------------
// Spawn buffers: one record per spawn in `kb` (the run's skeys; `vb`, its
// samps, is unused).  128-bit addresses: 32 bytes (address, value, zero
// padding), which fill exactly one 32-byte DRAM sector, so a spawn is stored
// as a whole sector and the memory system never has to read the sector's
// old contents to merge a partial write (spawns land in random buckets, so
// the sectors of separate 16-byte keys and 8-byte values were mostly written
// partly).  64-bit addresses: 16 bytes (address, value).  Entry i of bucket
// b is at spawn_slot(b, i, ...).
template <class K, class S> struct SpawnIO {
    static constexpr bool REC = sizeof(K) == 16;
    static constexpr size_t key_bytes = REC ? 32 : 16;  // bytes per entry of kb
    static constexpr size_t val_bytes = 0;              // bytes per entry of vb
    // A record is written by one store (256 or 128 bits): a random-bucket
    // store is one request to the memory system instead of two (measured on
    // the spawn kernel's store pattern: 4.9e8 32-byte records in 15 ms
    // against 27 ms as two 16-byte stores; c2's spawn kernel 9 % faster with
    // 16-byte records than with separate address and value arrays).  Records
    // are aligned to their size (the buffers are 256-byte aligned).
    __device__ __forceinline__ static void store(void* kb, void* vb, size_t i, K key, S v) {
        if constexpr (REC) {
            unsigned char* p = (unsigned char*)kb + i * 32;
            const unsigned long long lo = (unsigned long long)key;
            const unsigned long long hi = (unsigned long long)(key >> 32 >> 32);
            unsigned long long vbits = 0;
            memcpy(&vbits, &v, sizeof(S));
            asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};\n" ::"l"(p), "l"(lo), "l"(hi),
                         "l"(vbits), "l"(0ull)
                         : "memory");
        } else {
            unsigned long long vbits = 0;
            memcpy(&vbits, &v, sizeof(S));
            unsigned char* p = (unsigned char*)kb + i * 16;
            asm volatile("st.global.v2.b64 [%0], {%1, %2};\n" ::"l"(p), "l"((unsigned long long)key),
                         "l"(vbits)
                         : "memory");
        }
    }
    __device__ __forceinline__ static void load(const void* kb, const void* vb, size_t i, K& key,
                                                S& v) {
        if constexpr (REC) {
            const unsigned char* p = (const unsigned char*)kb + i * 32;
            unsigned long long lo, hi, vbits, pad;
            asm volatile("ld.global.v4.b64 {%0, %1, %2, %3}, [%4];\n"
                         : "=l"(lo), "=l"(hi), "=l"(vbits), "=l"(pad)
                         : "l"(p));
            (void)pad;
            key = (K)lo | ((K)hi << 32 << 32);
            memcpy(&v, &vbits, sizeof(S));
        } else {
            const unsigned char* p = (const unsigned char*)kb + i * 16;
            unsigned long long kk, vbits;
            asm volatile("ld.global.v2.b64 {%0, %1}, [%2];\n" : "=l"(kk), "=l"(vbits) : "l"(p));
            key = (K)kk;
            memcpy(&v, &vbits, sizeof(S));
        }
    }
};

// ---------------------------------------------------------------------------
// warp-level helpers

__device__ __forceinline__ unsigned warp_incl_scan(unsigned x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}
template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}
__device__ __forceinline__ void warp_sum128(unsigned long long& lo, unsigned long long& hi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long l = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
        const unsigned long long h = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
        add128(lo, hi, l, h);
    }
}
// contiguous range of segments for global warp w of nw
__device__ __forceinline__ void warp_range(unsigned G, unsigned w, unsigned nw, unsigned& g0,
                                           unsigned& g1) {
    g0 = (unsigned)(((unsigned long long)G * w) / nw);
    g1 = (unsigned)(((unsigned long long)G * (w + 1)) / nw);
}

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (cp.async, 16-byte chunks; a chunk
// with src_bytes < 16 reads only src_bytes and zero-fills the rest)

__device__ __forceinline__ void cp_async16(void* dst, const void* src, unsigned src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// L2 prefetch of `bytes` rounded up to 16 at a 16-byte aligned address,
// never past `cap` bytes (a multiple of 16: the region's capacity)
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes, unsigned cap) {
    bytes = min((bytes + 15u) & ~15u, cap);
    if (bytes)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// L2 prefetch of segment `seg` of vector buffer `buf` of run R: its stored
// entries' addresses and amplitudes (segments start 16-byte aligned: the
// capacity Cv is a multiple of 32 entries)
template <class K, class A>
__device__ __forceinline__ void prefetch_segment(const RunDesc* R, int buf, unsigned seg) {
    const unsigned Cv = min(R->Cv, 1u << 25);
    const unsigned n = min(R->vcount[buf][seg], Cv);
    const size_t o = (size_t)seg * R->Cv;
    prefetch_l2((const K*)R->vkeys[buf] + o, n * (unsigned)sizeof(K), Cv * (unsigned)sizeof(K));
    prefetch_l2((const A*)R->vamps[buf] + o, n * (unsigned)sizeof(A), Cv * (unsigned)sizeof(A));
}

// a warp copies `bytes` from global (16-byte aligned) to shared
__device__ __forceinline__ void warp_copy_async(void* dst, const void* src, unsigned bytes, int lane) {
    for (unsigned o = (unsigned)lane * 16u; o < bytes; o += 32u * 16u)
        cp_async16((unsigned char*)dst + o, (const unsigned char*)src + o,
                   bytes - o < 16u ? bytes - o : 16u);
}

// ---------------------------------------------------------------------------
// K1: spawning.  One warp per segment range; a segment is taken in batches
// of up to 32 * IPT entries, staged in shared memory by cp.async one batch
// ahead, each lane owning IPT consecutive entries; the batch's spawn
// indices are dealt round-robin to the lanes.  A spawn's bucket slot is
// reserved by an atomic whose result is used one round later, so the
// atomics' latency overlaps the next round's work.  No block barriers.

// dynamic shared memory of one spawn warp
template <class K, int AMP, int CH, int KIND> struct SpawnSmem {
    typedef typename AmpT<AMP>::A A;
    typedef typename AmpT<AMP>::C CO;
    static constexpr size_t al(size_t b) { return (b + 15) / 16 * 16; }
    static constexpr size_t key_off = 0;                                  // K [2][CH]
    static constexpr size_t amp_off = key_off + al(2 * CH * sizeof(K));   // A [2][CH]
    static constexpr size_t coef_off = amp_off + al(2 * CH * sizeof(A));  // CO [CH]
    static constexpr size_t off_off = coef_off + al(CH * sizeof(CO));     // unsigned [CH + 1]
    static constexpr size_t m_off = off_off + al((CH + 1) * sizeof(unsigned));  // unsigned [CH]
    // the run's model parameters (the part the model's column reads)
    static constexpr size_t mp_bytes =
        KIND == FQ_KIND_MOM_1D ? sizeof(ModelParams) : offsetof(ModelParams, eps);
    static constexpr size_t mp_off = m_off + al(CH * sizeof(unsigned));
    static constexpr size_t bytes = mp_off + al(mp_bytes);
};

template <class K, int AMP, int KIND, int V, int IPT>
__global__ void __launch_bounds__(Var<V>::WPB * 32, Var<V>::MINB)
k_spawn(const RunDesc* __restrict__ runs, const unsigned* __restrict__ seg_run, unsigned G) {
    constexpr int WPB = Var<V>::WPB;
    typedef typename AmpT<AMP>::A A;
    typedef typename AmpT<AMP>::S S;
    typedef typename AmpT<AMP>::C CO;
    typedef Model<KIND> MD;
    typedef typename MD::Col Col;
    typedef SpawnSmem<K, AMP, 32 * IPT, KIND> SM;
    constexpr int CH = 32 * IPT;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char* const wbase = smem + (size_t)wib * SM::bytes;
    K* const in_key = (K*)(wbase + SM::key_off);
    A* const in_amp = (A*)(wbase + SM::amp_off);
    CO* const wcoef = (CO*)(wbase + SM::coef_off);
    unsigned* const woff = (unsigned*)(wbase + SM::off_off);
    unsigned* const wm = (unsigned*)(wbase + SM::m_off);
    // the current run's model parameters, copied into the warp's shared
    // memory when the run is entered: read there, they are not reloaded
    // through L1 after every spawn store (which the compiler cannot tell
    // apart from the run descriptor)
    ModelParams* const wmp = (ModelParams*)(wbase + SM::mp_off);
    const ModelParams& mp = *wmp;
    unsigned g0, g1;
    warp_range(G, blockIdx.x * WPB + wib, gridDim.x * WPB, g0, g1);

    // the run of the current item: its segments [run_lo, run_hi) and per-step
    // constants
    const RunDesc* R = nullptr;
    unsigned run_lo = 0, run_hi = 0;
    unsigned err = 0;
    const K* vk0 = nullptr;
    const A* va0 = nullptr;
    const unsigned* vcnt = nullptr;
    unsigned Cv = 0, Cs = 0, Cp = 0, stepno = 0;
    void* sk = nullptr;
    void* sv = nullptr;
    unsigned* sfill = nullptr;
    int log2B = 0;
    double dt = 0.0;
    uint2 rkey = make_uint2(0, 0);
    int early = 0;
    // per-source constants of the run, in registers for the same reason
    int r_det = 0, r_trel_one = 0, r_mmax = 0;
    double r_trel = 0.0;
    const typename AmpT<AMP>::C* r_coef = nullptr;
    unsigned n_ex = 0, n_inex = 0, n_sp = 0;

    // the spawn whose bucket slot is being reserved (stored one spawn later)
    K pd = KeyOps<K>::empty();
    S pv = (S)0;
    unsigned pb = 0, pp = 0;
    bool ph = false;

    auto flush_pending = [&]() {
        if (!ph) return;
        if (pp < Cs) {
            SpawnIO<K, S>::store(sk, sv, spawn_slot(pb, pp, Cp, Cs, run_hi - run_lo), pd, pv);
        } else {
            atomicOr(&R->st->err, FQ_DERR_SPAWN_CAP);
        }
        ph = false;
    };
    auto flush_counts = [&]() {
        const unsigned long long a = warp_sum((unsigned long long)n_ex);
        const unsigned long long i = warp_sum((unsigned long long)n_inex);
        const unsigned long long p = warp_sum((unsigned long long)n_sp);
        if (lane == 0) {
            if (a) atomicAdd(&R->st->n_exact, a);
            if (i) atomicAdd(&R->st->n_inexact, i);
            if (p) atomicAdd(&R->st->n_spawns, p);
        }
        n_ex = n_inex = n_sp = 0;
    };
    // make run r current (warp-uniform)
    auto enter_run = [&](int r) {
        if (R) {
            flush_pending();
            flush_counts();
        }
        R = runs + r;
        // lane 0 reads, the warp shares: another warp may set an error bit
        unsigned e = 0, c = 0;
        if (lane == 0) {
            e = *(volatile unsigned*)&R->st->err;
            c = (unsigned)R->st->cur;
        }
        err = __shfl_sync(0xFFFFFFFFu, e, 0);
        const unsigned cur = __shfl_sync(0xFFFFFFFFu, c, 0);
        run_lo = R->seg_base;
        run_hi = run_lo + R->B;
        vk0 = (const K*)R->vkeys[cur];
        va0 = (const A*)R->vamps[cur];
        vcnt = R->vcount[cur];
        Cv = R->Cv;
        Cs = R->Cs;
        Cp = R->Cp;
        sk = R->skeys;
        sv = R->samps;
        sfill = R->sfill;
        log2B = R->log2B;
        dt = R->st->dt;
        stepno = (unsigned)(R->st->step + 1);
        rkey = make_uint2(R->key_x, R->key_y);
        early = R->early;
        r_det = R->mode_det;
        r_trel_one = R->trel_one;
        r_trel = R->t_rel;
        r_mmax = R->mmax;
        if constexpr (AMP == FQ_AMP_F32) r_coef = R->coef32;
        else if constexpr (AMP == FQ_AMP_F64) r_coef = R->coef64;
        __syncwarp();  // every lane is done with the previous run's parameters
        for (unsigned i = (unsigned)lane; i < (unsigned)(SM::mp_bytes / 4); i += 32u)
            ((unsigned*)wmp)[i] = ((const unsigned*)&R->mp)[i];
        __syncwarp();
    };
    // the next non-empty segment of the current run at or after g; the end
    // of the run's part of the range if none (n = its entry count)
    // the count of segment pre_g, loaded one segment ahead of its use
    unsigned pre_g = 0xFFFFFFFFu, pre_n = 0;
    auto next_segment = [&](unsigned g, unsigned& n) -> unsigned {
        const unsigned hi = min(g1, run_hi);
        if (err) return hi;
        for (; g < hi; ++g) {
            n = g == pre_g ? pre_n : vcnt[g - run_lo];
            if (n) return g;
        }
        return hi;
    };
    auto stage = [&](unsigned g, unsigned c0, unsigned cn, int b) {
        const size_t e0 = (size_t)(g - run_lo) * Cv + c0;
        warp_copy_async(in_key + b * CH, vk0 + e0, cn * (unsigned)sizeof(K), lane);
        warp_copy_async(in_amp + b * CH, va0 + e0, cn * (unsigned)sizeof(A), lane);
        cp_async_commit();
    };
    // attempt a of a source (key, its column data col, coefficient cf, mm =
    // m and flags): the destination and value; false when an integer spawn
    // rounds to nothing
    auto make_col = [&](K key, const Col& col, CO cf, unsigned mm, unsigned a, K& dest,
                        S& val) -> bool {
        const unsigned m = mm & 0x3FFFFFFFu;
        const bool ex = (AMP != FQ_AMP_INT) && (mm >> 31);
        uint4 w = make_uint4(0, 0, 0, 0);
        unsigned kk = a;
        if (!ex) {
            w = draw(rkey, stepno, a, KeyOps<K>::rng_h(key));
            kk = pick(w, m);
        }
        if constexpr (AMP == FQ_AMP_INT) {
            double hv;
            dest = MD::offdiag(mp, key, col, kk, hv);
            const double p = fabs(hv) * cf;
            const double fl = floor(p);
            const long long nw = (long long)fl + (uniform53(w) < p - fl ? 1 : 0);
            if (!nw) return false;
            const int sg = (hv > 0.0 ? -1 : 1) * ((mm & 0x40000000u) ? -1 : 1);
            val = (S)(sg * nw);
        } else {
            CO hv;
            dest = MD::offdiag(mp, key, col, kk, hv);
            val = hv * cf;
            if (early && !at_least_theta(val, R)) {
                // early compression: the pick's own draw decides; entry kk of
                // an exact column takes the draw of stream kk
                if (ex) w = draw(rkey, stepno, a, KeyOps<K>::rng_h(key));
                if (!pi_below(val, w, R)) return false;
            }
        }
        return true;
    };
    // the same, recomputing the column data from the address
    auto make = [&](K key, CO cf, unsigned mm, unsigned a, K& dest, S& val) -> bool {
        Col col;
        if constexpr (KIND != FQ_KIND_MOM_1D) col.n_occ = (int)((mm & 0x3FFFFFFFu) / (unsigned)MD::Z);
        else MD::num_offdiag(mp, key, col);
        return make_col(key, col, cf, mm, a, dest, val);
    };

    // reserve a bucket slot for this lane's spawn (if any) and store the
    // previous one, whose slot has arrived meanwhile
    auto emit = [&](bool has, K dest, S val) {
        unsigned bk = 0, pos = 0;
        if (has) {
            bk = segment_of(seg_hash(dest), log2B);
            pos = atomicAdd(&sfill[bk], 1u);
            ++n_sp;
        }
        flush_pending();
        if (has) {
            pd = dest;
            pv = val;
            pb = bk;
            pp = pos;
            ph = true;
        }
    };

    // current item (segment g, entries [c0, c0 + CH) of n), staged in buffer b
    unsigned g = g0, c0 = 0, n = 0;
    int b = 0;
    bool staged = false;
    while (true) {
        if (g < g1 && (g < run_lo || g >= run_hi)) {
            enter_run((int)seg_run[g]);
            staged = false;
        }
        if (!staged) {
            g = next_segment(g, n);
            if (g >= g1) break;
            if (g >= run_hi) continue;
            c0 = 0;
            stage(g, 0, min((unsigned)CH, n), b);
        }
        const unsigned cn = min((unsigned)CH, n - c0);
        cp_async_wait_all();
        __syncwarp();
        // stage the next item of the same run into the other buffer
        unsigned ng = g, nc0 = c0 + CH, nn = n;
        if (nc0 >= n) {
            nc0 = 0;
            ng = next_segment(g + 1, nn);
        }
        staged = ng < g1 && ng < run_hi;
        if (staged) stage(ng, nc0, min((unsigned)CH, nn - nc0), b ^ 1);
        if (staged && ng + 1 < min(g1, run_hi) && pre_g != ng + 1) {
            pre_g = ng + 1;
            pre_n = vcnt[pre_g - run_lo];
        }

        const K* wkey = in_key + b * CH;
        const A* wamp = in_amp + b * CH;
        // sources i = j * 32 + lane: the decision, the coefficient and the
        // first attempt at once; further attempts are counted (extras) and
        // dealt out below
        unsigned xoff = 0;
        for (int j = 0; j < IPT; ++j) {
            const unsigned i = (unsigned)j * 32u + (unsigned)lane;
            unsigned cnt = 0, mm = 0;
            CO cf = (CO)0;
            K key = KeyOps<K>::empty();
            Col col;
            if (i < cn) {
                key = wkey[i];
                const CO c = (CO)wamp[i];
                const unsigned m = MD::num_offdiag(mp, key, col);
                unsigned fl, ce;
                floor_ceil_abs(c, fl, ce);
                if (AMP == FQ_AMP_INT) {
                    // integer walkers: |c| attempts, never an exact column;
                    // the coefficient is dt m (spawn probability per |H_ji|)
                    cnt = m ? fl : 0u;
                    ++n_inex;
                    cf = (CO)(dt * (double)m);
                    mm = m | (c < (CO)0 ? 0x40000000u : 0u);
                } else {
                    bool ex;
                    if (r_det) ex = true;
                    else if (r_trel_one) ex = fl >= m;  // |c| >= m for an integer m
                    else ex = fabs((double)c) * r_trel >= (double)m;
                    cnt = ex ? m : ce;
                    if (ex) {
                        ++n_ex;
                        cf = (-(CO)dt) * c;
                    } else {
                        ++n_inex;
                        const int mmax = r_mmax;
                        if (KIND != FQ_KIND_MOM_1D && (int)m <= mmax && (int)ce <= mmax) {
                            // (-dt) (m / n) from the run's table for this dt
                            const size_t ri = (size_t)m * (size_t)(mmax + 1) + ce;
                            cf = __ldg(r_coef + ri) * c;
                        } else {
                            cf = ((-(CO)dt) * ((CO)m / (CO)ce)) * c;
                        }
                    }
                    mm = m | (ex ? 0x80000000u : 0u);
                }
                wcoef[i] = cf;
                wm[i] = mm;
            }
            const unsigned x = cnt > 1u ? cnt - 1u : 0u;
            if (__any_sync(0xFFFFFFFFu, x)) {
                const unsigned incl = warp_incl_scan(x, lane);
                woff[i] = xoff + incl - x;
                xoff += __shfl_sync(0xFFFFFFFFu, incl, 31);
            } else {  // no further attempts in this round (one pick per source)
                woff[i] = xoff;
            }
            K dest = KeyOps<K>::empty();
            S val = (S)0;
            const bool has = cnt >= 1u && make_col(key, col, cf, mm, 0u, dest, val);
            emit(has, dest, val);
        }
        __syncwarp();
        // attempts 1.. of every source, balanced over the lanes: spawn q
        // belongs to the last source whose offset is <= q
        for (unsigned q0 = 0; q0 < xoff; q0 += 32) {
            const unsigned q = q0 + (unsigned)lane;
            K dest = KeyOps<K>::empty();
            S val = (S)0;
            bool has = false;
            if (q < xoff) {
                unsigned i = 0;
#pragma unroll
                for (unsigned st = CH / 2; st >= 1; st >>= 1)
                    if (woff[i + st] <= q) i += st;
                has = make(wkey[i], wcoef[i], wm[i], 1u + (q - woff[i]), dest, val);
            }
            emit(has, dest, val);
        }
        __syncwarp();  // every lane is done with buffer b
        g = ng;
        if (!staged) continue;
        c0 = nc0;
        n = nn;
        b ^= 1;
    }
    if (R) {
        flush_pending();
        flush_counts();
    }
}

// ---------------------------------------------------------------------------
// on-chip open-addressing table (linear probing, CAS on the key)

__device__ __forceinline__ uint64_t key_cas(uint64_t* p, uint64_t cmp, uint64_t val) {
    return (uint64_t)atomicCAS((unsigned long long*)p, (unsigned long long)cmp,
                               (unsigned long long)val);
}
__device__ __forceinline__ u128 key_cas(u128* p, u128 cmp, u128 val) {
    return atomicCAS(p, cmp, val);
}

// home slot of `key` in a table of mask + 1 (a power of two) slots:
// multiplicative (Fibonacci) hashing of the address folded to 32 bits.  The
// keys of one bucket share the top bits of their segment hash, which this
// hash does not use.
__device__ __forceinline__ unsigned fold32(uint64_t k) { return (unsigned)k ^ (unsigned)(k >> 32); }
__device__ __forceinline__ unsigned fold32(u128 k) {
    return fold32((uint64_t)k ^ (uint64_t)(k >> 64));
}
template <class K> __device__ __forceinline__ unsigned table_home(K key, unsigned mask) {
    return (fold32(key) * 0x9E3779B1u) >> (32 - __popc(mask));
}

// slot of `key`, inserting it if absent (is_new set); -1 when the table is full
template <class K>
__device__ __forceinline__ int table_insert(K* tkey, unsigned mask, K key, bool& is_new) {
    const K EMPTY = KeyOps<K>::empty();
    unsigned q = table_home(key, mask);
    is_new = false;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const K seen = tkey[q];
        if (seen == key) return (int)q;
        if (seen == EMPTY) {
            const K old = key_cas(&tkey[q], EMPTY, key);
            if (old == EMPTY) { is_new = true; return (int)q; }
            if (old == key) return (int)q;
        }
        q = (q + 1) & mask;
    }
    return -1;
}

template <class K>
__device__ __forceinline__ int table_find(const K* tkey, unsigned mask, K key) {
    const K EMPTY = KeyOps<K>::empty();
    unsigned q = table_home(key, mask);
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const K seen = tkey[q];
        if (seen == key) return (int)q;
        if (seen == EMPTY) return -1;
        q = (q + 1) & mask;
    }
    return -1;
}

// The run's constants that Pi, the norm terms and the diagonal term read for
// every value, taken once per bucket: read from the run descriptor inside
// the loops they would be loaded again after every store of the compacted
// vector, which the compiler cannot tell apart from the descriptor.
// Seven registers: theta's bits, (float)theta, theta's exponent, two flags
// and the diagonal-factor table of the amplitude type.
struct StepConst {
    unsigned long long theta_bits;  // dbits(theta)
    float theta32;                  // (float)theta
    int theta_exp;
    int flags;                      // 1: theta is a power of two, 2: deterministic limit
    const void* diag;               // fac64 (FP64, integer walkers) or del32 (FP32)
    __device__ __forceinline__ double theta() const { return bdouble(theta_bits); }
    __device__ __forceinline__ bool pow2() const { return flags & 1; }
    __device__ __forceinline__ bool det() const { return flags & 2; }
};
template <int AMP>
__device__ __forceinline__ StepConst step_const(const RunDesc* R) {
    StepConst k;
    k.theta_bits = dbits(R->theta);
    k.theta32 = R->theta32;
    k.theta_exp = R->theta_exp;
    k.flags = (R->theta_pow2 ? 1 : 0) | (R->mode_det ? 2 : 0);
    if constexpr (AMP == FQ_AMP_F32) k.diag = R->del32;
    else k.diag = R->fac64;
    return k;
}

// Pi (Eq. vec-compression) of one merged value: keep |w| >= theta, else
// sign(w) theta with probability |w| / theta.  `out` is the stored value.
template <int AMP>
__device__ __forceinline__ bool compress(typename AmpT<AMP>::ACC w, const StepConst& R, uint2 rkey,
                                         unsigned stepno, uint64_t h,
                                         typename AmpT<AMP>::ACC& out) {
    typedef typename AmpT<AMP>::ACC ACC;
    if constexpr (AMP == FQ_AMP_INT) {
        out = w;
        return w != 0;
    } else {
        const unsigned long long ab = abs_dbits(w);
        if (R.det()) {
            out = w;
            return ab != 0;
        }
        if (ab == 0) return false;
        const double theta = R.theta();
        if (R.pow2()) {
            if (ab >= dbits(theta)) {
                out = w;
                return true;
            }
            const uint4 r = draw(rkey, stepno, 0xFFFFFFFFu, h);
            if (!below_scaled(u53_of(r), ab, R.theta_exp)) return false;
        } else {
            const double aw = bdouble(ab);
            if (aw >= theta) {
                out = w;
                return true;
            }
            const uint4 r = draw(rkey, stepno, 0xFFFFFFFFu, h);
            if (!(uniform53(r) < aw / theta)) return false;
        }
        // sign(w) theta, on the bits
        if constexpr (AMP == FQ_AMP_F64)
            out = bdouble(dbits(theta) | (dbits(w) & 0x8000000000000000ull));
        else
            out = __uint_as_float(__float_as_uint(R.theta32) | (__float_as_uint(w) & 0x80000000u));
        return true;
    }
}

// per-warp totals of one run, carried across buckets
struct MergeAcc {
    unsigned long long nlo, nhi, nlen;
    double nfp;
    bool full, over, range_bad;
    unsigned long long ntheta;  // stored values of magnitude theta (a power of two)
    unsigned n_onchip, n_scratch;  // buckets summed in each kind of table (warp-uniform)
};

// the two halves of Pi for one value, for early compression (Sec. 7.1, Eq.
// early-comp), where the draw is the one of the spawn or a stream of its own:
// |v| >= theta (kept as it is), decided on the bits
template <class V>
__device__ __forceinline__ bool at_least_theta(V v, const StepConst& k) {
    const unsigned long long ab = abs_dbits(v);
    return k.pow2() ? ab >= k.theta_bits : bdouble(ab) >= k.theta();
}
template <class V>
__device__ __forceinline__ bool at_least_theta(V v, const RunDesc* R) {
    return at_least_theta(v, step_const<FQ_AMP_F64>(R));  // the table is not read
}
// |v| < theta: v becomes sign(v) theta with probability |v| / theta (the
// 53-bit uniform of r against |v| / theta), else it is dropped (false)
template <class V>
__device__ __forceinline__ bool pi_below(V& v, uint4 r, const StepConst& k) {
    const unsigned long long ab = abs_dbits(v);
    if (ab == 0) return false;
    if (k.pow2()) {
        if (!below_scaled(u53_of(r), ab, k.theta_exp)) return false;
    } else {
        if (!(uniform53(r) < bdouble(ab) / k.theta())) return false;
    }
    if constexpr (sizeof(V) == 8)
        v = bdouble(k.theta_bits | (dbits(v) & 0x8000000000000000ull));
    else
        v = __uint_as_float(__float_as_uint(k.theta32) | (__float_as_uint(v) & 0x80000000u));
    return true;
}
template <class V>
__device__ __forceinline__ bool pi_below(V& v, uint4 r, const RunDesc* R) {
    return pi_below(v, r, step_const<FQ_AMP_F64>(R));  // the table is not read
}

// add a warp's share of one run's step totals to the run's accumulators
__device__ __forceinline__ void merge_flush(const RunDesc* R, MergeAcc a, int lane) {
    unsigned long long nlo = a.nlo, nhi = a.nhi;
    add128(nlo, nhi, a.ntheta << 52, a.ntheta >> 12);  // the values of magnitude theta
    warp_sum128(nlo, nhi);
    const unsigned long long nlen = warp_sum(a.nlen);
    const double nfp = warp_sum(a.nfp);
    const bool f = __any_sync(0xFFFFFFFFu, a.full), o = __any_sync(0xFFFFFFFFu, a.over),
               b = __any_sync(0xFFFFFFFFu, a.range_bad);
    if (lane == 0) {
        const unsigned long long old = atomicAdd(&R->st->norm_lo, nlo);
        atomicAdd(&R->st->norm_hi, nhi + (old + nlo < old ? 1ull : 0ull));
        atomicAdd(&R->st->len_acc, nlen);
        if (R->mode_det) atomicAdd(&R->st->norm_fp, nfp);
        if (a.n_onchip) atomicAdd(&R->st->merged_onchip, (unsigned long long)a.n_onchip);
        if (a.n_scratch) atomicAdd(&R->st->merged_scratch, (unsigned long long)a.n_scratch);
        if (f) atomicOr(&R->st->err, FQ_DERR_TABLE);
        if (o) atomicOr(&R->st->err, FQ_DERR_VEC_CAP);
        if (b) atomicOr(&R->st->err, FQ_DERR_RANGE);
    }
}

// bytes of one table slot: key, accumulator, list entry
template <class K, int AMP> __host__ __device__ constexpr size_t slot_bytes() {
    return sizeof(K) + sizeof(typename AmpT<AMP>::ACC) + sizeof(unsigned);
}

// a table sum that an entry of c^(n) has taken over (no valid sum has these
// bits: a NaN payload, or the most negative integer)
template <class ACC> __device__ __forceinline__ ACC taken_mark();
template <> __device__ __forceinline__ double taken_mark<double>() {
    return __longlong_as_double(0x7FF4C0DEC0DEC0DEll);
}
template <> __device__ __forceinline__ float taken_mark<float>() { return __int_as_float(0x7FA0C0DE); }
template <> __device__ __forceinline__ long long taken_mark<long long>() {
    return (long long)0x8000000000000000ull;
}
__device__ __forceinline__ bool is_taken(double x) {
    return __double_as_longlong(x) == 0x7FF4C0DEC0DEC0DEll;
}
__device__ __forceinline__ bool is_taken(float x) { return __float_as_int(x) == 0x7FA0C0DE; }
__device__ __forceinline__ bool is_taken(long long x) {
    return x == (long long)0x8000000000000000ull;
}

// Pi, compaction and the norm terms of one merged value, for a warp of lanes
// (keep: the lane has a value)
// compaction and the norm terms of the values a warp keeps (keep: the lane
// stores `out` at `key`)
template <class K, int AMP>
__device__ __forceinline__ void merge_store(const StepConst& R, bool keep, K key,
                                            typename AmpT<AMP>::ACC out, K* __restrict__ ok,
                                            typename AmpT<AMP>::A* __restrict__ oa, unsigned Cv,
                                            int nq, int det, int lane, unsigned& nout,
                                            MergeAcc& acc) {
    typedef typename AmpT<AMP>::A A;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
    if (keep) {
        const unsigned pos = nout + (unsigned)__popc(bal & ((1u << lane) - 1u));
        if (pos < Cv) {
            ok[pos] = key;
            oa[pos] = (A)out;
        } else {
            acc.over = true;
        }
        ++acc.nlen;
        if constexpr (AMP == FQ_AMP_INT) {
            const unsigned long long av = (unsigned long long)(out < 0 ? -out : out);
            add128(acc.nlo, acc.nhi, av, 0ull);
        } else {
            if (det) {
                acc.nfp += fabs((double)out);
            } else if (R.pow2() && abs_dbits(out) == R.theta_bits) {
                ++acc.ntheta;  // theta = 2^(nq + 52): 2^52 units, added at the flush
            } else {
                unsigned long long lo, hi;
                fixed_of(out, nq, lo, hi, acc.range_bad);
                add128(acc.nlo, acc.nhi, lo, hi);
            }
        }
    }
    nout += (unsigned)__popc(bal);
}

template <class K, int AMP>
__device__ __forceinline__ void merge_emit(const StepConst& R, bool has, K key,
                                           typename AmpT<AMP>::ACC w, uint2 rkey, unsigned stepno,
                                           K* __restrict__ ok, typename AmpT<AMP>::A* __restrict__ oa,
                                           unsigned Cv, int nq, int det, int early, int lane,
                                           unsigned& nout, MergeAcc& acc) {
    typedef typename AmpT<AMP>::ACC ACC;
    ACC out = (ACC)0;
    // early compression stores the sums as they are (Eq. early-comp)
    const bool keep = has && (early ? ((out = w) != (ACC)0)
                                    : compress<AMP>(w, R, rkey, stepno, KeyOps<K>::rng_h(key), out));
    merge_store<K, AMP>(R, keep, key, out, ok, oa, Cv, nq, det, lane, nout, acc);
}

// The end of a bucket: the projected-energy terms whose address falls in it
// (the survivors read back: this warp wrote them), the new segment's count,
// and the bucket's spawn counter cleared for the next step.
template <class K, int AMP>
__device__ __forceinline__ void bucket_finish(const RunDesc* R, unsigned seg, unsigned cur,
                                              unsigned nout, const K* ok,
                                              const typename AmpT<AMP>::A* oa, int lane) {
    const unsigned Cv = R->Cv;
    const unsigned e0 = R->ref_off[seg], e1 = R->ref_off[seg + 1];
    if (e1 > e0) {  // warp-uniform
        const K* rk = (const K*)R->ref_keys;
        const unsigned nw = nout <= Cv ? nout : Cv;
        double hp = 0.0, vp = 0.0;
        for (unsigned e = e0; e < e1; ++e) {
            const K want = rk[e];
            double cv = 0.0;
            for (unsigned i = lane; i < nw; i += 32)
                if (ok[i] == want) cv = (double)oa[i];
            cv = warp_sum(cv);  // at most one lane holds the address
            hp += R->ref_h[e] * cv;
            vp += R->ref_v[e] * cv;
        }
        if (lane == 0) {
            R->part_h[seg] = hp;
            R->part_v[seg] = vp;
        }
    }
    if (lane == 0) {
        R->vcount[cur ^ 1][seg] = nout <= Cv ? nout : Cv;
        R->sfill[seg] = 0u;
    }
}

// The diagonal term of an entry c of c^(n) at `key`: c (1 + dt (S - H_ii))
// (Eq. stochasticTransitionOperator; integer walkers round it stochastically
// with the draw of stream 0xFFFFFFFE); under early compression it is then
// compressed alone with the draw of stream 0xFFFFFFFD (0 when dropped).
template <class K, int AMP, int KIND>
__device__ __forceinline__ typename AmpT<AMP>::ACC diag_term(const RunDesc* R, const StepConst& kc,
                                                            K key, typename AmpT<AMP>::A c,
                                                            uint2 rkey, unsigned stepno, int early) {
    typedef typename AmpT<AMP>::ACC ACC;
    typedef Model<KIND> MD;
    ACC w;
    if constexpr (KIND != FQ_KIND_MOM_1D) {
        const int si = MD::diag_index(key);
        if constexpr (AMP == FQ_AMP_F32) {
            w = c + c * __ldg((const float*)kc.diag + si);
        } else if constexpr (AMP == FQ_AMP_F64) {
            w = c * __ldg((const double*)kc.diag + si);
        } else {
            const double x = (double)c * __ldg((const double*)kc.diag + si);
            const double fl = floor(x);
            const uint4 r4 = draw(rkey, stepno, 0xFFFFFFFEu, KeyOps<K>::rng_h(key));
            w = (ACC)((long long)fl + (uniform53(r4) < x - fl ? 1 : 0));
        }
    } else {
        const double hii = MD::diagonal(R->mp, key);
        const double S0 = R->st->shift, dt = R->st->dt;
        if constexpr (AMP == FQ_AMP_F32) {
            w = c + c * (float)(dt * (S0 - hii));
        } else if constexpr (AMP == FQ_AMP_F64) {
            w = c * (1.0 + dt * (S0 - hii));
        } else {
            const double x = (double)c * (1.0 + dt * (S0 - hii));
            const double fl = floor(x);
            const uint4 r4 = draw(rkey, stepno, 0xFFFFFFFEu, KeyOps<K>::rng_h(key));
            w = (ACC)((long long)fl + (uniform53(r4) < x - fl ? 1 : 0));
        }
    }
    if constexpr (AMP != FQ_AMP_INT) {
        if (early && !at_least_theta(w, kc)) {
            const uint4 r4 = draw(rkey, stepno, 0xFFFFFFFDu, KeyOps<K>::rng_h(key));
            if (!pi_below(w, r4, kc)) w = (ACC)0;
        }
    }
    return w;
}

// One bucket.  The spawns go into the table (tk, ta, tl; mask + 1 slots, all
// EMPTY / 0 on entry and on return), which sums them per address.  Then each
// entry of c^(n)'s segment, with its diagonal term, takes over the sum of
// its own address (if any) and is compressed and compacted; then the
// addresses that only spawns reached.  Last, the projected-energy terms of
// the bucket's addresses.
template <class K, int AMP, int KIND>
__device__ __forceinline__ void merge_bucket(const RunDesc* R, unsigned seg, unsigned cur,
                                             unsigned n_old, unsigned n_sp, K* tk,
                                             typename AmpT<AMP>::ACC* ta, unsigned* tl,
                                             unsigned mask, int lane, MergeAcc& acc) {
    typedef typename AmpT<AMP>::A A;
    typedef typename AmpT<AMP>::S S;
    typedef typename AmpT<AMP>::ACC ACC;
    typedef Model<KIND> MD;
    const K EMPTY = KeyOps<K>::empty();
    const unsigned Cv = R->Cv;
    const K* __restrict__ vk = (const K*)R->vkeys[cur] + (size_t)seg * Cv;
    const A* __restrict__ va = (const A*)R->vamps[cur] + (size_t)seg * Cv;
    K* __restrict__ ok = (K*)R->vkeys[cur ^ 1] + (size_t)seg * Cv;
    A* __restrict__ oa = (A*)R->vamps[cur ^ 1] + (size_t)seg * Cv;
    const void* const skb = R->skeys;
    const void* const svb = R->samps;
    const unsigned sCp = R->Cp, sCs = R->Cs, sB = R->B;
    const unsigned stepno = (unsigned)(R->st->step + 1);
    const uint2 rkey = make_uint2(R->key_x, R->key_y);
    const int nq = R->norm_q;
    const int det = R->mode_det;
    const int early = R->early;
    const StepConst kc = step_const<AMP>(R);

    // annihilation: every spawn to the bucket adds into its address; new
    // addresses join the list in warp order.  The next spawns are loaded
    // before the current ones are inserted.
    unsigned nl = 0;
    {
        K skey = EMPTY;
        S sval = (S)0;
        if (lane < n_sp)
            SpawnIO<K, S>::load(skb, svb, spawn_slot(seg, lane, sCp, sCs, sB), skey, sval);
        for (unsigned j0 = 0; j0 < n_sp; j0 += 32) {
            const unsigned j = j0 + lane;
            bool nw = false;
            int q = -1;
            const K key = skey;
            const S v = sval;
            if (j + 32 < n_sp)
                SpawnIO<K, S>::load(skb, svb, spawn_slot(seg, j + 32, sCp, sCs, sB), skey, sval);
            if (j < n_sp) {
                q = table_insert(tk, mask, key, nw);
                if (q < 0) acc.full = true;
            }
            // the table is the warp's own: only lanes of this round that hit
            // the same slot conflict.  They pass their values to the lowest
            // of them, which adds the group's sum with a plain update, or
            // stores it when a lane of the group created the slot this round
            // (its sum is still 0; nearly every spawn reaches a new address).
            const unsigned grp = __match_any_sync(0xFFFFFFFFu, q);
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, nw);
            if (q >= 0) {
                ACC sum = (ACC)v;
                for (unsigned o = grp & (grp - 1u); o; o &= o - 1u)
                    sum = sum + (ACC)__shfl_sync(grp, v, __ffs(o) - 1);
                if (lane == __ffs(grp) - 1) ta[q] = (bal & grp) ? sum : ta[q] + sum;
            }
            if (nw) tl[nl + __popc(bal & ((1u << lane) - 1u))] = (unsigned)q;
            nl += __popc(bal);
        }
    }
    __syncwarp();

    // c^(n)'s entries: diagonal term c_i (1 + dt (S - H_ii)) (integer walkers
    // round it stochastically) plus the spawns to i, then Pi
    unsigned nout = 0;
    {
        K nkey = lane < n_old ? vk[lane] : EMPTY;
        A ncv = lane < n_old ? va[lane] : (A)0;
        for (unsigned i0 = 0; i0 < n_old; i0 += 32) {
            const unsigned i = i0 + lane;
            const K key = nkey;
            const A c = ncv;
            if (i + 32 < n_old) {
                nkey = vk[i + 32];
                ncv = va[i + 32];
            }
            ACC w = (ACC)0;
            const bool has = i < n_old;
            if (has) {
                w = diag_term<K, AMP, KIND>(R, kc, key, c, rkey, stepno, early);
                if (n_sp) {
                    const int q = table_find(tk, mask, key);
                    if (q >= 0) {
                        w = w + ta[q];
                        ta[q] = taken_mark<ACC>();
                    }
                }
            }
            merge_emit<K, AMP>(kc, has, key, w, rkey, stepno, ok, oa, Cv, nq, det, early, lane,
                               nout, acc);
        }
    }
    __syncwarp();
    // addresses only spawns reached
    for (unsigned b0 = 0; b0 < nl; b0 += 32) {
        const unsigned i = b0 + lane;
        bool has = false;
        ACC w = (ACC)0;
        K key = EMPTY;
        if (i < nl) {
            const unsigned q = tl[i];
            w = ta[q];
            has = !is_taken(w);
            key = tk[q];
        }
        merge_emit<K, AMP>(kc, has, key, w, rkey, stepno, ok, oa, Cv, nq, det, early, lane, nout,
                           acc);
    }
    __syncwarp();
    bucket_finish<K, AMP>(R, seg, cur, nout, ok, oa, lane);
    // release the used slots for the next bucket
    for (unsigned i = lane; i < nl; i += 32) {
        const unsigned q = tl[i];
        tk[q] = EMPTY;
        ta[q] = (ACC)0;
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Annihilation by sorting (FQ_ANN_SORT).  A bucket's contributions -- the
// diagonal terms of c^(n)'s segment first, then the spawns in arrival order --
// are sorted by a 16-bit hash of their address with a stable LSD radix sort of
// two 8-bit digits: digit counts, their exclusive scan, then a scatter in
// rounds of 32 that ranks a round's equal digits by __match_any_sync.  Every
// address's contributions then lie in one run of equal hash, in their original
// order; the first occurrence of each address in its run sums the run's
// contributions to that address (a segmented reduction), and Pi, compaction
// and the norm terms follow as in the hash arm.  The address set and every
// decision are the hash arm's; FP sums differ only in their order.

// per-warp workspace of C elements: address, value, 16-bit hash and two
// 16-bit index arrays, then 256 digit counters
template <class K, int AMP> struct SortWs {
    typedef typename AmpT<AMP>::ACC ACC;
    __host__ __device__ static constexpr size_t al(size_t b) { return (b + 15) / 16 * 16; }
    __host__ __device__ static constexpr size_t val_off(unsigned C) { return al((size_t)C * sizeof(K)); }
    __host__ __device__ static constexpr size_t hash_off(unsigned C) {
        return val_off(C) + al((size_t)C * sizeof(ACC));
    }
    __host__ __device__ static constexpr size_t ia_off(unsigned C) { return hash_off(C) + al((size_t)C * 2); }
    __host__ __device__ static constexpr size_t ib_off(unsigned C) { return ia_off(C) + al((size_t)C * 2); }
    __host__ __device__ static constexpr size_t bins_off(unsigned C) { return ib_off(C) + al((size_t)C * 2); }
    __host__ __device__ static constexpr size_t bytes(unsigned C) { return bins_off(C) + 256 * 4; }
};

template <class K> __device__ __forceinline__ unsigned short hash16(K key) {
    return (unsigned short)((fold32(key) * 0x9E3779B1u) >> 16);
}

template <class K, int AMP, int KIND>
__device__ __forceinline__ void sort_bucket(const RunDesc* R, unsigned seg, unsigned cur,
                                            unsigned n_old, unsigned n_sp, unsigned char* ws,
                                            unsigned C, int lane, MergeAcc& acc) {
    typedef typename AmpT<AMP>::A A;
    typedef typename AmpT<AMP>::S S;
    typedef typename AmpT<AMP>::ACC ACC;
    typedef SortWs<K, AMP> L;
    const K EMPTY = KeyOps<K>::empty();
    const unsigned Cv = R->Cv;
    const K* __restrict__ vk = (const K*)R->vkeys[cur] + (size_t)seg * Cv;
    const A* __restrict__ va = (const A*)R->vamps[cur] + (size_t)seg * Cv;
    K* __restrict__ ok = (K*)R->vkeys[cur ^ 1] + (size_t)seg * Cv;
    A* __restrict__ oa = (A*)R->vamps[cur ^ 1] + (size_t)seg * Cv;
    const unsigned sCp = R->Cp, sCs = R->Cs, sB = R->B;
    const unsigned stepno = (unsigned)(R->st->step + 1);
    const uint2 rkey = make_uint2(R->key_x, R->key_y);
    const int nq = R->norm_q, det = R->mode_det, early = R->early;
    const StepConst kc = step_const<AMP>(R);
    K* const wk = (K*)ws;
    ACC* const wv = (ACC*)(ws + L::val_off(C));
    unsigned short* const wh = (unsigned short*)(ws + L::hash_off(C));
    unsigned short* const ia = (unsigned short*)(ws + L::ia_off(C));
    unsigned short* const ib = (unsigned short*)(ws + L::ib_off(C));
    unsigned* const bins = (unsigned*)(ws + L::bins_off(C));
    const unsigned n = n_old + n_sp;

    for (unsigned i = lane; i < n_old; i += 32) {
        const K key = vk[i];
        wk[i] = key;
        wv[i] = diag_term<K, AMP, KIND>(R, kc, key, va[i], rkey, stepno, early);
        wh[i] = hash16(key);
        ia[i] = (unsigned short)i;
    }
    for (unsigned j = lane; j < n_sp; j += 32) {
        K key;
        S sval;
        SpawnIO<K, S>::load(R->skeys, R->samps, spawn_slot(seg, j, sCp, sCs, sB), key, sval);
        const unsigned i = n_old + j;
        wk[i] = key;
        wv[i] = (ACC)sval;
        wh[i] = hash16(key);
        ia[i] = (unsigned short)i;
    }
    __syncwarp();
    for (int pass = 0; pass < 2; ++pass) {
        const int shift = 8 * pass;
        const unsigned short* src = pass ? ib : ia;
        unsigned short* dst = pass ? ia : ib;
        for (unsigned b = lane; b < 256; b += 32) bins[b] = 0u;
        __syncwarp();
        for (unsigned i = lane; i < n; i += 32) atomicAdd(&bins[(wh[src[i]] >> shift) & 255u], 1u);
        __syncwarp();
        unsigned v[8], t = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            v[k] = bins[8 * lane + k];
            t += v[k];
        }
        unsigned run = warp_incl_scan(t, lane) - t;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            bins[8 * lane + k] = run;
            run += v[k];
        }
        __syncwarp();
        for (unsigned i0 = 0; i0 < n; i0 += 32) {
            const unsigned i = i0 + lane;
            const bool valid = i < n;
            const unsigned e = valid ? src[i] : 0u;
            const unsigned d = valid ? ((unsigned)(wh[e] >> shift) & 255u) : 256u + (unsigned)lane;
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
            if (valid) dst[bins[d] + __popc(peers & ((1u << lane) - 1u))] = (unsigned short)e;
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) bins[d] += (unsigned)__popc(peers);
            __syncwarp();
        }
    }
    // sorted order in ia; each address's first position in its hash run sums
    unsigned nout = 0;
    for (unsigned i0 = 0; i0 < n; i0 += 32) {
        const unsigned i = i0 + lane;
        bool head = false;
        ACC w = (ACC)0;
        K key = EMPTY;
        if (i < n) {
            const unsigned e = ia[i];
            key = wk[e];
            const unsigned short h = wh[e];
            head = true;
            for (unsigned j = i; j > 0;) {
                const unsigned f = ia[--j];
                if (wh[f] != h) break;
                if (wk[f] == key) {
                    head = false;
                    break;
                }
            }
            if (head) {
                w = wv[e];
                for (unsigned j = i + 1; j < n; ++j) {
                    const unsigned f = ia[j];
                    if (wh[f] != h) break;
                    if (wk[f] == key) w = w + wv[f];
                }
            }
        }
        merge_emit<K, AMP>(kc, head, key, w, rkey, stepno, ok, oa, Cv, nq, det, early, lane, nout,
                           acc);
    }
    __syncwarp();
    bucket_finish<K, AMP>(R, seg, cur, nout, ok, oa, lane);
    __syncwarp();
}

// ---------------------------------------------------------------------------
// K4: diagonal update + annihilation + vector compression + compaction +
//     estimator accumulation.  One warp per bucket range; each warp owns an
//     on-chip table of SW slots (keys, sums, list of used slots).  A bucket
//     whose spawns could exceed 0.7 SW uses the warp's table of SS slots in
//     global scratch memory instead.  No block barriers.

// on-chip bytes of one merge warp: a hash table of SW slots, or a sort
// workspace of SW elements
template <class K, int AMP, int ANN> __host__ __device__ constexpr size_t merge_warp_bytes(unsigned SW) {
    return ANN == FQ_ANN_SORT_ARM ? SortWs<K, AMP>::bytes(SW) : (size_t)SW * slot_bytes<K, AMP>();
}

template <class K, int AMP, int KIND, int V, int ANN>
__global__ void __launch_bounds__(Var<V>::WPB * 32, Var<V>::MINB)
k_merge(const RunDesc* __restrict__ runs, const unsigned* __restrict__ seg_run, unsigned G,
        unsigned SW, unsigned char* __restrict__ scratch, unsigned SS) {
    constexpr int WPB = Var<V>::WPB;
    typedef typename AmpT<AMP>::ACC ACC;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned gw = blockIdx.x * WPB + wib;
    unsigned char* base_s = smem + (size_t)wib * merge_warp_bytes<K, AMP, ANN>(SW);
    // global scratch of the warp: a hash table of SS slots (hash arm), or a
    // sort workspace of SS elements (sort arm), for buckets beyond the
    // on-chip one
    unsigned char* base_g =
        scratch + (size_t)gw * (ANN == FQ_ANN_SORT_ARM ? SortWs<K, AMP>::bytes(SS)
                                                       : (size_t)SS * slot_bytes<K, AMP>());
    K* const sk_s = (K*)base_s;
    ACC* const sa_s = (ACC*)(base_s + (size_t)SW * sizeof(K));
    unsigned* const sl_s = (unsigned*)(base_s + (size_t)SW * (sizeof(K) + sizeof(ACC)));
    K* const sk_g = (K*)base_g;
    ACC* const sa_g = (ACC*)(base_g + (size_t)SS * sizeof(K));
    unsigned* const sl_g = (unsigned*)(base_g + (size_t)SS * (sizeof(K) + sizeof(ACC)));
    const K EMPTY = KeyOps<K>::empty();

    if constexpr (ANN != FQ_ANN_SORT_ARM) {
        for (unsigned q = lane; q < SW; q += 32) {
            sk_s[q] = EMPTY;
            sa_s[q] = (ACC)0;
        }
    }
    __syncwarp();
    unsigned g0, g1;
    warp_range(G, gw, gridDim.x * WPB, g0, g1);

    const RunDesc* R = nullptr;
    unsigned run_lo = 0, run_hi = 0;  // segments of the current run
    unsigned err = 0, cur = 0;
    MergeAcc acc = {0, 0, 0, 0.0, false, false, false, 0, 0, 0};
    // counts of buckets ahead_g and ahead2_g, loaded before they are needed
    unsigned ahead_g = 0xFFFFFFFFu, ahead2_g = 0xFFFFFFFFu;
    unsigned a1_old = 0, a1_sp = 0, a2_old = 0, a2_sp = 0;

    for (unsigned g = g0; g < g1; ++g) {
        if (g < run_lo || g >= run_hi) {  // warp-uniform
            if (R) {
                merge_flush(R, acc, lane);
                acc = MergeAcc{0, 0, 0, 0.0, false, false, false, 0, 0, 0};
            }
            R = runs + seg_run[g];
            run_lo = R->seg_base;
            run_hi = run_lo + R->B;
            // lane 0 reads, the warp shares: another warp may set an error bit
            unsigned e = 0, c = 0;
            if (lane == 0) {
                e = *(volatile unsigned*)&R->st->err;
                c = (unsigned)R->st->cur;
            }
            err = __shfl_sync(0xFFFFFFFFu, e, 0);
            cur = __shfl_sync(0xFFFFFFFFu, c, 0);
        }
        if (err) continue;
        const unsigned seg = g - R->seg_base;
        // this bucket's counts (loaded one bucket ahead when it was the next);
        // then the next bucket's data is prefetched into L2 and the counts of
        // the one after it are loaded
        unsigned n_old, n_sp;
        if (g == ahead_g) {
            n_old = a1_old;
            n_sp = a1_sp;
        } else {
            n_old = R->vcount[cur][seg];
            n_sp = R->sfill[seg];
        }
        const unsigned g_end = min(g1, R->seg_base + R->B);
        if (g + 1 < g_end) {
            unsigned o1, s1;
            if (g + 1 == ahead2_g) {
                o1 = a2_old;
                s1 = a2_sp;
            } else {
                o1 = R->vcount[cur][seg + 1];
                s1 = R->sfill[seg + 1];
            }
            if (lane == 0) {
                typedef typename AmpT<AMP>::A A;
                typedef typename AmpT<AMP>::S S;
                const size_t vo = (size_t)(seg + 1) * R->Cv;
                // capacities are multiples of 32 entries; sizes kept below 2^30
                const unsigned Cv = min(R->Cv, 1u << 25), Cs = min(R->Cs, 1u << 25);
                const unsigned Cp = min(R->Cp, Cs);
                const unsigned po = min(o1, Cv), ps = min(s1, Cs);
                prefetch_l2((const K*)R->vkeys[cur] + vo, po * (unsigned)sizeof(K),
                            Cv * (unsigned)sizeof(K));
                prefetch_l2((const A*)R->vamps[cur] + vo, po * (unsigned)sizeof(A),
                            Cv * (unsigned)sizeof(A));
                typedef SpawnIO<K, S> IO;
                // the bucket's primary slots, then those beyond them
                const unsigned p1 = min(ps, Cp), p2 = ps - p1;
                const size_t so1 = spawn_slot(seg + 1, 0, Cp, Cs, R->B),
                             so2 = spawn_slot(seg + 1, Cp, Cp, Cs, R->B);
                prefetch_l2((const unsigned char*)R->skeys + so1 * IO::key_bytes,
                            p1 * (unsigned)IO::key_bytes, Cp * (unsigned)IO::key_bytes);
                if (p2)
                    prefetch_l2((const unsigned char*)R->skeys + so2 * IO::key_bytes,
                                p2 * (unsigned)IO::key_bytes, (Cs - Cp) * (unsigned)IO::key_bytes);
                if (IO::val_bytes) {
                    prefetch_l2((const unsigned char*)R->samps + so1 * IO::val_bytes,
                                p1 * (unsigned)IO::val_bytes, Cp * (unsigned)IO::val_bytes);
                    if (p2)
                        prefetch_l2((const unsigned char*)R->samps + so2 * IO::val_bytes,
                                    p2 * (unsigned)IO::val_bytes,
                                    (Cs - Cp) * (unsigned)IO::val_bytes);
                }
            }
            ahead_g = g + 1;
            a1_old = o1;
            a1_sp = s1;
            if (g + 2 < g_end) {
                ahead2_g = g + 2;
                a2_old = R->vcount[cur][seg + 2];
                a2_sp = R->sfill[seg + 2];
            }
        }
        if constexpr (ANN == FQ_ANN_SORT_ARM) {
            // the workspace holds the bucket's entries and spawns
            const unsigned n = n_old + n_sp;
            if (n <= SW) {
                sort_bucket<K, AMP, KIND>(R, seg, cur, n_old, n_sp, base_s, SW, lane, acc);
                ++acc.n_onchip;
            } else if (n <= SS) {
                sort_bucket<K, AMP, KIND>(R, seg, cur, n_old, n_sp, base_g, SS, lane, acc);
                ++acc.n_scratch;
            } else {
                acc.full = true;
            }
            continue;
        }
        // the table holds the bucket's spawned addresses only
        const unsigned long long load = n_sp;
        if (load * 10ull <= (unsigned long long)SW * 7ull) {
            merge_bucket<K, AMP, KIND>(R, seg, cur, n_old, n_sp, sk_s, sa_s, sl_s, SW - 1u, lane,
                                       acc);
            ++acc.n_onchip;
        } else if (load * 10ull <= (unsigned long long)SS * 9ull) {
            merge_bucket<K, AMP, KIND>(R, seg, cur, n_old, n_sp, sk_g, sa_g, sl_g, SS - 1u, lane,
                                       acc);
            ++acc.n_scratch;
        } else {
            acc.full = true;  // even the scratch table cannot hold this bucket
        }
    }
    if (R) merge_flush(R, acc, lane);
}

// scratch tables start empty (keys EMPTY, sums 0); each use leaves them so
template <class K, int AMP>
__global__ void k_scratch_init(unsigned char* scratch, unsigned SS, unsigned nwarps) {
    typedef typename AmpT<AMP>::ACC ACC;
    const size_t total = (size_t)SS * nwarps;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t w = i / SS, q = i % SS;
        unsigned char* base = scratch + w * SS * slot_bytes<K, AMP>();
        ((K*)base)[q] = KeyOps<K>::empty();
        ((ACC*)(base + (size_t)SS * sizeof(K)))[q] = (ACC)0;
    }
}

// ---------------------------------------------------------------------------
// diagonal factors of the coming step: 1 + dt (S - H_ii) and its FP32
// increment, per value s = sum n(n-1) (real space, H_ii = (u/2) s)

__device__ __forceinline__ void write_factors(const RunDesc* R, double S, double dt) {
    for (int s = threadIdx.x; s <= R->smax; s += blockDim.x) {
        const double hii = (R->mp.u * 0.5) * (double)s;
        R->fac64[s] = 1.0 + dt * (S - hii);
        R->del32[s] = (float)(dt * (S - hii));
    }
}

// ... and, when dt is set, the spawn coefficients (-dt) (m / n) per (m, n)
// (m off-diagonal entries, n picks), in FP64 and in FP32 arithmetic
static __global__ void k_factors(const RunDesc* __restrict__ runs) {
    const RunDesc* R = runs + blockIdx.x;
    const double dt = R->st->dt;
    if (R->smax >= 0 && R->fac64) write_factors(R, R->st->shift, dt);
    if (R->coef64) {
        const int w = R->mmax + 1;
        const float dtf = (float)dt;
        for (int i = threadIdx.x; i < w * w; i += blockDim.x) {
            const int m = i / w, n = i % w;
            R->coef64[i] = n ? (-dt) * ((double)m / (double)n) : 0.0;
            R->coef32[i] = n ? (-dtf) * ((float)m / (float)n) : 0.0f;
        }
    }
}

// ---------------------------------------------------------------------------
// K5: shift update (Eq. shift-update), one block per run

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_shift(const RunDesc* __restrict__ runs) {
    const RunDesc* R = runs + blockIdx.x;
    RunState* st = R->st;
    __shared__ double s_S;
    __shared__ int s_ok;
    __shared__ double s_h[BLOCK], s_v[BLOCK];
    // the projected-energy partials of the reference buckets: strided over
    // the block, then a tree in a fixed order (the result does not depend on
    // timing)
    {
        double hp = 0.0, vp = 0.0;
        for (unsigned i = threadIdx.x; i < R->n_ref_bkt; i += BLOCK) {
            const unsigned b = R->ref_bkt[i];
            hp += R->part_h[b];
            vp += R->part_v[b];
        }
        s_h[threadIdx.x] = hp;
        s_v[threadIdx.x] = vp;
        __syncthreads();
        for (int o = BLOCK / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) {
                s_h[threadIdx.x] += s_h[threadIdx.x + o];
                s_v[threadIdx.x] += s_v[threadIdx.x + o];
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        s_ok = 0;
        if (!*(volatile unsigned*)&st->err) {
            double nrm;
            if (R->mode_det) nrm = st->norm_fp;
            else nrm = fixed_to_double(st->norm_lo, st->norm_hi, R->norm_q);
            const unsigned long long len = st->len_acc;
            const double hp = s_h[0], vp = s_v[0];
            if (nrm == 0.0 || len == 0) {
                st->err |= FQ_DERR_EMPTY;
            } else {
                const double dt = st->dt;
                const double zd = st->zeta / dt, xd = st->xi / dt;
                const double S1 =
                    (st->shift - zd * log(nrm / st->norm)) - xd * log(nrm / st->target);
                StatsRow row;
                row.step = st->step + 1;
                row.len = (long long)len;
                row.exact_steps = (long long)st->n_exact;
                row.inexact_steps = (long long)st->n_inexact;
                row.n_spawns = (long long)st->n_spawns;
                row.shift = S1;
                row.norm = nrm;
                row.hproj = hp;
                row.vproj = vp;
                R->hist[st->hist_head % FQ_HIST_CAP] = row;
                st->hist_head += 1;
                st->shift = S1;
                st->norm = nrm;
                st->step += 1;
                st->len = (long long)len;
                st->cur ^= 1;
                st->last_hproj = hp;
                st->last_vproj = vp;
                st->last_exact = row.exact_steps;
                st->last_inexact = row.inexact_steps;
                st->last_spawns = row.n_spawns;
                s_S = S1;
                s_ok = 1;
            }
            st->n_exact = 0;
            st->n_inexact = 0;
            st->n_spawns = 0;
            st->norm_lo = 0;
            st->norm_hi = 0;
            st->norm_fp = 0.0;
            st->len_acc = 0;
        }
    }
    __syncthreads();
    if (s_ok && R->smax >= 0 && R->fac64) write_factors(R, s_S, st->dt);
}

// ---------------------------------------------------------------------------
// replica overlaps (Sec. 4.3, Eq. RayleighQuotientReplica): for every pair
// (A, B) of a batch's runs and every segment, A's entries go into the warp's
// on-chip table and B's entries look up theirs; the products c_A,j c_B,j and
// G2(d)_jj c_A,j c_B,j (Eq. g2) are summed per warp.  Each warp writes its
// own partial sums (no atomics) and k_overlap_row adds them in warp order,
// so the result does not depend on timing.

// occupation numbers of the M modes of an address (modes without a run of
// ones stay 0)
template <class K>
__device__ __forceinline__ void occupations(K key, int M, unsigned char* occ) {
    for (int m = 0; m < M; ++m) occ[m] = 0;
    K st = run_starts(key);
    while (st) {
        const int P = KeyOps<K>::ctz(st);
        occ[P - KeyOps<K>::popc(key & KeyOps<K>::low(P))] = (unsigned char)run_from(key, P);
        st &= st - 1;
    }
}

template <class K, int AMP, int KIND>
__global__ void __launch_bounds__(128) k_overlap(const RunDesc* __restrict__ runs,
                                                 const OverlapDesc* __restrict__ od) {
    typedef typename AmpT<AMP>::A A;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const unsigned T = od->table;
    unsigned char* base = smem + (size_t)wib * T * (sizeof(K) + sizeof(double) + sizeof(unsigned));
    K* const tk = (K*)base;
    double* const ta = (double*)(base + (size_t)T * sizeof(K));
    unsigned* const tl = (unsigned*)(base + (size_t)T * (sizeof(K) + sizeof(double)));
    const K EMPTY = KeyOps<K>::empty();
    for (unsigned q = lane; q < T; q += 32) tk[q] = EMPTY;
    const unsigned gw = blockIdx.x * wpb + wib, nw = gridDim.x * wpb;
    const int P = od->P, nq = od->nq, W = 1 + nq;
    double* const part = od->part + (size_t)gw * P * W;
    for (int i = lane; i < P * W; i += 32) part[i] = 0.0;
    __syncwarp();
    const unsigned B = od->B;
    const unsigned long long total = (unsigned long long)P * B;
    const unsigned long long i0 = total * gw / nw, i1 = total * (gw + 1) / nw;
    double acc[1 + FQ_MAX_G2];
    for (int q = 0; q < W; ++q) acc[q] = 0.0;
    unsigned char occ[128];
    int cur_p = -1;
    const RunDesc *RA = nullptr, *RB = nullptr;
    int ca = 0, cb = 0;
    auto flush = [&]() {
        for (int q = 0; q < W; ++q) {
            const double v = warp_sum(acc[q]);
            if (lane == 0) part[cur_p * W + q] = v;
            acc[q] = 0.0;
        }
    };
    for (unsigned long long it = i0; it < i1; ++it) {
        const int p = (int)(it / B);
        const unsigned seg = (unsigned)(it % B);
        if (p != cur_p) {  // warp-uniform
            if (cur_p >= 0) flush();
            cur_p = p;
            RA = runs + od->pa[p];
            RB = runs + od->pb[p];
            ca = RA->st->cur;
            cb = RB->st->cur;
        }
        const unsigned na = min(RA->vcount[ca][seg], RA->Cv);
        const unsigned nb = min(RB->vcount[cb][seg], RB->Cv);
        // the next segment of the pair into L2 while this one is joined
        if (lane == 0 && it + 1 < i1 && seg + 1 < B) {
            prefetch_segment<K, A>(RA, ca, seg + 1);
            prefetch_segment<K, A>(RB, cb, seg + 1);
        }
        if (!na || !nb) continue;
        const K* ka = (const K*)RA->vkeys[ca] + (size_t)seg * RA->Cv;
        const A* aa = (const A*)RA->vamps[ca] + (size_t)seg * RA->Cv;
        const K* kb = (const K*)RB->vkeys[cb] + (size_t)seg * RB->Cv;
        const A* ab = (const A*)RB->vamps[cb] + (size_t)seg * RB->Cv;
        // A's entries (distinct addresses; the table has more slots than a
        // segment's capacity, so an insert always finds one)
        unsigned nl = 0;
        for (unsigned j0 = 0; j0 < na; j0 += 32) {
            const unsigned j = j0 + lane;
            bool is_new = false;
            int q = -1;
            if (j < na) {
                q = table_insert(tk, T - 1u, ka[j], is_new);
                if (q >= 0) ta[q] = (double)aa[j];
            }
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, is_new);
            if (is_new) tl[nl + __popc(bal & ((1u << lane) - 1u))] = (unsigned)q;
            nl += __popc(bal);
        }
        __syncwarp();
        for (unsigned j0 = 0; j0 < nb; j0 += 32) {
            const unsigned j = j0 + lane;
            if (j < nb) {
                const K key = kb[j];
                const int q = table_find(tk, T - 1u, key);
                if (q >= 0) {
                    const double prod = ta[q] * (double)ab[j];
                    acc[0] += prod;
                    if (nq) {
                        const int M = RA->mp.M;
                        occupations(key, M, occ);
                        for (int k = 0; k < nq; ++k) {
                            const int d = od->d[k];
                            long long sn = 0;
                            for (int i = 0; i < M; ++i) {
                                const int i2 = i + d < M ? i + d : i + d - M;
                                sn += (long long)occ[i] * ((long long)occ[i2] - (d == 0 ? 1 : 0));
                            }
                            acc[1 + k] += ((double)sn / (double)M) * prod;
                        }
                    }
                }
            }
        }
        __syncwarp();
        for (unsigned j = lane; j < nl; j += 32) tk[tl[j]] = EMPTY;
        __syncwarp();
    }
    if (cur_p >= 0) flush();
}

// one row of overlaps: the per-warp partial sums added in warp order; no row
// when a run of the batch failed this step (it will be rolled back)
static __global__ void k_overlap_row(const RunDesc* __restrict__ runs,
                                     const OverlapDesc* __restrict__ od, unsigned nwarps) {
    __shared__ int ok;
    const int n = od->P * (1 + od->nq);
    if (threadIdx.x == 0) {
        ok = 1;
        for (int r = 0; r < od->R; ++r)
            if (*(volatile unsigned*)&runs[r].st->err) ok = 0;
    }
    __syncthreads();
    if (!ok) return;
    const unsigned long long h = *od->head;
    double* row = od->ring + (size_t)(h % od->cap) * (size_t)(1 + n);
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        double s = 0.0;
        for (unsigned w = 0; w < nwarps; ++w) s += od->part[(size_t)w * n + t];
        row[1 + t] = s;
    }
    if (threadIdx.x == 0) row[0] = (double)runs[0].st->step;
    __syncthreads();
    if (threadIdx.x == 0) *od->head = h + 1;
}

// ---------------------------------------------------------------------------
// excited states (Sec. 2.2): Gram-Schmidt on the step's new vectors (in
// buffer cur ^ 1 until k_shift flips it).  For the run k being
// orthogonalised: k_gs_dots sums c_j^T c_k and c_j^T c_j for j < k per warp,
// k_gs_alpha adds the partials in warp order and forms alpha_j =
// (c_j^T c_k) / (c_j^T c_j), and k_gs_axpy forms c_k - sum_j alpha_j c_j
// segment by segment in an on-chip table (subtracting j = 0, 1, ... in turn),
// compresses every changed value by Pi with the draw of stream 0xFFFFFFFC of
// its address, and rewrites run k's segment in place with its norm terms.

template <class K, int AMP>
__global__ void __launch_bounds__(128) k_gs_dots(const RunDesc* __restrict__ runs,
                                                 const GsDesc* __restrict__ gs, int k) {
    typedef typename AmpT<AMP>::A A;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const unsigned T = gs->table;
    unsigned char* base = smem + (size_t)wib * T * (sizeof(K) + sizeof(double) + sizeof(unsigned));
    K* const tk = (K*)base;
    double* const ta = (double*)(base + (size_t)T * sizeof(K));
    unsigned* const tl = (unsigned*)(base + (size_t)T * (sizeof(K) + sizeof(double)));
    const K EMPTY = KeyOps<K>::empty();
    for (unsigned q = lane; q < T; q += 32) tk[q] = EMPTY;
    __syncwarp();
    const unsigned gw = blockIdx.x * wpb + wib, nw = gridDim.x * wpb;
    double acc[2 * FQ_MAX_SPECTRAL];
    for (int i = 0; i < 2 * k; ++i) acc[i] = 0.0;
    const RunDesc* Rk = runs + k;
    const int ck = Rk->st->cur ^ 1;
    unsigned g0, g1;
    warp_range(gs->B, gw, nw, g0, g1);
    for (unsigned seg = g0; seg < g1; ++seg) {
        if (lane == 0 && seg + 1 < g1) {  // the next segment of every state into L2
            prefetch_segment<K, A>(Rk, ck, seg + 1);
            for (int j = 0; j < k; ++j) prefetch_segment<K, A>(runs + j, runs[j].st->cur ^ 1, seg + 1);
        }
        const unsigned nk = min(Rk->vcount[ck][seg], Rk->Cv);
        const K* kk = (const K*)Rk->vkeys[ck] + (size_t)seg * Rk->Cv;
        const A* ka = (const A*)Rk->vamps[ck] + (size_t)seg * Rk->Cv;
        unsigned nl = 0;
        for (unsigned i0 = 0; i0 < nk; i0 += 32) {
            const unsigned i = i0 + lane;
            bool is_new = false;
            int q = -1;
            if (i < nk) {
                q = table_insert(tk, T - 1u, kk[i], is_new);
                if (q >= 0) ta[q] = (double)ka[i];
            }
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, is_new);
            if (is_new) tl[nl + __popc(bal & ((1u << lane) - 1u))] = (unsigned)q;
            nl += __popc(bal);
        }
        __syncwarp();
        for (int j = 0; j < k; ++j) {
            const RunDesc* Rj = runs + j;
            const int cj = Rj->st->cur ^ 1;
            const unsigned nj = min(Rj->vcount[cj][seg], Rj->Cv);
            const K* jk = (const K*)Rj->vkeys[cj] + (size_t)seg * Rj->Cv;
            const A* ja = (const A*)Rj->vamps[cj] + (size_t)seg * Rj->Cv;
            for (unsigned i = lane; i < nj; i += 32) {
                const double v = (double)ja[i];
                acc[2 * j + 1] += v * v;
                if (nk) {
                    const int q = table_find(tk, T - 1u, jk[i]);
                    if (q >= 0) acc[2 * j] += v * ta[q];
                }
            }
        }
        __syncwarp();
        for (unsigned i = lane; i < nl; i += 32) tk[tl[i]] = EMPTY;
        __syncwarp();
    }
    double* part = gs->part + (size_t)gw * 2 * FQ_MAX_SPECTRAL;
    for (int i = 0; i < 2 * k; ++i) {
        const double v = warp_sum(acc[i]);
        if (lane == 0) part[i] = v;
    }
}

// the coefficients alpha_j of run k from the per-warp partial sums (warp
// order); run k's norm accumulators restart for k_gs_axpy
static __global__ void k_gs_alpha(const RunDesc* __restrict__ runs, const GsDesc* __restrict__ gs,
                                  int k, unsigned nwarps) {
    __shared__ double d[2 * FQ_MAX_SPECTRAL];
    const int t = threadIdx.x;
    if (t < 2 * k) {
        double s = 0.0;
        for (unsigned w = 0; w < nwarps; ++w) s += gs->part[(size_t)w * 2 * FQ_MAX_SPECTRAL + t];
        d[t] = s;
    }
    __syncthreads();
    if (t == 0) {
        for (int j = 0; j < k; ++j) gs->alpha[j] = d[2 * j + 1] != 0.0 ? d[2 * j] / d[2 * j + 1] : 0.0;
        RunState* st = runs[k].st;
        st->norm_lo = 0;
        st->norm_hi = 0;
        st->norm_fp = 0.0;
        st->len_acc = 0;
    }
}

template <class K, int AMP, int KIND>
__global__ void __launch_bounds__(128) k_gs_axpy(const RunDesc* __restrict__ runs,
                                                 const GsDesc* __restrict__ gs, int k) {
    typedef typename AmpT<AMP>::A A;
    typedef typename AmpT<AMP>::ACC ACC;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const unsigned T = gs->table;
    unsigned char* base =
        smem + (size_t)wib * T * (sizeof(K) + sizeof(ACC) + sizeof(unsigned) + 1);
    K* const tk = (K*)base;
    ACC* const ta = (ACC*)(base + (size_t)T * sizeof(K));
    unsigned* const tl = (unsigned*)(base + (size_t)T * (sizeof(K) + sizeof(ACC)));
    unsigned char* const tc = base + (size_t)T * (sizeof(K) + sizeof(ACC) + sizeof(unsigned));
    const K EMPTY = KeyOps<K>::empty();
    for (unsigned q = lane; q < T; q += 32) {
        tk[q] = EMPTY;
        tc[q] = 0;
    }
    __syncwarp();
    const unsigned gw = blockIdx.x * wpb + wib, nw = gridDim.x * wpb;
    const RunDesc* R = runs + k;
    unsigned e = 0;
    if (lane == 0)
        for (int j = 0; j <= k; ++j) e |= *(volatile unsigned*)&runs[j].st->err;
    if (__shfl_sync(0xFFFFFFFFu, e, 0)) return;  // the step fails and is rolled back
    const int cur = R->st->cur, ck = cur ^ 1;
    const unsigned Cv = R->Cv;
    const unsigned stepno = (unsigned)(R->st->step + 1);
    const uint2 rkey = make_uint2(R->key_x, R->key_y);
    const int nq = R->norm_q, det = R->mode_det;
    double alpha[FQ_MAX_SPECTRAL];
    for (int j = 0; j < k; ++j) alpha[j] = gs->alpha[j];
    MergeAcc acc = {0, 0, 0, 0.0, false, false, false, 0, 0, 0};
    unsigned g0, g1;
    warp_range(gs->B, gw, nw, g0, g1);
    for (unsigned seg = g0; seg < g1; ++seg) {
        if (lane == 0 && seg + 1 < g1) {  // the next segment of every state into L2
            prefetch_segment<K, A>(R, ck, seg + 1);
            for (int j = 0; j < k; ++j) prefetch_segment<K, A>(runs + j, runs[j].st->cur ^ 1, seg + 1);
        }
        const unsigned nk = min(R->vcount[ck][seg], Cv);
        K* const kk = (K*)R->vkeys[ck] + (size_t)seg * Cv;
        A* const ka = (A*)R->vamps[ck] + (size_t)seg * Cv;
        unsigned nl = 0;
        // run k's entries, then each earlier run's contribution in turn
        for (int j = -1; j < k; ++j) {
            const RunDesc* Rj = j < 0 ? R : runs + j;
            const int cj = j < 0 ? ck : (Rj->st->cur ^ 1);
            const unsigned nj = j < 0 ? nk : min(Rj->vcount[cj][seg], Rj->Cv);
            const K* jk = (const K*)Rj->vkeys[cj] + (size_t)seg * Rj->Cv;
            const A* ja = (const A*)Rj->vamps[cj] + (size_t)seg * Rj->Cv;
            for (unsigned i0 = 0; i0 < nj; i0 += 32) {
                const unsigned i = i0 + lane;
                bool is_new = false;
                int q = -1;
                if (i < nj) {
                    q = table_insert(tk, T - 1u, jk[i], is_new);
                    if (q < 0) {
                        acc.full = true;
                    } else if (j < 0) {
                        ta[q] = (ACC)ja[i];
                    } else {
                        const ACC v = is_new ? (ACC)0 : ta[q];
                        if constexpr (AMP == FQ_AMP_F32)
                            ta[q] = v - (float)alpha[j] * ja[i];
                        else
                            ta[q] = v - (ACC)(alpha[j] * (double)ja[i]);
                        tc[q] = 1;
                    }
                }
                const unsigned bal = __ballot_sync(0xFFFFFFFFu, is_new);
                if (is_new) tl[nl + __popc(bal & ((1u << lane) - 1u))] = (unsigned)q;
                nl += __popc(bal);
            }
            __syncwarp();
        }
        // changed values compressed (Pi, stream 0xFFFFFFFC), then compacted
        // back into run k's segment
        unsigned nout = 0;
        for (unsigned b0 = 0; b0 < nl; b0 += 32) {
            const unsigned i = b0 + lane;
            bool keep = false;
            ACC w = (ACC)0;
            K key = EMPTY;
            if (i < nl) {
                const unsigned q = tl[i];
                key = tk[q];
                w = ta[q];
                keep = w != (ACC)0;
                if constexpr (AMP != FQ_AMP_INT) {  // integer walkers never get here
                    if (keep && tc[q] && !det && !at_least_theta(w, R)) {
                        const uint4 r4 = draw(rkey, stepno, 0xFFFFFFFCu, KeyOps<K>::rng_h(key));
                        keep = pi_below(w, r4, R);
                    }
                }
            }
            merge_store<K, AMP>(step_const<AMP>(R), keep, key, w, kk, ka, Cv, nq, det, lane, nout, acc);
        }
        __syncwarp();
        bucket_finish<K, AMP>(R, seg, cur, nout, kk, ka, lane);
        for (unsigned i = lane; i < nl; i += 32) {
            tk[tl[i]] = EMPTY;
            tc[tl[i]] = 0;
        }
        __syncwarp();
    }
    merge_flush(R, acc, lane);
}

// ---------------------------------------------------------------------------
// set-up and read-out helpers (not on the per-step path)

// sqrt(k), -(t sqrt(k)) and its FP32 rounding for k <= kmax; m / n in FP64
// and FP32 for 1 <= n <= m <= mmax
static __global__ void k_tables(double t, int kmax, double* sq, double* hop, float* hop32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= kmax) {
        const double s = sqrt((double)i);
        sq[i] = s;
        hop[i] = -(t * s);
        hop32[i] = (float)hop[i];
    }
}

template <class K, int AMP>
__global__ void k_seed(const RunDesc* __restrict__ R, const K* __restrict__ keys,
                       const double* __restrict__ amps, size_t n) {
    typedef typename AmpT<AMP>::A A;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int cur = R->st->cur;
    const K key = keys[i];
    const unsigned b = segment_of(seg_hash(key), R->log2B);
    const unsigned pos = atomicAdd(&R->vcount[cur][b], 1u);
    if (pos < R->Cv) {
        ((K*)R->vkeys[cur])[(size_t)b * R->Cv + pos] = key;
        ((A*)R->vamps[cur])[(size_t)b * R->Cv + pos] = (A)amps[i];
    } else {
        atomicOr(&R->st->err, FQ_DERR_VEC_CAP);
    }
}

// copy each segment's entries from stride `oc` to stride `nc` (capacity growth)
template <class K, class A>
__global__ void k_restride(const K* __restrict__ ok, const A* __restrict__ oa, unsigned oc,
                           const unsigned* __restrict__ cnt, unsigned B, K* __restrict__ nk,
                           A* __restrict__ na, unsigned nc) {
    for (unsigned b = blockIdx.x; b < B; b += gridDim.x) {
        const unsigned n = min(cnt[b], oc);
        for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
            nk[(size_t)b * nc + i] = ok[(size_t)b * oc + i];
            na[(size_t)b * nc + i] = oa[(size_t)b * oc + i];
        }
    }
}

// amplitude of each query address in the vector (0 when absent): the
// address's segment is scanned
template <class K, int AMP>
__global__ void k_lookup(const RunDesc* __restrict__ R, const K* __restrict__ q, size_t n,
                         double* __restrict__ out) {
    typedef typename AmpT<AMP>::A A;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int cur = R->st->cur;
    const K key = q[i];
    const unsigned b = segment_of(seg_hash(key), R->log2B);
    const unsigned c = min(R->vcount[cur][b], R->Cv);
    const K* vk = (const K*)R->vkeys[cur] + (size_t)b * R->Cv;
    const A* va = (const A*)R->vamps[cur] + (size_t)b * R->Cv;
    double v = 0.0;
    for (unsigned j = 0; j < c; ++j)
        if (vk[j] == key) {
            v = (double)va[j];
            break;
        }
    out[i] = v;
}

// copy segments (counts from `cnt`, offsets `off`) into dense arrays
template <class K, class T>
__global__ void k_gather(const K* __restrict__ keys, const T* __restrict__ vals, unsigned cap,
                         const unsigned* __restrict__ cnt, const unsigned* __restrict__ off,
                         unsigned B, K* __restrict__ okeys, double* __restrict__ ovals,
                         const unsigned* __restrict__ segs) {
    for (unsigned x = blockIdx.x; x < B; x += gridDim.x) {
        const unsigned b = segs ? segs[x] : x;
        const unsigned n = min(cnt[b], cap), o = off[x];
        for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
            okeys[o + i] = keys[(size_t)b * cap + i];
            ovals[o + i] = (double)vals[(size_t)b * cap + i];
        }
    }
}

// the same for spawn buckets, in their layout
template <class K, class S>
__global__ void k_gather_spawns(const void* __restrict__ kb, const void* __restrict__ vb,
                                unsigned cap, unsigned Cp, const unsigned* __restrict__ cnt,
                                const unsigned* __restrict__ off, unsigned B, K* __restrict__ okeys,
                                double* __restrict__ ovals) {
    for (unsigned b = blockIdx.x; b < B; b += gridDim.x) {
        const unsigned n = min(cnt[b], cap), o = off[b];
        for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
            K key;
            S v;
            SpawnIO<K, S>::load(kb, vb, spawn_slot(b, i, Cp, cap, B), key, v);
            okeys[o + i] = key;
            ovals[o + i] = (double)v;
        }
    }
}

// diagonal, m and the whole column of one address (utility, single thread)
template <class K, int KIND>
__global__ void k_column(ModelParams mp, K key, K* dest, double* val, unsigned cap, double* diag,
                         unsigned* m_out) {
    if (threadIdx.x || blockIdx.x) return;
    typedef Model<KIND> MD;
    typename MD::Col col;
    const unsigned m = MD::num_offdiag(mp, key, col);
    *diag = MD::diagonal(mp, key);
    *m_out = m;
    for (unsigned k = 0; k < m && k < cap; ++k) dest[k] = MD::offdiag(mp, key, col, k, val[k]);
}

// projected-energy terms: for each reference address r with weight y_r, the
// term (r, y_r H_rr, y_r) followed by (j, y_r H_rj, 0) for its column
template <class K, int KIND>
__global__ void k_ref_terms(ModelParams mp, const K* __restrict__ refs, const double* __restrict__ y,
                            int n, const unsigned* __restrict__ off, K* tkeys, double* th,
                            double* tv, unsigned* tseg, int log2B) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    typedef Model<KIND> MD;
    typename MD::Col col;
    const K key = refs[r];
    const unsigned m = MD::num_offdiag(mp, key, col);
    unsigned o = off[r];
    tkeys[o] = key;
    th[o] = y[r] * MD::diagonal(mp, key);
    tv[o] = y[r];
    tseg[o] = segment_of(seg_hash(key), log2B);
    ++o;
    for (unsigned k = 0; k < m; ++k, ++o) {
        double hv;
        const K d = MD::offdiag(mp, key, col, k, hv);
        tkeys[o] = d;
        th[o] = y[r] * hv;
        tv[o] = 0.0;
        tseg[o] = segment_of(seg_hash(d), log2B);
    }
}

template <class K, int KIND>
__global__ void k_ref_count(ModelParams mp, const K* __restrict__ refs, int n, unsigned* m) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    typename Model<KIND>::Col col;
    m[r] = Model<KIND>::num_offdiag(mp, refs[r], col) + 1;
}

}  // namespace fq
