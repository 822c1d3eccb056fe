// fq_kernels.cuh -- the FCIQMC step as three kernels per step for a batch of
// independent runs (Rimu.jl paper, Eq. stochasticTransitionOperator):
//
//   k_spawn  For every occupied entry c_i of c^(n): decide an exact or a
//            stochastic column (|c_i| t_rel >= m_i, Sec. 7.1), then write the
//            column's spawns H_ji coef_i, coef_i = -dt c_i (exact) or
//            -dt (m_i / n_i) c_i for n_i = ceil|c_i| uniform picks (Eq.
//            column-compression), into the bucket owning each destination.
//   k_merge  For every bucket: put c^(n)'s segment, with the diagonal factor
//            1 + dt (S - H_ii) applied, and every spawn to the bucket into an
//            on-chip open-addressing table, which sums contributions per
//            address (annihilation); apply vector compression Pi (Eq.
//            vec-compression); compact the survivors into c^(n+1)'s
//            segment; accumulate ||c||_1 (exactly), len and the
//            projected-energy terms.
//   k_shift  One block per run: Eq. shift-update, a history row, the buffer
//            flip, and the diagonal-factor table of the next step.
//
// Layout: the vector of a run is hash-segmented (the paper's PDVec segments,
// Sec. 6.4, as thousands of small segments sized for one SM's shared
// memory): segment b = top log2(B) bits of fmix64(h(address)), capacity Cv
// entries each, structure-of-arrays keys/amplitudes.  Spawn buckets use the
// same segment map with capacity Cs.  All sizes and pointers are read from
// device memory, so one captured CUDA graph replays any number of steps.
//
// GB300 executes FP64 at a small fraction of its FP32/integer rate, so the
// kernels keep FP64 work to about one multiply per spawn and per entry (FP64
// amplitudes) or none (FP32 amplitudes); decisions whose result is exact are
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

// ---------------------------------------------------------------------------
// block-wide helpers (deterministic for a fixed block size)

template <int BLOCK>
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* s_warp, unsigned& total) {
    constexpr int NW = BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < NW ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[NW - 1];
    const unsigned r = x - v + (warp ? s_warp[warp - 1] : 0u);
    __syncthreads();
    return r;
}

template <int BLOCK, class T>
__device__ __forceinline__ T block_sum(T v, T* s_red) {
    constexpr int NW = BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    T r = 0;
    if (warp == 0) {
        r = lane < NW ? s_red[lane] : (T)0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xFFFFFFFFu, r, o);
    }
    __syncthreads();
    return r;  // valid in thread 0
}

// exact 128-bit sum over the block; valid in thread 0
template <int BLOCK>
__device__ __forceinline__ void block_sum128(unsigned long long& lo, unsigned long long& hi,
                                             unsigned long long* s_red) {
    constexpr int NW = BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long l = __shfl_down_sync(0xFFFFFFFFu, lo, o);
        const unsigned long long h = __shfl_down_sync(0xFFFFFFFFu, hi, o);
        add128(lo, hi, l, h);
    }
    if (lane == 0) {
        s_red[2 * warp] = lo;
        s_red[2 * warp + 1] = hi;
    }
    __syncthreads();
    if (warp == 0) {
        lo = lane < NW ? s_red[2 * lane] : 0ull;
        hi = lane < NW ? s_red[2 * lane + 1] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long l = __shfl_down_sync(0xFFFFFFFFu, lo, o);
            const unsigned long long h = __shfl_down_sync(0xFFFFFFFFu, hi, o);
            add128(lo, hi, l, h);
        }
    }
    __syncthreads();
}

// contiguous range of segments for this block
__device__ __forceinline__ void block_range(unsigned G, unsigned& g0, unsigned& g1) {
    g0 = (unsigned)(((unsigned long long)G * blockIdx.x) / gridDim.x);
    g1 = (unsigned)(((unsigned long long)G * (blockIdx.x + 1)) / gridDim.x);
}

// ---------------------------------------------------------------------------
// K1: spawning

template <class K, int AMP, int KIND, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK)
k_spawn(const RunDesc* __restrict__ runs, const unsigned* __restrict__ seg_run, unsigned G) {
    typedef typename AmpT<AMP>::A A;
    typedef typename AmpT<AMP>::S S;
    typedef typename AmpT<AMP>::C CO;
    typedef Model<KIND> MD;
    typedef typename MD::Col Col;
    constexpr int CH = BLOCK * IPT;
    __shared__ K s_key[CH];
    __shared__ CO s_coef[CH];
    __shared__ unsigned s_off[CH + 1];
    __shared__ unsigned s_m[CH];
    __shared__ unsigned s_warp[BLOCK / 32];
    __shared__ unsigned long long s_red[BLOCK / 32];
    __shared__ unsigned s_ctl[2];
    const int tid = threadIdx.x;
    unsigned g0, g1;
    block_range(G, g0, g1);

    const RunDesc* R = nullptr;
    int cur_r = -1;
    unsigned err = 0, cur = 0;
    unsigned long long n_ex = 0, n_inex = 0, n_sp = 0;

    for (unsigned g = g0; g < g1; ++g) {
        const int r = (int)seg_run[g];
        if (r != cur_r) {  // uniform: every thread reads the same r
            if (R) {
                const unsigned long long e = block_sum<BLOCK>(n_ex, s_red);
                const unsigned long long ie = block_sum<BLOCK>(n_inex, s_red);
                const unsigned long long sp = block_sum<BLOCK>(n_sp, s_red);
                if (tid == 0) {
                    if (e) atomicAdd(&R->st->n_exact, e);
                    if (ie) atomicAdd(&R->st->n_inexact, ie);
                    if (sp) atomicAdd(&R->st->n_spawns, sp);
                }
                n_ex = n_inex = n_sp = 0;
            }
            R = runs + r;
            cur_r = r;
            // one thread reads, all use the same values: another block may
            // set an error bit meanwhile
            if (tid == 0) {
                s_ctl[0] = *(volatile unsigned*)&R->st->err;
                s_ctl[1] = (unsigned)R->st->cur;
            }
            __syncthreads();
            err = s_ctl[0];
            cur = s_ctl[1];
            __syncthreads();
        }
        if (err) continue;
        const unsigned seg = g - R->seg_base;
        const unsigned n = R->vcount[cur][seg];
        if (n == 0) continue;

        const ModelParams& mp = R->mp;
        const K* __restrict__ vk = (const K*)R->vkeys[cur] + (size_t)seg * R->Cv;
        const A* __restrict__ va = (const A*)R->vamps[cur] + (size_t)seg * R->Cv;
        K* __restrict__ sk = (K*)R->skeys;
        S* __restrict__ sv = (S*)R->samps;
        unsigned* __restrict__ sfill = R->sfill;
        const unsigned Cs = R->Cs;
        const int log2B = R->log2B;
        const double dt = R->st->dt;
        const int det = R->mode_det, trel_one = R->trel_one;
        const double t_rel = R->t_rel;
        const int mmax = R->mmax;
        const unsigned stepno = (unsigned)(R->st->step + 1);
        const uint2 rkey = make_uint2(R->key_x, R->key_y);

        for (unsigned c0 = 0; c0 < n; c0 += CH) {
            const unsigned cn = min((unsigned)CH, n - c0);
            // stage keys and amplitudes (coalesced); amplitudes go through
            // s_coef, overwritten by the coefficients below
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                const unsigned i = j * BLOCK + tid;
                if (i < cn) {
                    s_key[i] = vk[c0 + i];
                    s_coef[i] = (CO)va[c0 + i];
                }
            }
            __syncthreads();
            unsigned cnt[IPT], tsum = 0;
            CO coef[IPT];
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                const unsigned i = tid * IPT + j;
                unsigned c_i = 0;
                coef[j] = (CO)0;
                if (i < cn) {
                    const K key = s_key[i];
                    const CO c = s_coef[i];
                    Col col;
                    const unsigned m = MD::num_offdiag(mp, key, col);
                    unsigned fl, ce;
                    floor_ceil_abs(c, fl, ce);
                    if (AMP == FQ_AMP_INT) {
                        // integer walkers: |c| attempts, never an exact column;
                        // the coefficient is dt m (spawn probability per |H_ji|)
                        c_i = m ? fl : 0u;
                        ++n_inex;
                        coef[j] = (CO)(dt * (double)m);
                        s_m[i] = m | (c < (CO)0 ? 0x40000000u : 0u);
                    } else {
                        bool ex;
                        if (det) ex = true;
                        else if (trel_one) ex = fl >= m;  // |c| >= m for an integer m
                        else ex = fabs((double)c) * t_rel >= (double)m;
                        c_i = ex ? m : ce;
                        if (ex) {
                            ++n_ex;
                            coef[j] = (-(CO)dt) * c;
                        } else {
                            ++n_inex;
                            CO ratio;
                            if (KIND != FQ_KIND_MOM_1D && (int)m <= mmax && (int)ce <= mmax) {
                                const size_t ri = (size_t)m * (size_t)(mmax + 1) + ce;
                                if constexpr (AMP == FQ_AMP_F32) ratio = __ldg(R->ratio32 + ri);
                                else ratio = __ldg(R->ratio64 + ri);
                            } else {
                                ratio = (CO)m / (CO)ce;
                            }
                            coef[j] = ((-(CO)dt) * ratio) * c;
                        }
                        s_m[i] = m | (ex ? 0x80000000u : 0u);
                    }
                }
                cnt[j] = c_i;
                tsum += c_i;
            }
            unsigned total;
            unsigned off = block_excl_scan<BLOCK>(tsum, s_warp, total);
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                s_off[tid * IPT + j] = off;
                s_coef[tid * IPT + j] = coef[j];
                off += cnt[j];
            }
            if (tid == 0) s_off[CH] = total;
            __syncthreads();

            // each thread takes a contiguous run of spawn indices
            const unsigned q0 = (unsigned)(((unsigned long long)total * tid) / BLOCK);
            const unsigned q1 = (unsigned)(((unsigned long long)total * (tid + 1)) / BLOCK);
            if (q0 < q1) {
                int i;
                {
                    int lo = 0, hi = CH - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (s_off[mid] <= q0) lo = mid; else hi = mid - 1;
                    }
                    i = lo;
                }
                K key = s_key[i];
                CO cf = s_coef[i];
                unsigned mm = s_m[i];
                unsigned end_i = s_off[i + 1];
                Col col;
                MD::num_offdiag(mp, key, col);
                for (unsigned q = q0; q < q1; ++q) {
                    if (q >= end_i) {
                        do { ++i; } while (q >= s_off[i + 1]);
                        key = s_key[i];
                        cf = s_coef[i];
                        mm = s_m[i];
                        end_i = s_off[i + 1];
                        MD::num_offdiag(mp, key, col);
                    }
                    const unsigned a = q - s_off[i];
                    const unsigned m = mm & 0x3FFFFFFFu;
                    const bool ex = (AMP != FQ_AMP_INT) && (mm >> 31);
                    uint4 w = make_uint4(0, 0, 0, 0);
                    unsigned kk = a;
                    if (!ex) {
                        w = draw(rkey, stepno, a, KeyOps<K>::rng_h(key));
                        kk = pick(w, m);
                    }
                    S val;
                    K dest;
                    if constexpr (AMP == FQ_AMP_INT) {
                        double hv;
                        dest = MD::offdiag(mp, key, col, kk, hv);
                        const double p = fabs(hv) * cf;
                        const double fl = floor(p);
                        const long long nw = (long long)fl + (uniform53(w) < p - fl ? 1 : 0);
                        if (!nw) continue;
                        const int sg = (hv > 0.0 ? -1 : 1) * ((mm & 0x40000000u) ? -1 : 1);
                        val = (S)(sg * nw);
                    } else {
                        CO hv;
                        dest = MD::offdiag(mp, key, col, kk, hv);
                        val = hv * cf;
                    }
                    ++n_sp;
                    const unsigned b = segment_of(fmix64(KeyOps<K>::rng_h(dest)), log2B);
                    const unsigned pos = atomicAdd(&sfill[b], 1u);
                    if (pos < Cs) {
                        sk[(size_t)b * Cs + pos] = dest;
                        sv[(size_t)b * Cs + pos] = val;
                    } else {
                        atomicOr(&R->st->err, FQ_DERR_SPAWN_CAP);
                    }
                }
            }
            __syncthreads();
        }
    }
    if (R) {
        const unsigned long long e = block_sum<BLOCK>(n_ex, s_red);
        const unsigned long long ie = block_sum<BLOCK>(n_inex, s_red);
        const unsigned long long sp = block_sum<BLOCK>(n_sp, s_red);
        if (tid == 0) {
            if (e) atomicAdd(&R->st->n_exact, e);
            if (ie) atomicAdd(&R->st->n_inexact, ie);
            if (sp) atomicAdd(&R->st->n_spawns, sp);
        }
    }
}

// ---------------------------------------------------------------------------
// on-chip open-addressing table (linear probing, CAS on the key)

__device__ __forceinline__ void acc_add(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void acc_add(float* p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void acc_add(long long* p, long long v) {
    atomicAdd((unsigned long long*)p, (unsigned long long)v);
}

__device__ __forceinline__ uint64_t key_cas(uint64_t* p, uint64_t cmp, uint64_t val) {
    return (uint64_t)atomicCAS((unsigned long long*)p, (unsigned long long)cmp,
                               (unsigned long long)val);
}
__device__ __forceinline__ u128 key_cas(u128* p, u128 cmp, u128 val) {
    return atomicCAS(p, cmp, val);
}

// slot of `key`, inserting it if absent (is_new set); -1 when the table is full
template <class K>
__device__ __forceinline__ int table_insert(K* tkey, unsigned mask, K key, bool& is_new) {
    const K EMPTY = KeyOps<K>::empty();
    unsigned q = (unsigned)fmix64(KeyOps<K>::rng_h(key)) & mask;
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
    unsigned q = (unsigned)fmix64(KeyOps<K>::rng_h(key)) & mask;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const K seen = tkey[q];
        if (seen == key) return (int)q;
        if (seen == EMPTY) return -1;
        q = (q + 1) & mask;
    }
    return -1;
}

// Pi (Eq. vec-compression) of one merged value: keep |w| >= theta, else
// sign(w) theta with probability |w| / theta.  `out` is the stored value.
template <int AMP>
__device__ __forceinline__ bool compress(typename AmpT<AMP>::ACC w, const RunDesc* R, uint2 rkey,
                                         unsigned stepno, uint64_t h,
                                         typename AmpT<AMP>::ACC& out) {
    typedef typename AmpT<AMP>::ACC ACC;
    if constexpr (AMP == FQ_AMP_INT) {
        out = w;
        return w != 0;
    } else {
        const unsigned long long ab = abs_dbits(w);
        if (R->mode_det) {
            out = w;
            return ab != 0;
        }
        if (ab == 0) return false;
        const double theta = R->theta;
        if (R->theta_pow2) {
            if (ab >= dbits(theta)) {
                out = w;
                return true;
            }
            const uint4 r = draw(rkey, stepno, 0xFFFFFFFFu, h);
            if (!below_scaled(u53_of(r), ab, R->theta_exp)) return false;
        } else {
            const double aw = bdouble(ab);
            if (aw >= theta) {
                out = w;
                return true;
            }
            const uint4 r = draw(rkey, stepno, 0xFFFFFFFFu, h);
            if (!(uniform53(r) < aw / theta)) return false;
        }
        out = w < (ACC)0 ? (ACC)(-theta) : (ACC)theta;
        return true;
    }
}

// add a block's share of one run's step totals to the run's accumulators
template <int BLOCK>
__device__ __forceinline__ void merge_flush(const RunDesc* R, unsigned long long nlo,
                                            unsigned long long nhi, unsigned long long nlen,
                                            double nfp, bool full, bool over, bool range_bad,
                                            unsigned long long* s_red, double* s_redd) {
    block_sum128<BLOCK>(nlo, nhi, s_red);
    const unsigned long long ln = block_sum<BLOCK>(nlen, s_red);
    const double fp = block_sum<BLOCK>(nfp, s_redd);
    const int f = __syncthreads_or(full), o = __syncthreads_or(over),
              b = __syncthreads_or(range_bad);
    if (threadIdx.x == 0) {
        const unsigned long long old = atomicAdd(&R->st->norm_lo, nlo);
        atomicAdd(&R->st->norm_hi, nhi + (old + nlo < old ? 1ull : 0ull));
        atomicAdd(&R->st->len_acc, ln);
        if (R->mode_det) atomicAdd(&R->st->norm_fp, fp);
        if (f) atomicOr(&R->st->err, FQ_DERR_TABLE);
        if (o) atomicOr(&R->st->err, FQ_DERR_VEC_CAP);
        if (b) atomicOr(&R->st->err, FQ_DERR_RANGE);
    }
}

// ---------------------------------------------------------------------------
// K4: diagonal update + annihilation + vector compression + compaction +
//     estimator accumulation, one bucket per block iteration

template <class K, int AMP, int KIND, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_merge(const RunDesc* __restrict__ runs, const unsigned* __restrict__ seg_run, unsigned G,
        unsigned SLOTS) {
    typedef typename AmpT<AMP>::A A;
    typedef typename AmpT<AMP>::S S;
    typedef typename AmpT<AMP>::ACC ACC;
    typedef Model<KIND> MD;
    extern __shared__ __align__(16) unsigned char smem[];
    K* tkey = (K*)smem;
    ACC* tacc = (ACC*)(smem + (size_t)SLOTS * sizeof(K));
    unsigned short* tlist = (unsigned short*)(smem + (size_t)SLOTS * (sizeof(K) + sizeof(ACC)));
    __shared__ unsigned long long s_red[2 * (BLOCK / 32)];
    __shared__ double s_redd[BLOCK / 32];
    __shared__ unsigned s_nlist, s_nout;
    __shared__ unsigned s_ctl[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned mask = SLOTS - 1;
    const K EMPTY = KeyOps<K>::empty();

    for (unsigned q = tid; q < SLOTS; q += BLOCK) {
        tkey[q] = EMPTY;
        tacc[q] = (ACC)0;
    }
    unsigned g0, g1;
    block_range(G, g0, g1);

    const RunDesc* R = nullptr;
    int cur_r = -1;
    unsigned err = 0, cur = 0;
    unsigned long long nlo = 0, nhi = 0, nlen = 0;
    double nfp = 0.0;
    bool range_bad = false, full = false, over = false;
    __syncthreads();

    for (unsigned g = g0; g < g1; ++g) {
        const int r = (int)seg_run[g];
        if (r != cur_r) {  // uniform
            if (R) {
                merge_flush<BLOCK>(R, nlo, nhi, nlen, nfp, full, over, range_bad, s_red, s_redd);
                nlo = nhi = nlen = 0;
                nfp = 0.0;
                full = over = range_bad = false;
            }
            R = runs + r;
            cur_r = r;
            // one thread reads, all use the same values: another block may
            // set an error bit meanwhile
            if (tid == 0) {
                s_ctl[0] = *(volatile unsigned*)&R->st->err;
                s_ctl[1] = (unsigned)R->st->cur;
            }
            __syncthreads();
            err = s_ctl[0];
            cur = s_ctl[1];
            __syncthreads();
        }
        if (err) continue;
        const unsigned seg = g - R->seg_base;
        const unsigned n_old = R->vcount[cur][seg];
        const unsigned n_sp = R->sfill[seg];
        const unsigned Cv = R->Cv;
        const K* __restrict__ vk = (const K*)R->vkeys[cur] + (size_t)seg * Cv;
        const A* __restrict__ va = (const A*)R->vamps[cur] + (size_t)seg * Cv;
        K* __restrict__ ok = (K*)R->vkeys[cur ^ 1] + (size_t)seg * Cv;
        A* __restrict__ oa = (A*)R->vamps[cur ^ 1] + (size_t)seg * Cv;
        const K* __restrict__ sk = (const K*)R->skeys + (size_t)seg * R->Cs;
        const S* __restrict__ sv = (const S*)R->samps + (size_t)seg * R->Cs;
        const unsigned stepno = (unsigned)(R->st->step + 1);
        const uint2 rkey = make_uint2(R->key_x, R->key_y);
        const int nq = R->norm_q;
        const int det = R->mode_det;
        if (tid == 0) {
            s_nlist = n_old;
            s_nout = 0;
        }

        // diagonal term c_i (1 + dt (S - H_ii)); integer walkers round it
        // stochastically
        for (unsigned i = tid; i < n_old; i += BLOCK) {
            const K key = vk[i];
            const A c = va[i];
            ACC d;
            if constexpr (KIND != FQ_KIND_MOM_1D) {
                const int s = MD::diag_index(key);
                if constexpr (AMP == FQ_AMP_F32) {
                    d = c + c * __ldg(R->del32 + s);
                } else if constexpr (AMP == FQ_AMP_F64) {
                    d = c * __ldg(R->fac64 + s);
                } else {
                    const double x = (double)c * __ldg(R->fac64 + s);
                    const double fl = floor(x);
                    const uint4 w = draw(rkey, stepno, 0xFFFFFFFEu, KeyOps<K>::rng_h(key));
                    d = (ACC)((long long)fl + (uniform53(w) < x - fl ? 1 : 0));
                }
            } else {
                const double hii = MD::diagonal(R->mp, key);
                const double S0 = R->st->shift, dt = R->st->dt;
                if constexpr (AMP == FQ_AMP_F32) {
                    d = c + c * (float)(dt * (S0 - hii));
                } else if constexpr (AMP == FQ_AMP_F64) {
                    d = c * (1.0 + dt * (S0 - hii));
                } else {
                    const double x = (double)c * (1.0 + dt * (S0 - hii));
                    const double fl = floor(x);
                    const uint4 w = draw(rkey, stepno, 0xFFFFFFFEu, KeyOps<K>::rng_h(key));
                    d = (ACC)((long long)fl + (uniform53(w) < x - fl ? 1 : 0));
                }
            }
            bool nw;
            const int q = table_insert(tkey, mask, key, nw);
            if (q < 0) {
                full = true;
                tlist[i] = 0;
            } else {
                tlist[i] = (unsigned short)q;
                tacc[q] = d;
            }
        }
        __syncthreads();
        // annihilation: every spawn to the bucket adds into its address
        for (unsigned j = tid; j < n_sp; j += BLOCK) {
            const K key = sk[j];
            const ACC v = (ACC)sv[j];
            bool nw;
            const int q = table_insert(tkey, mask, key, nw);
            if (q < 0) {
                full = true;
                continue;
            }
            if (nw) tlist[atomicAdd(&s_nlist, 1u)] = (unsigned short)q;
            acc_add(&tacc[q], v);
        }
        __syncthreads();
        const unsigned nl = s_nlist;

        // Pi over the used slots; survivors leave warp by warp
        for (unsigned base = (unsigned)warp * 32; base < nl; base += BLOCK) {
            const unsigned i = base + lane;
            bool keep = false;
            ACC out = (ACC)0;
            K key = EMPTY;
            int q = -1;
            if (i < nl) {
                q = tlist[i];
                key = tkey[q];
                keep = compress<AMP>(tacc[q], R, rkey, stepno, KeyOps<K>::rng_h(key), out);
                if (!keep) out = (ACC)0;
                tacc[q] = out;
            }
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
            unsigned pos0 = 0;
            if (lane == 0 && bal) pos0 = atomicAdd(&s_nout, (unsigned)__popc(bal));
            pos0 = __shfl_sync(0xFFFFFFFFu, pos0, 0);
            if (keep) {
                const unsigned pos = pos0 + (unsigned)__popc(bal & ((1u << lane) - 1u));
                if (pos < Cv) {
                    ok[pos] = key;
                    oa[pos] = (A)out;
                } else {
                    over = true;
                }
                ++nlen;
                if constexpr (AMP == FQ_AMP_INT) {
                    const unsigned long long a = (unsigned long long)(out < 0 ? -out : out);
                    add128(nlo, nhi, a, 0ull);
                } else {
                    if (det) {
                        nfp += fabs((double)out);
                    } else {
                        unsigned long long lo, hi;
                        fixed_of(out, nq, lo, hi, range_bad);
                        add128(nlo, nhi, lo, hi);
                    }
                }
            }
        }
        __syncthreads();
        // projected-energy terms whose address falls in this bucket
        const unsigned e0 = R->ref_off[seg], e1 = R->ref_off[seg + 1];
        if (e1 > e0) {  // uniform
            double hp = 0.0, vp = 0.0;
            const K* rk = (const K*)R->ref_keys;
            for (unsigned e = e0 + tid; e < e1; e += BLOCK) {
                const int q = table_find(tkey, mask, rk[e]);
                const double cv = q >= 0 ? (double)tacc[q] : 0.0;
                hp += R->ref_h[e] * cv;
                vp += R->ref_v[e] * cv;
            }
            const double bh = block_sum<BLOCK>(hp, s_redd);
            const double bv = block_sum<BLOCK>(vp, s_redd);
            if (tid == 0) {
                R->part_h[seg] = bh;
                R->part_v[seg] = bv;
            }
        }
        // release the used slots for the next bucket
        for (unsigned i = tid; i < nl; i += BLOCK) {
            const unsigned q = tlist[i];
            tkey[q] = EMPTY;
            tacc[q] = (ACC)0;
        }
        if (tid == 0) {
            const unsigned nout = s_nout;
            R->vcount[cur ^ 1][seg] = nout <= Cv ? nout : Cv;
            R->sfill[seg] = 0u;
        }
        __syncthreads();
    }
    if (R) merge_flush<BLOCK>(R, nlo, nhi, nlen, nfp, full, over, range_bad, s_red, s_redd);
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

static __global__ void k_factors(const RunDesc* __restrict__ runs) {
    const RunDesc* R = runs + blockIdx.x;
    if (R->smax >= 0 && R->fac64) write_factors(R, R->st->shift, R->st->dt);
}

// ---------------------------------------------------------------------------
// K5: shift update (Eq. shift-update), one block per run

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_shift(const RunDesc* __restrict__ runs) {
    const RunDesc* R = runs + blockIdx.x;
    RunState* st = R->st;
    __shared__ double s_S;
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        s_ok = 0;
        if (!*(volatile unsigned*)&st->err) {
            double nrm;
            if (R->mode_det) nrm = st->norm_fp;
            else nrm = fixed_to_double(st->norm_lo, st->norm_hi, R->norm_q);
            const unsigned long long len = st->len_acc;
            double hp = 0.0, vp = 0.0;
            for (unsigned i = 0; i < R->n_ref_bkt; ++i) {
                hp += R->part_h[R->ref_bkt[i]];
                vp += R->part_v[R->ref_bkt[i]];
            }
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
// set-up and read-out helpers (not on the per-step path)

// sqrt(k), -(t sqrt(k)) and its FP32 rounding for k <= kmax; m / n in FP64
// and FP32 for 1 <= n <= m <= mmax
static __global__ void k_tables(double t, int kmax, double* sq, double* hop, float* hop32, int mmax,
                         double* r64, float* r32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= kmax) {
        const double s = sqrt((double)i);
        sq[i] = s;
        hop[i] = -(t * s);
        hop32[i] = (float)hop[i];
    }
    if (r64 && i < (mmax + 1) * (mmax + 1)) {
        const int m = i / (mmax + 1), n = i % (mmax + 1);
        r64[i] = n ? (double)m / (double)n : 0.0;
        r32[i] = n ? (float)m / (float)n : 0.0f;
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
    const unsigned b = segment_of(fmix64(KeyOps<K>::rng_h(key)), R->log2B);
    const unsigned pos = atomicAdd(&R->vcount[cur][b], 1u);
    if (pos < R->Cv) {
        ((K*)R->vkeys[cur])[(size_t)b * R->Cv + pos] = key;
        ((A*)R->vamps[cur])[(size_t)b * R->Cv + pos] = (A)amps[i];
    } else {
        atomicOr(&R->st->err, FQ_DERR_VEC_CAP);
    }
}

// copy segments (counts from `cnt`, offsets `off`) into dense arrays
template <class K, class T>
__global__ void k_gather(const K* __restrict__ keys, const T* __restrict__ vals, unsigned cap,
                         const unsigned* __restrict__ cnt, const unsigned* __restrict__ off,
                         unsigned B, K* __restrict__ okeys, double* __restrict__ ovals) {
    for (unsigned b = blockIdx.x; b < B; b += gridDim.x) {
        const unsigned n = min(cnt[b], cap), o = off[b];
        for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
            okeys[o + i] = keys[(size_t)b * cap + i];
            ovals[o + i] = (double)vals[(size_t)b * cap + i];
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
    tseg[o] = segment_of(fmix64(KeyOps<K>::rng_h(key)), log2B);
    ++o;
    for (unsigned k = 0; k < m; ++k, ++o) {
        double hv;
        const K d = MD::offdiag(mp, key, col, k, hv);
        tkeys[o] = d;
        th[o] = y[r] * hv;
        tv[o] = 0.0;
        tseg[o] = segment_of(fmix64(KeyOps<K>::rng_h(d)), log2B);
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
