// fq_kernels.cuh -- the FCIQMC step as three kernels per step for a batch of
// independent runs (Rimu.jl paper, Eq. stochasticTransitionOperator):
//
//   k_spawn  For every occupied entry c_i of c^(n): decide an exact or a
//            stochastic column (|c_i| t_rel >= m_i, Sec. 7.1), then write the
//            column's spawns -dt H_ji c_i (exact) or n_i = ceil|c_i| uniform
//            picks scaled by m_i/n_i (Eq. column-compression) into the bucket
//            that owns each destination address.
//   k_merge  For every bucket: put c^(n)'s segment, with the diagonal factor
//            1 + dt (S - H_ii) applied, and every spawn to the bucket into an
//            on-chip open-addressing table, which sums contributions per
//            address (annihilation); apply vector compression Pi (Eq.
//            vec-compression); compact the survivors into c^(n+1)'s
//            segment; reduce ||c||_1, len and the projected-energy terms.
//   k_shift  One block per run: reduce the per-segment partial sums in a
//            fixed order, apply Eq. shift-update, append a history row and
//            flip the vector buffers.
//
// Layout: the vector of a run is hash-segmented (the paper's PDVec segments,
// Sec. 6.4, with thousands of small segments sized for one SM's shared
// memory): segment b = top log2(B) bits of fmix64(h(address)), capacity Cv
// entries each, structure-of-arrays keys/amplitudes.  Spawn buckets use the
// same segment map with capacity Cs.  All sizes and pointers are read from
// device memory, so one captured CUDA graph replays any number of steps.
#pragma once

#include <cuda_runtime.h>

#include "fq_device.cuh"
#include "fq_shared.h"

namespace fq {

template <int AMP> struct AmpT;
template <> struct AmpT<FQ_AMP_INT> { typedef long long A; typedef int S; typedef long long ACC; };
template <> struct AmpT<FQ_AMP_F64> { typedef double A; typedef double S; typedef double ACC; };
template <> struct AmpT<FQ_AMP_F32> { typedef float A; typedef float S; typedef double ACC; };

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

// ---------------------------------------------------------------------------
// K1: spawning

template <class K, int AMP, int KIND, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK)
k_spawn(const RunDesc* __restrict__ runs, const unsigned* __restrict__ seg_run, unsigned G) {
    typedef typename AmpT<AMP>::A A;
    typedef typename AmpT<AMP>::S S;
    typedef Model<KIND> MD;
    typedef typename MD::Col Col;
    constexpr int CH = BLOCK * IPT;
    __shared__ K s_key[CH];
    __shared__ double s_amp[CH];
    __shared__ unsigned s_off[CH + 1];
    __shared__ unsigned s_m[CH];
    __shared__ unsigned s_warp[BLOCK / 32];
    __shared__ unsigned long long s_red[BLOCK / 32];
    __shared__ unsigned s_ctl[4];
    const int tid = threadIdx.x;

    for (unsigned g = blockIdx.x; g < G; g += gridDim.x) {
        const RunDesc* R = runs + seg_run[g];
        const unsigned seg = g - R->seg_base;
        RunState* st = R->st;
        if (tid == 0) {
            const int cur = st->cur;
            s_ctl[0] = *(volatile unsigned*)&st->err;
            s_ctl[1] = (unsigned)cur;
            s_ctl[2] = R->vcount[cur][seg];
        }
        __syncthreads();
        const unsigned err = s_ctl[0], cur = s_ctl[1], n = s_ctl[2];
        __syncthreads();
        if (err || n == 0) continue;

        const ModelParams& mp = R->mp;
        const K* __restrict__ vk = (const K*)R->vkeys[cur] + (size_t)seg * R->Cv;
        const A* __restrict__ va = (const A*)R->vamps[cur] + (size_t)seg * R->Cv;
        K* __restrict__ sk = (K*)R->skeys;
        S* __restrict__ sv = (S*)R->samps;
        unsigned* __restrict__ sfill = R->sfill;
        const unsigned Cs = R->Cs;
        const int log2B = R->log2B;
        const double dt = st->dt, t_rel = R->t_rel;
        const int det = R->mode_det;
        const unsigned stepno = (unsigned)(st->step + 1);
        const uint2 rkey = make_uint2(R->key_x, R->key_y);
        unsigned long long n_ex = 0, n_inex = 0, n_sp = 0;

        for (unsigned c0 = 0; c0 < n; c0 += CH) {
            const unsigned cn = min((unsigned)CH, n - c0);
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                const unsigned i = j * BLOCK + tid;
                if (i < cn) {
                    s_key[i] = vk[c0 + i];
                    s_amp[i] = (double)va[c0 + i];
                }
            }
            __syncthreads();
            unsigned cnt[IPT], tsum = 0;
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                const unsigned i = tid * IPT + j;
                unsigned c_i = 0;
                if (i < cn) {
                    const K key = s_key[i];
                    const double c = s_amp[i];
                    Col col;
                    const unsigned m = MD::num_offdiag(mp, key, col);
                    if (AMP == FQ_AMP_INT) {
                        // integer walkers: |c| attempts, never an exact column
                        c_i = m ? (unsigned)fabs(c) : 0u;
                        ++n_inex;
                        s_m[i] = m;
                    } else {
                        const bool ex = det || fabs(c) * t_rel >= (double)m;
                        c_i = ex ? m : (unsigned)ceil(fabs(c));
                        if (ex) ++n_ex; else ++n_inex;
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
                off += cnt[j];
            }
            if (tid == 0) s_off[CH] = total;
            __syncthreads();

            for (unsigned q = tid; q < total; q += BLOCK) {
                int lo = 0, hi = CH - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_off[mid] <= q) lo = mid; else hi = mid - 1;
                }
                const unsigned a = q - s_off[lo];
                const K key = s_key[lo];
                const double c = s_amp[lo];
                const unsigned mm = s_m[lo];
                const unsigned m = mm & 0x7FFFFFFFu;
                const bool ex = (AMP != FQ_AMP_INT) && (mm >> 31);
                Col col;
                MD::num_offdiag(mp, key, col);
                uint4 w = make_uint4(0, 0, 0, 0);
                unsigned kk = a;
                if (!ex) {
                    w = draw(rkey, stepno, a, KeyOps<K>::rng_h(key));
                    kk = pick(w, m);
                }
                double hv;
                const K dest = MD::offdiag(mp, key, col, kk, hv);
                S val;
                if (AMP == FQ_AMP_INT) {
                    const double p = (dt * fabs(hv)) * (double)m;
                    const double fl = floor(p);
                    const long long nw = (long long)fl + (uniform53(w) < p - fl ? 1 : 0);
                    if (!nw) continue;
                    const int sg = (hv > 0.0 ? -1 : 1) * (c > 0.0 ? 1 : -1);
                    val = (S)(sg * nw);
                } else if (ex) {
                    val = (S)((-(dt * hv)) * c);
                } else {
                    const double scale = (double)m / ceil(fabs(c));
                    val = (S)(((-(dt * hv)) * scale) * c);
                }
                ++n_sp;
                const unsigned b = segment_of(fmix64(KeyOps<K>::rng_h(dest)), log2B);
                const unsigned pos = atomicAdd(&sfill[b], 1u);
                if (pos < Cs) {
                    sk[(size_t)b * Cs + pos] = dest;
                    sv[(size_t)b * Cs + pos] = val;
                } else {
                    atomicOr(&st->err, FQ_DERR_SPAWN_CAP);
                }
            }
            __syncthreads();
        }
        const unsigned long long e = block_sum<BLOCK>(n_ex, s_red);
        const unsigned long long ie = block_sum<BLOCK>(n_inex, s_red);
        const unsigned long long sp = block_sum<BLOCK>(n_sp, s_red);
        if (tid == 0) {
            if (e) atomicAdd(&st->n_exact, e);
            if (ie) atomicAdd(&st->n_inexact, ie);
            if (sp) atomicAdd(&st->n_spawns, sp);
        }
    }
}

// ---------------------------------------------------------------------------
// accumulation into a table slot: FP64 add, or a two's-complement add for
// integer walkers (exact in any order)
__device__ __forceinline__ void acc_add(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void acc_add(long long* p, long long v) {
    atomicAdd((unsigned long long*)p, (unsigned long long)v);
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

template <class K>
__device__ __forceinline__ int table_insert(K* tkey, unsigned mask, K key) {
    const K EMPTY = KeyOps<K>::empty();
    unsigned q = (unsigned)fmix64(KeyOps<K>::rng_h(key)) & mask;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const K seen = tkey[q];
        if (seen == key) return (int)q;
        if (seen == EMPTY) {
            const K old = key_cas(&tkey[q], EMPTY, key);
            if (old == EMPTY || old == key) return (int)q;
        }
        q = (q + 1) & mask;
    }
    return -1;  // table full
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

// ---------------------------------------------------------------------------
// K4: diagonal update + annihilation + vector compression + compaction +
//     estimator partial sums, one bucket per block iteration

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
    __shared__ unsigned s_warp[BLOCK / 32];
    __shared__ double s_redd[BLOCK / 32];
    __shared__ unsigned s_ctl[4];
    const int tid = threadIdx.x;
    const unsigned mask = SLOTS - 1;
    const unsigned spt = SLOTS / BLOCK;
    const K EMPTY = KeyOps<K>::empty();

    for (unsigned g = blockIdx.x; g < G; g += gridDim.x) {
        const RunDesc* R = runs + seg_run[g];
        const unsigned seg = g - R->seg_base;
        RunState* st = R->st;
        if (tid == 0) {
            const int cur = st->cur;
            s_ctl[0] = *(volatile unsigned*)&st->err;
            s_ctl[1] = (unsigned)cur;
            s_ctl[2] = R->vcount[cur][seg];
            s_ctl[3] = R->sfill[seg];
        }
        __syncthreads();
        const unsigned err = s_ctl[0], cur = s_ctl[1], n_old = s_ctl[2], n_sp = s_ctl[3];
        __syncthreads();
        if (err) continue;

        const ModelParams& mp = R->mp;
        const unsigned Cv = R->Cv;
        const K* __restrict__ vk = (const K*)R->vkeys[cur] + (size_t)seg * Cv;
        const A* __restrict__ va = (const A*)R->vamps[cur] + (size_t)seg * Cv;
        K* __restrict__ ok = (K*)R->vkeys[cur ^ 1] + (size_t)seg * Cv;
        A* __restrict__ oa = (A*)R->vamps[cur ^ 1] + (size_t)seg * Cv;
        const K* __restrict__ sk = (const K*)R->skeys + (size_t)seg * R->Cs;
        const S* __restrict__ sv = (const S*)R->samps + (size_t)seg * R->Cs;
        const double S0 = st->shift, dt = st->dt, theta = R->theta;
        const int det = R->mode_det;
        const unsigned stepno = (unsigned)(st->step + 1);
        const uint2 rkey = make_uint2(R->key_x, R->key_y);

        for (unsigned q = tid; q < SLOTS; q += BLOCK) {
            tkey[q] = EMPTY;
            tacc[q] = (ACC)0;
        }
        __syncthreads();

        // diagonal term c_i (1 + dt (S - H_ii)); integer walkers round it
        // stochastically
        bool full = false;
        for (unsigned i = tid; i < n_old; i += BLOCK) {
            const K key = vk[i];
            const double c = (double)va[i];
            const double hii = MD::diagonal(mp, key);
            const double x = c * (1.0 + dt * (S0 - hii));
            ACC d;
            if (AMP == FQ_AMP_INT) {
                const double fl = floor(x);
                const uint4 w = draw(rkey, stepno, 0xFFFFFFFEu, KeyOps<K>::rng_h(key));
                d = (ACC)((long long)fl + (uniform53(w) < x - fl ? 1 : 0));
            } else {
                d = (ACC)x;
            }
            const int q = table_insert(tkey, mask, key);
            if (q < 0) full = true; else tacc[q] = d;
        }
        __syncthreads();
        // annihilation: every spawn to the bucket adds into its address
        for (unsigned j = tid; j < n_sp; j += BLOCK) {
            const K key = sk[j];
            const ACC v = (ACC)sv[j];
            const int q = table_insert(tkey, mask, key);
            if (q < 0) full = true; else acc_add(&tacc[q], v);
        }
        if (full) atomicOr(&st->err, FQ_DERR_TABLE);
        __syncthreads();

        // vector compression Pi on each merged value; kept values are
        // written back so that estimator lookups see c^(n+1)
        unsigned kept = 0;
        double nrm = 0.0;
        const unsigned q0 = tid * spt;
        for (unsigned q = q0; q < q0 + spt; ++q) {
            const K key = tkey[q];
            if (key == EMPTY) continue;
            const ACC w = tacc[q];
            if (AMP == FQ_AMP_INT) {
                if (w != 0) { ++kept; nrm += fabs((double)w); }
            } else if (det) {
                if (w != 0.0) { ++kept; nrm += fabs((double)w); }
            } else {
                const double aw = fabs((double)w);
                double out = 0.0;
                if (aw >= theta) {
                    out = (double)w;
                } else if (aw > 0.0) {
                    const uint4 r = draw(rkey, stepno, 0xFFFFFFFFu, KeyOps<K>::rng_h(key));
                    if (uniform53(r) < aw / theta) out = copysign(theta, (double)w);
                }
                if (AMP == FQ_AMP_F32) out = (double)(float)out;
                tacc[q] = (ACC)out;
                if (out != 0.0) { ++kept; nrm += fabs(out); }
            }
        }
        unsigned total;
        unsigned off = block_excl_scan<BLOCK>(kept, s_warp, total);
        const bool fits = total <= Cv;
        if (fits) {
            for (unsigned q = q0; q < q0 + spt; ++q) {
                const K key = tkey[q];
                if (key == EMPTY) continue;
                const ACC w = tacc[q];
                if (w != (ACC)0) {
                    ok[off] = key;
                    oa[off] = (A)w;
                    ++off;
                }
            }
        }
        __syncthreads();
        // projected-energy terms whose address falls in this bucket
        double hp = 0.0, vp = 0.0;
        const unsigned e0 = R->ref_off[seg], e1 = R->ref_off[seg + 1];
        const K* rk = (const K*)R->ref_keys;
        for (unsigned e = e0 + tid; e < e1; e += BLOCK) {
            const int q = table_find(tkey, mask, rk[e]);
            const double cv = q >= 0 ? (double)tacc[q] : 0.0;
            hp += R->ref_h[e] * cv;
            vp += R->ref_v[e] * cv;
        }
        const double bn = block_sum<BLOCK>(nrm, s_redd);
        const double bh = block_sum<BLOCK>(hp, s_redd);
        const double bv = block_sum<BLOCK>(vp, s_redd);
        if (tid == 0) {
            if (!fits) atomicOr(&st->err, FQ_DERR_VEC_CAP);
            R->vcount[cur ^ 1][seg] = fits ? total : 0u;
            R->part_norm[seg] = bn;
            R->part_len[seg] = total;
            R->part_h[seg] = bh;
            R->part_v[seg] = bv;
            R->sfill[seg] = 0u;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// K5: shift update (Eq. shift-update), one block per run

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_shift(const RunDesc* __restrict__ runs) {
    const RunDesc* R = runs + blockIdx.x;
    RunState* st = R->st;
    __shared__ double s_redd[BLOCK / 32];
    __shared__ unsigned long long s_redl[BLOCK / 32];
    if (*(volatile unsigned*)&st->err) return;
    double nrm = 0.0, hp = 0.0, vp = 0.0;
    unsigned long long len = 0;
    for (unsigned s = threadIdx.x; s < R->B; s += BLOCK) {
        nrm += R->part_norm[s];
        hp += R->part_h[s];
        vp += R->part_v[s];
        len += R->part_len[s];
    }
    nrm = block_sum<BLOCK>(nrm, s_redd);
    hp = block_sum<BLOCK>(hp, s_redd);
    vp = block_sum<BLOCK>(vp, s_redd);
    len = block_sum<BLOCK>(len, s_redl);
    if (threadIdx.x != 0) return;
    if (nrm == 0.0 || len == 0) {
        st->err |= FQ_DERR_EMPTY;
        return;
    }
    const double dt = st->dt;
    const double zd = st->zeta / dt, xd = st->xi / dt;
    const double S1 = (st->shift - zd * log(nrm / st->norm)) - xd * log(nrm / st->target);
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
    st->n_exact = 0;
    st->n_inexact = 0;
    st->n_spawns = 0;
}

// ---------------------------------------------------------------------------
// set-up and read-out helpers (not on the per-step path)

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
