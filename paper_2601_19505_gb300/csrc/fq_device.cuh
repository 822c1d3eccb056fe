// fq_device.cuh -- device-side building blocks of the FCIQMC step:
// Fock-address bit operations, the Bose-Hubbard Hamiltonians evaluated
// column by column, Philox4x32-10 draws keyed by content, and hashing.
//
// Addresses (Sec. 6.1 of the Rimu.jl paper): a bit string of N + M - 1 bits,
// n_m ones for mode m, one zero between consecutive modes, mode 0 at the
// least significant bit.  Keys are uint64_t when N + M - 1 <= 64, else
// unsigned __int128.  Every bit that is not part of the address is 0, so
// the M - 1 separators are the M - 1 lowest zero bits of the key.
//
// Everything here is compiled without FMA contraction (--fmad=false) so that
// each floating-point expression rounds exactly as written.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fq_shared.h"

namespace fq {

typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------
// bit helpers

__device__ __forceinline__ int nth_set64(uint64_t x, int j) {
    // position of the j-th (0-based) set bit of x; requires j < popc(x)
    int pos = 0, c;
    c = __popc((unsigned)x);
    if (j >= c) { j -= c; x >>= 32; pos += 32; }
    c = __popc((unsigned)(x & 0xFFFFu));
    if (j >= c) { j -= c; x >>= 16; pos += 16; }
    c = __popc((unsigned)(x & 0xFFu));
    if (j >= c) { j -= c; x >>= 8; pos += 8; }
    c = __popc((unsigned)(x & 0xFu));
    if (j >= c) { j -= c; x >>= 4; pos += 4; }
    c = __popc((unsigned)(x & 0x3u));
    if (j >= c) { j -= c; x >>= 2; pos += 2; }
    c = (int)(x & 1u);
    if (j >= c) pos += 1;
    return pos;
}

template <class K> struct KeyOps;

template <> struct KeyOps<uint64_t> {
    static constexpr int W = 64;
    __device__ __forceinline__ static uint64_t empty() { return ~0ull; }
    __device__ __forceinline__ static int popc(uint64_t k) { return __popcll(k); }
    __device__ __forceinline__ static int nth(uint64_t k, int j) { return nth_set64(k, j); }
    __device__ __forceinline__ static uint64_t shr(uint64_t x, int s) { return s >= 64 ? 0ull : x >> s; }
    __device__ __forceinline__ static uint64_t shl(uint64_t x, int s) { return s >= 64 ? 0ull : x << s; }
    __device__ __forceinline__ static uint64_t low(int p) { return p >= 64 ? ~0ull : ((1ull << p) - 1ull); }
    __device__ __forceinline__ static int ctz(uint64_t x) { return x ? __ffsll((long long)x) - 1 : 64; }
    __device__ __forceinline__ static uint64_t bit(int p) { return 1ull << p; }
    __device__ __forceinline__ static uint64_t rng_h(uint64_t k) { return k; }
};

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    // splitmix64 (Steele, Lea, Flood 2014)
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// 128-bit addresses.  Shifts by a variable amount are written out on the two
// 64-bit halves, with the amounts 0, 64 and >= 128 taken explicitly: the
// compiled unsigned __int128 shift by exactly 64 bits produced a wrong low
// word (bit(64) came out as bits 0 and 64), which corrupted hops whose bit
// position is 64.  Shifts by a constant stay on the 128-bit type.
template <> struct KeyOps<u128> {
    static constexpr int W = 128;
    __device__ __forceinline__ static u128 make(uint64_t lo, uint64_t hi) {
        return ((u128)hi << 64) | (u128)lo;
    }
    __device__ __forceinline__ static u128 empty() { return ~(u128)0; }
    __device__ __forceinline__ static int popc(u128 k) {
        return __popcll((uint64_t)k) + __popcll((uint64_t)(k >> 64));
    }
    // the word is selected first, so one 64-bit search runs
    __device__ __forceinline__ static int nth(u128 k, int j) {
        const uint64_t lo = (uint64_t)k, hi = (uint64_t)(k >> 64);
        const int c = __popcll(lo);
        const bool in_lo = j < c;
        return (in_lo ? 0 : 64) + nth_set64(in_lo ? lo : hi, in_lo ? j : j - c);
    }
    // s >= 0; every 64-bit shift below is by 0..63 and the cases are
    // selected, not branched to (lanes of a warp take different amounts)
    __device__ __forceinline__ static u128 shr(u128 x, int s) {
        const uint64_t lo = (uint64_t)x, hi = (uint64_t)(x >> 64);
        const int s1 = s & 63;
        const uint64_t cross = s1 ? hi << (64 - s1) : 0ull;
        const uint64_t nlo = s < 64 ? (lo >> s1) | cross : (s < 128 ? hi >> s1 : 0ull);
        const uint64_t nhi = s < 64 ? hi >> s1 : 0ull;
        return make(nlo, nhi);
    }
    __device__ __forceinline__ static u128 shl(u128 x, int s) {
        const uint64_t lo = (uint64_t)x, hi = (uint64_t)(x >> 64);
        const int s1 = s & 63;
        const uint64_t cross = s1 ? lo >> (64 - s1) : 0ull;
        const uint64_t nlo = s < 64 ? lo << s1 : 0ull;
        const uint64_t nhi = s < 64 ? (hi << s1) | cross : (s < 128 ? lo << s1 : 0ull);
        return make(nlo, nhi);
    }
    // bits 0 .. p - 1 (0 <= p <= 128)
    __device__ __forceinline__ static u128 low(int p) {
        const uint64_t m = (1ull << (p & 63)) - 1ull;
        return make(p >= 64 ? ~0ull : m, p >= 128 ? ~0ull : (p >= 64 ? m : 0ull));
    }
    __device__ __forceinline__ static int ctz(u128 x) {
        const uint64_t lo = (uint64_t)x, hi = (uint64_t)(x >> 64);
        const int a = __ffsll((long long)lo) - 1, b = __ffsll((long long)hi) - 1;
        return lo ? a : (hi ? 64 + b : 128);
    }
    __device__ __forceinline__ static u128 bit(int p) {
        const uint64_t b = 1ull << (p & 63);
        return make(p < 64 ? b : 0ull, p < 64 ? 0ull : b);
    }
    __device__ __forceinline__ static uint64_t rng_h(u128 k) {
        return (uint64_t)k ^ splitmix64((uint64_t)(k >> 64));
    }
};

__device__ __forceinline__ int clz_k(uint64_t x) { return __clzll((long long)x); }
__device__ __forceinline__ int clz_k(u128 x) {
    const uint64_t hi = (uint64_t)(x >> 64);
    return hi ? __clzll((long long)hi) : 64 + __clzll((long long)(uint64_t)x);
}

// start bit of mode s (0-based): one past the s-th separator
template <class K> __device__ __forceinline__ int mode_start(K k, int s) {
    return s == 0 ? 0 : KeyOps<K>::nth(~k, s - 1) + 1;
}
// length of the run of ones starting at bit p
template <class K> __device__ __forceinline__ int run_from(K k, int p) {
    return KeyOps<K>::ctz(~KeyOps<K>::shr(k, p));
}
template <class K> __device__ __forceinline__ int mode_occ(K k, int s) {
    return run_from(k, mode_start(k, s));
}
// remove the bit at p, shifting the higher bits down
template <class K> __device__ __forceinline__ K del_bit(K x, int p) {
    typedef KeyOps<K> O;
    return (x & O::low(p)) | O::shl(O::shr(x, p + 1), p);
}
// insert a one at p, shifting bits >= p up
template <class K> __device__ __forceinline__ K ins_one(K x, int p) {
    typedef KeyOps<K> O;
    return (x & O::low(p)) | O::bit(p) | O::shl(O::shr(x, p), p + 1);
}
template <class K> __device__ __forceinline__ K remove_boson(K k, int s) {
    return del_bit(k, mode_start(k, s));
}
template <class K> __device__ __forceinline__ K add_boson(K k, int s) {
    return ins_one(k, mode_start(k, s));
}
// bits that start a run of ones: one per occupied mode
template <class K> __device__ __forceinline__ K run_starts(K k) { return k & ~(k << 1); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the draw layout:
//   key     = (seed_lo32, seed_hi32 ^ run_id * 0x9E3779B9)
//   counter = (step, stream, h_lo32, h_hi32), h = KeyOps<K>::rng_h(address)
//   stream  = attempt index for picks, 0xFFFFFFFF for vector compression,
//             0xFFFFFFFE for integer diagonal rounding, 0xFFFFFFFD for the
//             early compression of a diagonal term (a spawn's early
//             compression reuses the draw of its pick, or of stream k for
//             entry k of an exact column)

__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        // one 32 x 32 -> 64-bit product gives both halves
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        const unsigned lo0 = (unsigned)p0, hi0 = (unsigned)(p0 >> 32);
        const unsigned lo1 = (unsigned)p1, hi1 = (unsigned)(p1 >> 32);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw(uint2 key, unsigned step, unsigned stream, uint64_t h) {
    return philox10(make_uint4(step, stream, (unsigned)h, (unsigned)(h >> 32)), key);
}
// uniform in [0, 1) with 53 random bits, exact in FP64
__device__ __forceinline__ double uniform53(uint4 w) {
    return ((double)(w.x >> 5) * 67108864.0 + (double)(w.y >> 6)) * (1.0 / 9007199254740992.0);
}
// index in [0, m)
__device__ __forceinline__ unsigned pick(uint4 w, unsigned m) {
    return (unsigned)(((unsigned long long)w.z * (unsigned long long)m) >> 32);
}

// segment hash; the segment is the top bits.  64-bit addresses: one
// multiply by an odd constant (multiplicative hashing), unrelated to the
// golden-ratio constant of the merge table's slot hash (with related
// constants, small addresses that share a segment would also share a few
// table slots).
// 128-bit addresses fold the high word in by a multiply with another odd
// constant, then take the same multiply: two 64-bit multiplies in all.
__device__ __forceinline__ uint64_t seg_hash(uint64_t k) { return k * 0xD6E8FEB86659FD93ull; }
__device__ __forceinline__ uint64_t seg_hash(u128 k) {
    return ((uint64_t)k ^ ((uint64_t)(k >> 64) * 0xC2B2AE3D27D4EB4Full)) * 0xD6E8FEB86659FD93ull;
}
__device__ __forceinline__ unsigned segment_of(uint64_t mixed, int log2B) {
    return log2B ? (unsigned)(mixed >> (64 - log2B)) : 0u;
}

// ---------------------------------------------------------------------------
// Hamiltonians

template <int KIND> struct Model;

// Real space (Eq. bose-hubbard-hamiltonian): H_ii = (u/2) sum n(n-1); each
// (direction, occupied site) pair hops one boson to a neighbour with value
// -t sqrt(n_s (n_s' + 1)).  Entry k: direction k / n_occ, occupied site
// k mod n_occ (ascending); directions (+1, -1) in 1D, (+x, -x, +y, -y) in 2D.
template <int KIND> struct RealModel {
    static constexpr int Z = KIND == FQ_KIND_REAL_1D ? 2 : 4;

    struct Col {  // per-source data reused by every pick of a column
        int n_occ;
    };

    template <class K> __device__ __forceinline__ static double diagonal(const ModelParams& p, K k) {
        K st = run_starts(k);
        long long s = 0;
        while (st) {
            int P = KeyOps<K>::ctz(st);
            long long n = run_from(k, P);
            s += n * (n - 1);
            st &= st - 1;
        }
        return (p.u * 0.5) * (double)s;
    }
    template <class K> __device__ __forceinline__ static unsigned num_offdiag(const ModelParams&, K k, Col& c) {
        c.n_occ = KeyOps<K>::popc(run_starts(k));
        return (unsigned)(Z * c.n_occ);
    }
    // k-th off-diagonal entry of the column at `key`; val in FP64, or the
    // FP32 rounding of the same FP64 value
    template <class K, class V>
    __device__ __forceinline__ static K offdiag(const ModelParams& p, K key, const Col& c, unsigned kk,
                                                V& val) {
        // direction d = kk / n_occ < Z and rank r = kk mod n_occ, by comparisons
        const unsigned no = (unsigned)c.n_occ;
        int d = (int)(kk >= no);
        if (Z == 4) d += (int)(kk >= 2u * no) + (int)(kk >= 3u * no);
        const int r = (int)(kk - (unsigned)d * no);
        const int P = KeyOps<K>::nth(run_starts(key), r);
        if constexpr (KIND == FQ_KIND_REAL_1D) {
            // a hop to a neighbouring site only moves one separator: swap
            // the last one-bit of the run with the zero above it (+1), or the
            // zero below the run with its first one-bit (-1); across the ring's
            // seam the whole string shifts by one bit
            typedef KeyOps<K> O;
            const int nb = p.nbits;
            const int ns = run_from(key, P);
            int nt;
            K dest;
            if (d == 0) {
                if (P + ns == nb) {  // last mode -> mode 0
                    nt = run_from(key, 0);
                    dest = O::shl(key & ~O::bit(nb - 1), 1) | (K)1;
                } else {
                    nt = run_from(key, P + ns + 1);
                    dest = key ^ O::shl((K)3, P + ns - 1);
                }
            } else {
                if (P == 0) {  // mode 0 -> last mode
                    const K z = ~key & O::low(nb);
                    nt = nb - 1 - (O::W - 1 - clz_k(z));
                    dest = O::shr(key, 1) | O::bit(nb - 1);
                } else {
                    const K z = ~key & O::low(P - 1);
                    nt = z ? (P - 2 - (O::W - 1 - clz_k(z))) : (P - 1);
                    dest = key ^ O::shl((K)3, P - 1);
                }
            }
            if constexpr (sizeof(V) == 4) val = __ldg(p.hop32_tab + ns * (nt + 1));
            else val = __ldg(p.hop_tab + ns * (nt + 1));
            return dest;
        }
        // 2D: the neighbouring site from the model's table; every direction
        // takes the same path (no divergence within a warp): remove the
        // one-bit at P and insert one at the start q of the target run,
        // located by a search from bit 0 (one code path measured 8 % faster
        // than separator swaps for neighbours along x and this path for the
        // rest).  Bits below P and below q, computed once, give the mode
        // index, both run lengths (the first zero at or above a run's start)
        // and the moved stretch: [P, q) rotates down by one when s' > s,
        // [q, P] up by one when s' < s, the boson landing at its far end.
        typedef KeyOps<K> O;
        const K lowP = O::low(P), nk = ~key;
        const int s = P - O::popc(key & lowP);
        const int ns = O::ctz(nk & ~lowP) - P;
        const int s2 = p.nbr[d][s];  // the table load measured faster than computing it
        const int q = mode_start(key, s2);
        const K lowq = O::low(q);
        const int nt = O::ctz(nk & ~lowq) - q;
        const bool up = s2 > s;
        const K Mu = lowq ^ lowP;
        const K M = up ? Mu : (Mu | O::bit(P));
        const K sh = up ? (key >> 1) : (key << 1);
        const K dest = (key & ~M) | (sh & M) | O::bit(q - (up ? 1 : 0));
        // -(t sqrt(n_s (n_s' + 1))) from the table
        if constexpr (sizeof(V) == 4) val = __ldg(p.hop32_tab + ns * (nt + 1));
        else val = __ldg(p.hop_tab + ns * (nt + 1));
        return dest;
    }
    // sum over modes of n (n - 1), so H_ii = (u/2) times this: windows of
    // w >= 2 consecutive one-bits lie inside one mode's run, and a run of n
    // ones holds n(n-1)/2 of them
    template <class K> __device__ __forceinline__ static int diag_index(K k) {
        K x = k & (k >> 1);
        int s = 0;
        while (x) {
            s += KeyOps<K>::popc(x);
            x &= x >> 1;
        }
        return 2 * s;
    }
};

// Momentum space (Sec. 6.3): H = sum eps_k n_k + (u/2M) sum_{p,k,q}
// a+_{p+q} a+_{k-q} a_k a_p.  Diagonal: sum eps n + (u/2M)(2N^2 - N - sum n^2).
// Off-diagonal entries move an annihilated pair {p, q} to a created pair
// {r, s}, r + s = p + q (mod M), {r,s} != {p,q}.  Enumeration order:
// same-parity pairs (distinct even modes, distinct odd modes, double
// occupancies) each with cE created pairs, then (even, odd) pairs with cO;
// created pairs in ascending r with the identity skipped.  The pick is
// unranked in O(1) from bit masks instead of walking the list.
struct MomModel {
    struct Col {
        uint64_t occm, ge2;  // occupied modes, modes with n >= 2
        int a, b, D;         // #occupied even modes, #odd modes, #double occupancies
        unsigned ne, no;     // #same-parity pairs, #(even,odd) pairs
        unsigned cE, cO;     // created pairs per annihilated pair of each class
    };

    template <class K> __device__ __forceinline__ static double diagonal(const ModelParams& p, K k) {
        K st = run_starts(k);
        double kin = 0.0;
        long long sq = 0;
        while (st) {
            int P = KeyOps<K>::ctz(st);
            int s = P - KeyOps<K>::popc(k & KeyOps<K>::low(P));
            long long n = run_from(k, P);
            kin += p.eps[s] * (double)n;
            sq += n * n;
            st &= st - 1;
        }
        long long N = p.N;
        long long ic = 2 * N * N - N - sq;
        return kin + p.g * (double)ic;
    }

    __device__ __forceinline__ static unsigned pairs_for(int M, int P) {
        // unordered {r <= s} with r + s = P (mod M), P in [0, M)
        return (unsigned)(P / 2 + 1 + (P + M) / 2 - P);
    }

    template <class K> __device__ __forceinline__ static unsigned num_offdiag(const ModelParams& p, K k, Col& c) {
        K st = run_starts(k);
        uint64_t occm = 0, ge2 = 0;
        while (st) {
            int P = KeyOps<K>::ctz(st);
            int s = P - KeyOps<K>::popc(k & KeyOps<K>::low(P));
            occm |= 1ull << s;
            if (run_from(k, P) >= 2) ge2 |= 1ull << s;
            st &= st - 1;
        }
        c.occm = occm; c.ge2 = ge2;
        c.a = __popcll(occm & 0x5555555555555555ull);
        c.b = __popcll(occm & 0xAAAAAAAAAAAAAAAAull);
        c.D = __popcll(ge2);
        c.ne = (unsigned)(c.a * (c.a - 1) / 2 + c.b * (c.b - 1) / 2 + c.D);
        c.no = (unsigned)(c.a * c.b);
        c.cE = pairs_for(p.M, 0) - 1;
        c.cO = pairs_for(p.M, 1 % p.M) - 1;
        return c.ne * c.cE + c.no * c.cO;
    }

    __device__ __forceinline__ static void tri_unrank(unsigned t, int n, int& i, int& j) {
        // t-th pair (i < j) of n items in lexicographic order
        i = 0;
        while (t >= (unsigned)(n - 1 - i)) { t -= (unsigned)(n - 1 - i); ++i; }
        j = i + 1 + (int)t;
    }

    template <class K, class V>
    __device__ __forceinline__ static K offdiag(const ModelParams& pm, K key, const Col& c, unsigned kk,
                                                V& val) {
        const int M = pm.M;
        const uint64_t E = c.occm & 0x5555555555555555ull, O = c.occm & 0xAAAAAAAAAAAAAAAAull;
        int p, q;
        unsigned cr;
        if (kk < c.ne * c.cE) {
            unsigned t = kk / c.cE;
            cr = kk % c.cE;
            const unsigned tE = (unsigned)(c.a * (c.a - 1) / 2), tO = (unsigned)(c.b * (c.b - 1) / 2);
            int i, j;
            if (t < tE) {
                tri_unrank(t, c.a, i, j);
                p = nth_set64(E, i); q = nth_set64(E, j);
            } else if (t < tE + tO) {
                tri_unrank(t - tE, c.b, i, j);
                p = nth_set64(O, i); q = nth_set64(O, j);
            } else {
                p = q = nth_set64(c.ge2, (int)(t - tE - tO));
            }
        } else {
            unsigned k2 = kk - c.ne * c.cE;
            unsigned t = k2 / c.cO;
            cr = k2 % c.cO;
            p = nth_set64(E, (int)(t / (unsigned)c.b));
            q = nth_set64(O, (int)(t % (unsigned)c.b));
        }
        const int P = (p + q) % M;
        const int lo = p < q ? p : q;
        const int half = P / 2;
        const unsigned rank_id = lo <= half ? (unsigned)lo : (unsigned)(half + 1 + (lo - P - 1));
        if (cr >= rank_id) ++cr;
        const int r = (int)cr <= half ? (int)cr : P + 1 + ((int)cr - half - 1);
        const int s = r <= P ? P - r : P + M - r;
        const long long np = mode_occ(key, p), nq = mode_occ(key, q);
        const long long A = np * (nq - (p == q ? 1 : 0));
        K k1 = remove_boson(remove_boson(key, p), q);
        const long long nr = mode_occ(k1, r), ns = mode_occ(k1, s);
        const long long B = (nr + 1) * (ns + 1 + (r == s ? 1 : 0));
        const int F = (p != q ? 2 : 1) * (r != s ? 2 : 1);
        val = (V)(((pm.g * (double)F) * __ldg(pm.sqrt_tab + A)) * __ldg(pm.sqrt_tab + B));
        return add_boson(add_boson(k1, r), s);
    }
};

// ---------------------------------------------------------------------------
// exact bit-level arithmetic: GB300 issues FP64 at a small fraction of its
// FP32/INT rate, so every operation whose result is exact is done on the
// integer bits instead (same results as the FP64 expressions they replace)

__device__ __forceinline__ unsigned long long dbits(double x) {
    return (unsigned long long)__double_as_longlong(x);
}
__device__ __forceinline__ double bdouble(unsigned long long b) {
    return __longlong_as_double((long long)b);
}
constexpr unsigned long long ABS64 = 0x7FFFFFFFFFFFFFFFull;
constexpr unsigned ABS32 = 0x7FFFFFFFu;

// floor(|x|) and ceil(|x|) of a finite double, saturated at 2^32 - 1
__device__ __forceinline__ void floor_ceil_abs(double x, unsigned& fl, unsigned& ce) {
    const unsigned long long b = dbits(x) & ABS64;
    const int E = (int)(b >> 52);
    if (b == 0) { fl = ce = 0; return; }
    if (E < 1023) { fl = 0; ce = 1; return; }
    const int e = E - 1023;
    if (e >= 32) { fl = ce = 0xFFFFFFFFu; return; }
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    const unsigned long long f = m >> (52 - e);
    fl = (unsigned)f;
    ce = (unsigned)f + ((m & ((1ull << (52 - e)) - 1)) ? 1u : 0u);
}
__device__ __forceinline__ void floor_ceil_abs(float x, unsigned& fl, unsigned& ce) {
    const unsigned b = __float_as_uint(x) & ABS32;
    const int E = (int)(b >> 23);
    if (b == 0) { fl = ce = 0; return; }
    if (E < 127) { fl = 0; ce = 1; return; }
    const int e = E - 127;
    if (e >= 32) { fl = ce = 0xFFFFFFFFu; return; }
    const unsigned long long m = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u);
    if (e >= 23) { fl = ce = (unsigned)(m << (e - 23)); return; }
    const unsigned long long f = m >> (23 - e);
    fl = (unsigned)f;
    ce = (unsigned)f + ((m & ((1ull << (23 - e)) - 1)) ? 1u : 0u);
}

// 53 random bits of a draw: the integer u53 with uniform53 = u53 * 2^-53
__device__ __forceinline__ unsigned long long u53_of(uint4 w) {
    return ((unsigned long long)(w.x >> 5) << 26) | (unsigned long long)(w.y >> 6);
}

// u53 * 2^-53 < a * 2^-e for a = m53 * 2^(E - 1075) (biased exponent E,
// E >= 1 normal), decided exactly in integers: with k = 1022 + e - E the
// test is u53 * 2^k < m53 (k >= 0 whenever a < 2^e)
__device__ __forceinline__ bool below_scaled(unsigned long long u53, unsigned long long abits,
                                             int e) {
    const int E = (int)(abits >> 52);
    unsigned long long m;
    int k;
    if (E == 0) {  // subnormal: a = m 2^(1 - 1075)
        m = abits & 0xFFFFFFFFFFFFFull;
        k = 1021 + e;
    } else {
        m = (abits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
        k = 1022 + e - E;
    }
    if (k < 0) return true;  // a >= 2^e (not reached by callers)
    if (k >= 64) return u53 == 0 && m != 0;
    if (k > 0 && (u53 >> (64 - k))) return false;
    return (u53 << k) < m;
}

// bits of (double)|x| for a float x
__device__ __forceinline__ unsigned long long abs_dbits(float x) {
    const unsigned b = __float_as_uint(x) & ABS32;
    if (b == 0) return 0ull;
    if ((b >> 23) == 0) return dbits(fabs((double)x));  // subnormal float
    return ((unsigned long long)((b >> 23) - 127 + 1023) << 52) |
           ((unsigned long long)(b & 0x7FFFFFu) << 29);
}
__device__ __forceinline__ unsigned long long abs_dbits(double x) { return dbits(x) & ABS64; }

// (hi:lo) 2^q rounded to the nearest double, ties to even
__device__ __forceinline__ double fixed_to_double(unsigned long long lo, unsigned long long hi,
                                                  int q) {
    if (!hi) return scalbn(__ull2double_rn(lo), q);
    const int lz = __clzll((long long)hi);
    const int sh = 64 - lz;
    unsigned long long top = sh == 64 ? hi : ((hi << lz) | (lo >> sh));
    const unsigned long long rest = sh == 64 ? lo : (lo & ((1ull << sh) - 1ull));
    if (rest) top |= 1ull;
    return scalbn(__ull2double_rn(top), q + sh);
}

// |x| in units of 2^q as a 128-bit integer (|x| >= 2^(q + 52) so it is
// integral); sets `bad` when it would not fit in 2^116
__device__ __forceinline__ void fixed_of(double x, int q, unsigned long long& lo,
                                         unsigned long long& hi, bool& bad) {
    const unsigned long long b = dbits(x) & ABS64;
    lo = hi = 0;
    if (!b) return;
    const int E = (int)(b >> 52);
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    const int sh = E - 1075 - q;  // |x| = m 2^(E - 1075)
    if (E == 0 || sh > 63) { bad = true; return; }
    if (sh < 0) {  // below 2^(q + 52): exact only if the bits under 2^q are 0
        if (sh < -52 || (m & ((1ull << -sh) - 1ull))) { bad = true; return; }
        lo = m >> -sh;
        return;
    }
    lo = m << sh;
    hi = sh ? (m >> (64 - sh)) : 0ull;
}
__device__ __forceinline__ void fixed_of(float x, int q, unsigned long long& lo,
                                         unsigned long long& hi, bool& bad) {
    const unsigned b = __float_as_uint(x) & ABS32;
    lo = hi = 0;
    if (!b) return;
    const int E = (int)(b >> 23);
    const unsigned long long m = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u);
    const int sh = E - 150 - q;  // |x| = m 2^(E - 150)
    if (E == 0 || sh > 63 + 40) { bad = true; return; }
    if (sh < 0) {  // exact only if the bits under 2^q are 0
        if (sh < -23 || (m & ((1ull << -sh) - 1ull))) { bad = true; return; }
        lo = m >> -sh;
        return;
    }
    if (sh < 64) {
        lo = m << sh;
        hi = sh ? (m >> (64 - sh)) : 0ull;
    } else {
        lo = 0;
        hi = m << (sh - 64);
    }
}
__device__ __forceinline__ void add128(unsigned long long& lo, unsigned long long& hi,
                                       unsigned long long blo, unsigned long long bhi) {
    const unsigned long long l = lo + blo;
    hi += bhi + (l < lo ? 1ull : 0ull);
    lo = l;
}

template <> struct Model<FQ_KIND_REAL_1D> : RealModel<FQ_KIND_REAL_1D> {};
template <> struct Model<FQ_KIND_REAL_2D> : RealModel<FQ_KIND_REAL_2D> {};
template <> struct Model<FQ_KIND_MOM_1D> : MomModel {};

}  // namespace fq
