/*
 * fq_oracle.c -- plain, slow, single-threaded CPU restatement of one FCIQMC
 * time step for Bose-Hubbard Hamiltonians (Rimu.jl paper, arXiv 2601.19505).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and the cpu_baseline
 * leg of bench.py do.  It shares no code, header, table or constant generator
 * with the CUDA path; the two are written independently from the paper.
 *
 * Everything here follows the paper's text directly, with no blocking, fusion
 * or reordering:
 *   - Fock addresses as bit strings (Sec. 6.1): n_m ones for mode m, one zero
 *     between consecutive modes, mode 1 in the least significant bit.
 *   - Real-space Bose-Hubbard Hamiltonian (Eq. bose-hubbard-hamiltonian) and
 *     its momentum-space form (Sec. 6.3 worked example), columns enumerated
 *     on the fly (Sec. 6.2, operator_column / offdiagonals).
 *   - The stochastic step c' = Pi[1 + dt (S - H~)] c (Eq. stochasticTransition-
 *     Operator): matrix compression (Eq. column-compression) with the
 *     semistochastic exact-column rule |c_i| t_rel >= m_i (Sec. 7.1), the
 *     diagonal death/clone factor, annihilation as a plain sum per address,
 *     then vector compression Pi (Eq. vec-compression).  The integer-walker
 *     variant (Sec. 1) and the deterministic limit (Eq. fciqmc) are included.
 *   - The shift update (Eq. shift-update) and the projected-energy numerator
 *     and denominator (Eq. ProjectedEnergy).
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) as the random source;
 *     the paper does not name its generator, so the keyed layout of the draws
 *     is this project's own definition.
 *   - Early compression (Sec. 7.1, Eq. early-comp) as the alternative to the
 *     late compression above, and the replica overlaps c_A^T c_B and
 *     c_A^T G2(d) c_B of Sec. 4.3 (Eqs. RayleighQuotientReplica, g2).
 * Readings of places where the paper is silent or garbled are stated at each
 * function.  Compile with -ffp-contract=off: no fused multiply-adds.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXM 128

enum { OR_REAL_1D = 1, OR_REAL_2D = 2, OR_MOM_1D = 3 };
enum { OR_INT = 0, OR_REAL64 = 1, OR_REAL32 = 2, OR_DETERMINISTIC = 3 };

typedef struct { uint64_t lo, hi; } okey;

typedef struct {
    int kind, Lx, Ly, M, N, nbits;
    double t, u;
    double eps[OR_MAXM]; /* momentum-space single-particle energies */
} or_model;

typedef struct {
    double dt, target, zeta, xi, threshold, t_rel;
    int32_t mode, pad0;
    uint64_t seed;
    uint32_t run_id;
    int32_t compression; /* 0: late (Eq. late-comp), 1: early (Eq. early-comp) */
} or_params;

typedef struct {
    int64_t step, len, exact_steps, inexact_steps, n_spawns;
    double shift, norm, hproj, vproj;
} or_stats;

/* ------------------------------------------------------------------------ */
/* bit strings                                                              */

static int key_bit(okey k, int p) {
    return p < 64 ? (int)((k.lo >> p) & 1u) : (int)((k.hi >> (p - 64)) & 1u);
}
static void key_set(okey *k, int p) {
    if (p < 64) k->lo |= (1ull << p); else k->hi |= (1ull << (p - 64));
}
static int key_cmp(okey a, okey b) {
    if (a.hi != b.hi) return a.hi < b.hi ? -1 : 1;
    if (a.lo != b.lo) return a.lo < b.lo ? -1 : 1;
    return 0;
}

/* Sec. 6.1: scan modes 1..M; emit n_m one-bits, then one zero-bit unless m is
 * the last mode; the first bit emitted is the least significant. */
static okey encode_occ(const or_model *md, const uint8_t *occ) {
    okey k = {0, 0};
    int pos = 0;
    for (int m = 0; m < md->M; ++m) {
        for (int j = 0; j < occ[m]; ++j) key_set(&k, pos++);
        if (m < md->M - 1) pos++;
    }
    return k;
}

static void decode_key(const or_model *md, okey k, uint8_t *occ) {
    memset(occ, 0, (size_t)md->M);
    int m = 0;
    for (int p = 0; p < md->nbits; ++p) {
        if (key_bit(k, p)) occ[m]++;
        else m++;
    }
}

/* ------------------------------------------------------------------------ */
/* model                                                                    */

void *or_model_new(int kind, int Lx, int Ly, int N, double t, double u) {
    if (kind != OR_REAL_1D && kind != OR_REAL_2D && kind != OR_MOM_1D) return NULL;
    if (N < 1 || N > 255) return NULL;
    int M;
    if (kind == OR_REAL_2D) {
        if (Lx < 3 || Ly < 3) return NULL;
        M = Lx * Ly;
    } else {
        if (Ly != 1) return NULL;
        if (kind == OR_REAL_1D && Lx < 3) return NULL;
        if (kind == OR_MOM_1D && Lx < 2) return NULL;
        M = Lx;
    }
    if (M > OR_MAXM || N + M - 1 > 128) return NULL;
    or_model *md = (or_model *)calloc(1, sizeof(or_model));
    md->kind = kind; md->Lx = Lx; md->Ly = Ly; md->M = M; md->N = N;
    md->nbits = N + M - 1;
    md->t = t; md->u = u;
    if (kind == OR_MOM_1D) {
        /* Reading: modes j = 1..M carry k_j = 2 pi (j - floor(M/2)) / M, so
         * mode floor(M/2) is k = 0; eps_j = -2 t cos k_j. */
        for (int m = 0; m < M; ++m) {
            double k = (2.0 * M_PI * (double)(m + 1 - M / 2)) / (double)M;
            md->eps[m] = (-2.0 * t) * cos(k);
        }
    }
    return md;
}

void or_model_free(void *p) { free(p); }

int or_model_info(const void *p, int *M, int *nbits) {
    const or_model *md = (const or_model *)p;
    *M = md->M; *nbits = md->nbits;
    return 0;
}

double or_model_eps(const void *p, int m) { return ((const or_model *)p)->eps[m]; }

int or_encode(const void *p, const uint8_t *occ, okey *out) {
    const or_model *md = (const or_model *)p;
    int s = 0;
    for (int m = 0; m < md->M; ++m) s += occ[m];
    if (s != md->N) return -1;
    *out = encode_occ(md, occ);
    return 0;
}

int or_decode(const void *p, const okey *k, uint8_t *occ) {
    const or_model *md = (const or_model *)p;
    int ones = 0;
    for (int q = 0; q < 128; ++q) {
        if (key_bit(*k, q)) {
            if (q >= md->nbits) return -1;
            ones++;
        }
    }
    if (ones != md->N) return -1;
    decode_key(md, *k, occ);
    return 0;
}

/* Starting address: near_uniform for real space (floor(N/M) per site, the
 * first N mod M sites one more); all bosons in the k = 0 mode for momentum
 * space (reading). */
int or_start(const void *p, okey *out) {
    const or_model *md = (const or_model *)p;
    uint8_t occ[OR_MAXM];
    memset(occ, 0, sizeof occ);
    if (md->kind == OR_MOM_1D) {
        occ[md->M / 2 - 1] = (uint8_t)md->N;
    } else {
        for (int m = 0; m < md->M; ++m)
            occ[m] = (uint8_t)(md->N / md->M + (m < md->N % md->M ? 1 : 0));
    }
    *out = encode_occ(md, occ);
    return 0;
}

/* Diagonal element.  Real space: (u/2) sum_i n_i (n_i - 1).
 * Momentum space: sum_k eps_k n_k + (u / 2M) (2 N^2 - N - sum_k n_k^2), the
 * q = 0 and exchange terms of the two-body sum. */
static double diagonal(const or_model *md, const uint8_t *occ) {
    if (md->kind != OR_MOM_1D) {
        long long s = 0;
        for (int m = 0; m < md->M; ++m) s += (long long)occ[m] * (occ[m] - 1);
        return (md->u * 0.5) * (double)s;
    }
    double kin = 0.0;
    long long sq = 0;
    for (int m = 0; m < md->M; ++m) {
        if (occ[m]) {
            kin += md->eps[m] * (double)occ[m];
            sq += (long long)occ[m] * occ[m];
        }
    }
    long long N = md->N;
    long long ic = 2 * N * N - N - sq;
    return kin + (md->u / (double)(2 * md->M)) * (double)ic;
}

double or_diagonal(const void *p, const okey *k) {
    const or_model *md = (const or_model *)p;
    uint8_t occ[OR_MAXM];
    decode_key(md, *k, occ);
    return diagonal(md, occ);
}

static int neighbour(const or_model *md, int s, int d) {
    if (md->kind == OR_REAL_1D) {
        return d == 0 ? (s + 1) % md->M : (s + md->M - 1) % md->M;
    }
    int x = s % md->Lx, y = s / md->Lx;
    switch (d) {
    case 0: x = (x + 1) % md->Lx; break;
    case 1: x = (x + md->Lx - 1) % md->Lx; break;
    case 2: y = (y + 1) % md->Ly; break;
    default: y = (y + md->Ly - 1) % md->Ly; break;
    }
    return x + md->Lx * y;
}

typedef struct { okey key; double val; } colent;

/* The column of H at `occ`, off-diagonal entries only, in enumeration order.
 * Returns m_i; writes min(m_i, cap) entries (entries may be NULL to count).
 *
 * Real space (Eq. bose-hubbard-hamiltonian): every (direction, occupied site)
 * pair moves one boson from site s to its neighbour s', value
 * -t sqrt(n_s (n_s' + 1)).  Order: direction-major, occupied sites ascending
 * within a direction; 1D directions (+1, -1) as in the 24-entry column the
 * paper prints for |1...1> (Sec. 6.2); 2D directions (+x, -x, +y, -y) (reading).
 *
 * Momentum space (reading; the paper prints entries, not the order): the
 * two-body term (u/2M) sum_{p,k,q} a+_{p+q} a+_{k-q} a_k a_p moves an
 * annihilated pair {p <= k} to a created pair {r <= s} with r + s = p + k
 * (mod M) and {r, s} != {p, k}.  Annihilation pairs come in this order:
 *   1. pairs of distinct occupied even modes, lexicographic;
 *   2. pairs of distinct occupied odd modes, lexicographic;
 *   3. double occupancies (m, m) with n_m >= 2, ascending;
 *   4. (even mode, odd mode) pairs, even-mode-major.
 * For each, the created pairs follow in ascending r over
 * r = 0..M-1, s = (p + k - r) mod M, r <= s, skipping the identity.  Value
 * ((u/2M) F) sqrt(A) sqrt(B) with F = (2 if p != k else 1)(2 if r != s else 1),
 * A = n_p (n_k - [p == k]), B = (m_r + 1)(m_s + 1 + [r == s]),
 * m = n - e_p - e_k. */
static long column(const or_model *md, const uint8_t *occ, colent *ent, long cap) {
    long m = 0;
    uint8_t d[OR_MAXM];
    if (md->kind != OR_MOM_1D) {
        int z = md->kind == OR_REAL_1D ? 2 : 4;
        for (int dir = 0; dir < z; ++dir) {
            for (int s = 0; s < md->M; ++s) {
                if (!occ[s]) continue;
                int s2 = neighbour(md, s, dir);
                if (ent && m < cap) {
                    memcpy(d, occ, (size_t)md->M);
                    d[s]--; d[s2]++;
                    ent[m].key = encode_occ(md, d);
                    ent[m].val = -(md->t * sqrt((double)(occ[s] * (occ[s2] + 1))));
                }
                m++;
            }
        }
        return m;
    }
    int M = md->M;
    int pp[OR_MAXM * OR_MAXM], kk[OR_MAXM * OR_MAXM];
    int npairs = 0;
    for (int par = 0; par < 2; ++par)              /* 1. and 2. */
        for (int a = par; a < M; a += 2)
            for (int b = a + 2; b < M; b += 2)
                if (occ[a] && occ[b]) { pp[npairs] = a; kk[npairs] = b; npairs++; }
    for (int a = 0; a < M; ++a)                    /* 3. */
        if (occ[a] >= 2) { pp[npairs] = a; kk[npairs] = a; npairs++; }
    for (int a = 0; a < M; a += 2)                 /* 4. */
        for (int b = 1; b < M; b += 2)
            if (occ[a] && occ[b]) { pp[npairs] = a; kk[npairs] = b; npairs++; }
    double g = md->u / (double)(2 * M);
    for (int i = 0; i < npairs; ++i) {
        int p = pp[i], k = kk[i];
        int lo = p < k ? p : k, hi = p < k ? k : p;
        int P = (p + k) % M;
        for (int r = 0; r < M; ++r) {
            int s = ((P - r) % M + M) % M;
            if (r > s) continue;
            if (r == lo && s == hi) continue;
            if (ent && m < cap) {
                memcpy(d, occ, (size_t)M);
                long long A = (long long)occ[p] * (occ[k] - (p == k ? 1 : 0));
                d[p]--; d[k]--;
                long long B = (long long)(d[r] + 1) * (d[s] + 1 + (r == s ? 1 : 0));
                d[r]++; d[s]++;
                int F = (p != k ? 2 : 1) * (r != s ? 2 : 1);
                ent[m].key = encode_occ(md, d);
                ent[m].val = ((g * (double)F) * sqrt((double)A)) * sqrt((double)B);
            }
            m++;
        }
    }
    return m;
}

long or_column(const void *p, const okey *k, okey *keys, double *vals, long cap) {
    const or_model *md = (const or_model *)p;
    uint8_t occ[OR_MAXM];
    decode_key(md, *k, occ);
    long m = column(md, occ, NULL, 0);
    colent *ent = (colent *)malloc(sizeof(colent) * (size_t)(m > 0 ? m : 1));
    column(md, occ, ent, m);
    for (long i = 0; i < m && i < cap; ++i) { keys[i] = ent[i].key; vals[i] = ent[i].val; }
    free(ent);
    return m;
}

/* Momentum space written straight from the second-quantised sum, for pins:
 * apply (u/2M) a+_{p+q} a+_{k-q} a_k a_p for every ordered (p, k, q) and add
 * equal destinations.  Returns the number of distinct off-diagonal
 * destinations (unordered), the interaction part of the diagonal in *diag. */
long or_column_bruteforce(const void *pm, const okey *key, okey *keys, double *vals, long cap,
                          double *diag) {
    const or_model *md = (const or_model *)pm;
    int M = md->M;
    uint8_t occ[OR_MAXM], d[OR_MAXM];
    decode_key(md, *key, occ);
    long n = 0;
    *diag = 0.0;
    double g = md->u / (double)(2 * M);
    for (int p = 0; p < M; ++p)
        for (int k = 0; k < M; ++k)
            for (int q = 0; q < M; ++q) {
                memcpy(d, occ, (size_t)M);
                double f = 1.0;
                if (!d[p]) continue;
                f *= sqrt((double)d[p]); d[p]--;
                if (!d[k]) continue;
                f *= sqrt((double)d[k]); d[k]--;
                int c1 = ((k - q) % M + M) % M, c2 = (p + q) % M;
                f *= sqrt((double)(d[c1] + 1)); d[c1]++;
                f *= sqrt((double)(d[c2] + 1)); d[c2]++;
                okey dk = encode_occ(md, d);
                if (key_cmp(dk, *key) == 0) { *diag += g * f; continue; }
                long j;
                for (j = 0; j < n; ++j) if (key_cmp(keys[j], dk) == 0) break;
                if (j == n) {
                    if (n >= cap) return -1;
                    keys[n] = dk; vals[n] = 0.0; n++;
                }
                vals[j] += g * f;
            }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products
 * with multipliers 0xD2511F53 and 0xCD9E8D57; the key is bumped by the Weyl
 * constants 0x9E3779B9 and 0xBB67AE85 between rounds.                      */

static void philox_round(uint32_t x[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)0xD2511F53u * x[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * x[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x[1] ^ k[0];
    uint32_t y2 = hi0 ^ x[3] ^ k[1];
    x[0] = y0; x[1] = lo1; x[2] = y2; x[3] = lo0;
}

void or_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
    uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
        philox_round(x, k);
    }
    memcpy(out, x, sizeof x);
}

/* splitmix64 (Steele, Lea, Flood 2014): golden-ratio increment + finaliser. */
static uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Draw layout (this project's definition; the paper fixes none):
 *   Philox key     = (seed_lo32, seed_hi32 ^ run_id * 0x9E3779B9)
 *   Philox counter = (step, stream, h_lo32, h_hi32)
 *   h = the address itself when it fits 64 bits, else lo ^ splitmix64(hi)
 *   stream = attempt index for spawn picks, 0xFFFFFFFF for vector
 *   compression of a destination, 0xFFFFFFFE for integer diagonal rounding.
 *   uniform in [0,1) = ((w0 >> 5) 2^26 + (w1 >> 6)) 2^-53
 *   index in [0,m)   = (w2 m) >> 32                                       */
static uint64_t rng_h(const or_model *md, okey k) {
    return md->nbits <= 64 ? k.lo : (k.lo ^ splitmix64(k.hi));
}

static void draw(const or_params *pr, uint32_t step, uint32_t stream, uint64_t h, uint32_t w[4]) {
    uint32_t ctr[4] = {step, stream, (uint32_t)h, (uint32_t)(h >> 32)};
    uint32_t key[2] = {(uint32_t)pr->seed,
                       (uint32_t)(pr->seed >> 32) ^ (uint32_t)(pr->run_id * 0x9E3779B9u)};
    or_philox(ctr, key, w);
}

static double uniform53(const uint32_t w[4]) {
    return ((double)(w[0] >> 5) * 67108864.0 + (double)(w[1] >> 6)) * (1.0 / 9007199254740992.0);
}

static uint32_t pick(const uint32_t w[4], uint32_t m) {
    return (uint32_t)(((uint64_t)w[2] * (uint64_t)m) >> 32);
}

/* ------------------------------------------------------------------------ */
/* one step                                                                 */

typedef struct {
    okey dest, src;
    uint32_t attempt;
    int32_t is_spawn; /* 0 = diagonal term, 1 = spawn */
    double val;
} contrib;

typedef struct { okey key; double amp; } entry;

typedef struct {
    or_model md;
    or_params pr;
    entry *vec;
    long n, cap;
    double shift, norm;
    int64_t step;
    /* projected-energy reference y */
    okey *ref_key; double *ref_y; long n_ref;
    /* history */
    or_stats *hist; long n_hist, cap_hist;
    /* spawn list of the most recent step, in generation order */
    int record;
    okey *sp_key; okey *sp_src; double *sp_val; long n_sp, cap_sp;
} or_run;

static int cmp_contrib(const void *a, const void *b) {
    const contrib *x = (const contrib *)a, *y = (const contrib *)b;
    int c = key_cmp(x->dest, y->dest);
    if (c) return c;
    if (x->is_spawn != y->is_spawn) return x->is_spawn < y->is_spawn ? -1 : 1;
    c = key_cmp(x->src, y->src);
    if (c) return c;
    if (x->attempt != y->attempt) return x->attempt < y->attempt ? -1 : 1;
    return 0;
}

typedef struct { contrib *c; long n, cap; } clist;

static void push(clist *l, okey dest, okey src, uint32_t a, int is_spawn, double v) {
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 1024;
        l->c = (contrib *)realloc(l->c, sizeof(contrib) * (size_t)l->cap);
    }
    contrib *e = &l->c[l->n++];
    e->dest = dest; e->src = src; e->attempt = a; e->is_spawn = is_spawn; e->val = v;
}

static double store_round(int mode, double v) {
    return mode == OR_REAL32 ? (double)(float)v : v;
}

static int compress_one(const or_params *pr, const uint32_t w[4], double v, double *out);

/* Early compression applies to real-valued walkers only (integer walkers
 * are integral already; the deterministic limit compresses nothing). */
static int early(const or_params *pr) {
    return pr->compression == 1 && (pr->mode == OR_REAL64 || pr->mode == OR_REAL32);
}

/* Push one spawn or diagonal term; under early compression (Sec. 7.1) it is
 * first compressed on its own with the 53-bit uniform of draw `w`, and a
 * dropped value is not pushed.  Returns 1 when a value was pushed. */
static int push_term(clist *out, const or_params *pr, const uint32_t w[4], okey dest, okey src,
                     uint32_t a, int is_spawn, double v) {
    if (early(pr)) {
        double o;
        if (!compress_one(pr, w, v, &o)) return 0;
        v = o;
    }
    push(out, dest, src, a, is_spawn, v);
    return 1;
}

/* Every contribution of source entry (key, c) at step `step`, shift `shift`:
 * the diagonal term and the spawns (Eq. column-compression).  Counts
 * exact/inexact columns.  Under early compression the draws of the
 * individual compressions are: the pick's own draw (attempt a) for a
 * stochastic spawn, the draw of stream k for entry k of an exact column, and
 * stream 0xFFFFFFFD for the diagonal term, all keyed by the source. */
static void source_contribs(const or_model *md, const or_params *pr, uint32_t step, double shift,
                            okey key, double c, clist *out, int64_t *n_exact, int64_t *n_inexact,
                            int64_t *n_spawns) {
    uint8_t occ[OR_MAXM];
    decode_key(md, key, occ);
    double hii = diagonal(md, occ);
    long m = column(md, occ, NULL, 0);
    colent *col = (colent *)malloc(sizeof(colent) * (size_t)(m > 0 ? m : 1));
    column(md, occ, col, m);
    uint64_t h = rng_h(md, key);
    double dt = pr->dt;
    double factor = 1.0 + dt * (shift - hii); /* T_ii of Eq. propagator */

    if (pr->mode == OR_INT) {
        /* Integer walkers (reading of the original integer formulation):
         * |c| attempts, each picks one off-diagonal uniformly and spawns
         * floor(p) + [u < p - floor(p)] walkers, p = dt |H_ji| m, of sign
         * -sign(H_ji) sign(c); the diagonal x = c T_ii is rounded
         * stochastically to an integer. */
        (*n_inexact)++;
        int64_t nat = (int64_t)fabs(c);
        double dtm = dt * (double)m;
        for (int64_t a = 0; a < nat && m > 0; ++a) {
            uint32_t w[4];
            draw(pr, step, (uint32_t)a, h, w);
            uint32_t k = pick(w, (uint32_t)m);
            double hv = col[k].val;
            double p = fabs(hv) * dtm;
            double fl = floor(p);
            int64_t cnt = (int64_t)fl + (uniform53(w) < p - fl ? 1 : 0);
            if (cnt) {
                int64_t sg = (hv > 0.0 ? -1 : 1) * (c > 0.0 ? 1 : -1);
                push(out, col[k].key, key, (uint32_t)a, 1, (double)(sg * cnt));
                (*n_spawns)++;
            }
        }
        double x = c * factor;
        double fl = floor(x);
        uint32_t w[4];
        draw(pr, step, 0xFFFFFFFEu, h, w);
        double xr = fl + (uniform53(w) < x - fl ? 1.0 : 0.0);
        push(out, key, key, 0, 0, xr);
        free(col);
        return;
    }

    /* Exact column when |c_i| t_rel >= m_i (Sec. 7.1); always in the
     * deterministic limit. */
    if (pr->mode == OR_REAL32) {
        /* FP32 amplitudes: every per-entry product in FP32; the diagonal term
         * is c + c delta with delta = dt (S - H_ii) rounded once to FP32, so
         * that the factor 1 + delta carries no rounding bias of its own. */
        const float cf = (float)c, dtf = (float)dt;
        const float delta = (float)(dt * (shift - hii));
        int exact = fabs(c) * pr->t_rel >= (double)m;
        if (exact) {
            (*n_exact)++;
            const float coef = (-dtf) * cf;
            for (long k = 0; k < m; ++k) {
                const float v = (float)col[k].val * coef;
                uint32_t w[4] = {0, 0, 0, 0};
                if (early(pr)) draw(pr, step, (uint32_t)k, h, w);
                *n_spawns += push_term(out, pr, w, col[k].key, key, (uint32_t)k, 1, (double)v);
            }
        } else {
            (*n_inexact)++;
            const uint32_t n = (uint32_t)ceil(fabs(c));
            const float coef = ((-dtf) * ((float)m / (float)n)) * cf;
            for (uint32_t a = 0; a < n; ++a) {
                uint32_t w[4];
                draw(pr, step, a, h, w);
                uint32_t k = pick(w, (uint32_t)m);
                const float v = (float)col[k].val * coef;
                *n_spawns += push_term(out, pr, w, col[k].key, key, a, 1, (double)v);
            }
        }
        const float d = cf + cf * delta;
        uint32_t wd[4] = {0, 0, 0, 0};
        if (early(pr)) draw(pr, step, 0xFFFFFFFDu, h, wd);
        push_term(out, pr, wd, key, key, 0, 0, (double)d);
        free(col);
        return;
    }

    /* Each spawn is H_ji coef with coef = -dt c_i (exact column) or
     * -dt (m_i / n_i) c_i (n_i picks), the factors of Eq. column-compression
     * multiplied in this order. */
    int exact = pr->mode == OR_DETERMINISTIC || fabs(c) * pr->t_rel >= (double)m;
    if (exact) {
        (*n_exact)++;
        double coef = (-dt) * c;
        for (long k = 0; k < m; ++k) {
            double v = col[k].val * coef;
            uint32_t w[4] = {0, 0, 0, 0};
            if (early(pr)) draw(pr, step, (uint32_t)k, h, w);
            *n_spawns += push_term(out, pr, w, col[k].key, key, (uint32_t)k, 1,
                                   store_round(pr->mode, v));
        }
    } else {
        (*n_inexact)++;
        double nd = ceil(fabs(c));
        uint32_t n = (uint32_t)nd;
        double coef = ((-dt) * ((double)m / (double)n)) * c;
        for (uint32_t a = 0; a < n; ++a) {
            uint32_t w[4];
            draw(pr, step, a, h, w);
            uint32_t k = pick(w, (uint32_t)m);
            double v = col[k].val * coef;
            *n_spawns += push_term(out, pr, w, col[k].key, key, a, 1, store_round(pr->mode, v));
        }
    }
    uint32_t wd[4] = {0, 0, 0, 0};
    if (early(pr)) draw(pr, step, 0xFFFFFFFDu, h, wd);
    push_term(out, pr, wd, key, key, 0, 0, c * factor);
    free(col);
}

/* Vector compression Pi (Eq. vec-compression) of one merged value.  Reading:
 * a kept small value is sign(w) theta, not 1, so the map is unbiased for
 * negative w and for theta != 1.  Returns 0 when the entry is dropped. */
static int compress(const or_model *md, const or_params *pr, uint32_t step, okey key, double w,
                    double *out) {
    if (w == 0.0) return 0;
    if (pr->mode == OR_INT || pr->mode == OR_DETERMINISTIC) { *out = w; return 1; }
    double aw = fabs(w);
    if (aw >= pr->threshold) { *out = store_round(pr->mode, w); return 1; }
    uint32_t r[4];
    draw(pr, step, 0xFFFFFFFFu, rng_h(md, key), r);
    if (uniform53(r) < aw / pr->threshold) {
        *out = store_round(pr->mode, copysign(pr->threshold, w));
        return 1;
    }
    return 0;
}

/* Early compression (Sec. 7.1, Eq. early-comp): Pi applied to the
 * contribution of one column before any sum.  Reading: the text says each
 * spawn is compressed individually, so every spawn value and the diagonal
 * term d_i are compressed on their own; nothing is compressed after the
 * sum.  The value v is kept when |v| >= theta, else it becomes sign(v) theta
 * with probability |v| / theta (as in late compression), decided by the
 * 53-bit uniform of the draw `w`.  Returns 0 when the value is dropped. */
static int compress_one(const or_params *pr, const uint32_t w[4], double v, double *out) {
    if (v == 0.0) return 0;
    double av = fabs(v);
    if (av >= pr->threshold) { *out = v; return 1; }
    if (uniform53(w) < av / pr->threshold) {
        *out = store_round(pr->mode, copysign(pr->threshold, v));
        return 1;
    }
    return 0;
}

/* The one-norm ||c||_1 = sum_i |c_i|, evaluated exactly and rounded once to
 * the nearest double.  After vector compression every stored |c_i| is at
 * least theta (or an integer in integer mode), so each is an integer
 * multiple of 2^q with q = ilogb(theta) - 52 (q = 0 for integer walkers): the
 * sum is taken in 128-bit integers of that unit.  The deterministic limit has
 * no such floor; there the sum is the plain sequential one. */
static int norm_unit(const or_params *pr) {
    if (pr->mode == OR_INT) return 0;
    return ilogb(pr->threshold) - 52;
}

static double exact_norm(const or_run *r) {
    if (r->pr.mode == OR_DETERMINISTIC) {
        double s = 0.0;
        for (long i = 0; i < r->n; ++i) s += fabs(r->vec[i].amp);
        return s;
    }
    int q = norm_unit(&r->pr);
    unsigned __int128 acc = 0;
    for (long i = 0; i < r->n; ++i)
        acc += (unsigned __int128)ldexp(fabs(r->vec[i].amp), -q);
    /* round to nearest, ties to even: keep the top 64 bits, fold every bit
     * below them into the lowest kept bit, convert (64 > 53 + 1 bits) */
    uint64_t hi = (uint64_t)(acc >> 64), lo = (uint64_t)acc;
    if (!hi) return ldexp((double)lo, q);
    int lz = __builtin_clzll(hi);
    int sh = 64 - lz;
    uint64_t top = sh == 64 ? hi : ((hi << lz) | (lo >> sh));
    uint64_t rest = sh == 64 ? lo : (lo & ((1ull << sh) - 1));
    if (rest) top |= 1u;
    return ldexp((double)top, q + sh);
}

double or_exact_norm_of(const double *amps, long n, double threshold, int mode) {
    or_run r;
    memset(&r, 0, sizeof r);
    r.pr.threshold = threshold;
    r.pr.mode = mode;
    entry *e = (entry *)malloc(sizeof(entry) * (size_t)(n > 0 ? n : 1));
    for (long i = 0; i < n; ++i) { e[i].amp = amps[i]; e[i].key.lo = e[i].key.hi = 0; }
    r.vec = e; r.n = n;
    double s = exact_norm(&r);
    free(e);
    return s;
}

static double lookup(const or_run *r, okey k) {
    long lo = 0, hi = r->n - 1;
    while (lo <= hi) {
        long mid = (lo + hi) / 2;
        int c = key_cmp(r->vec[mid].key, k);
        if (c == 0) return r->vec[mid].amp;
        if (c < 0) lo = mid + 1; else hi = mid - 1;
    }
    return 0.0;
}

/* y^T H c and y^T c for the stored vector (Eq. ProjectedEnergy).  Order: for
 * each reference entry r in the order given, the diagonal term then the
 * off-diagonal terms in enumeration order. */
static void projections(const or_run *r, double *hproj, double *vproj) {
    double hp = 0.0, vp = 0.0;
    for (long i = 0; i < r->n_ref; ++i) {
        okey rk = r->ref_key[i];
        double y = r->ref_y[i];
        uint8_t occ[OR_MAXM];
        decode_key(&r->md, rk, occ);
        double cr = lookup(r, rk);
        vp += y * cr;
        hp += (y * diagonal(&r->md, occ)) * cr;
        long m = column(&r->md, occ, NULL, 0);
        colent *col = (colent *)malloc(sizeof(colent) * (size_t)(m > 0 ? m : 1));
        column(&r->md, occ, col, m);
        for (long k = 0; k < m; ++k) hp += (y * col[k].val) * lookup(r, col[k].key);
        free(col);
    }
    *hproj = hp; *vproj = vp;
}

void *or_run_new(const void *model, const or_params *pr) {
    or_run *r = (or_run *)calloc(1, sizeof(or_run));
    r->md = *(const or_model *)model;
    r->pr = *pr;
    return r;
}

void or_run_free(void *p) {
    or_run *r = (or_run *)p;
    if (!r) return;
    free(r->vec); free(r->ref_key); free(r->ref_y); free(r->hist);
    free(r->sp_key); free(r->sp_src); free(r->sp_val);
    free(r);
}

/* Eq. shift-update: S' = S - (zeta/dt) ln(N'/N) - (xi/dt) ln(N'/N_t). */
double or_shift_update(double S, double N0, double N1, double dt, double zeta, double xi,
                       double target) {
    double zd = zeta / dt, xd = xi / dt;
    return (S - zd * log(N1 / N0)) - xd * log(N1 / target);
}

static int cmp_entry(const void *a, const void *b) {
    return key_cmp(((const entry *)a)->key, ((const entry *)b)->key);
}

/* Replace the stored vector; entries are sorted by address and must be
 * distinct; zero amplitudes are dropped.  The norm is sum |c|. */
int or_run_seed(void *p, const okey *keys, const double *amps, long n, double shift, int64_t step) {
    or_run *r = (or_run *)p;
    free(r->vec);
    r->vec = (entry *)malloc(sizeof(entry) * (size_t)(n > 0 ? n : 1));
    long j = 0;
    for (long i = 0; i < n; ++i) {
        if (amps[i] == 0.0) continue;
        r->vec[j].key = keys[i];
        r->vec[j].amp = store_round(r->pr.mode, amps[i]);
        j++;
    }
    r->n = j; r->cap = j;
    qsort(r->vec, (size_t)r->n, sizeof(entry), cmp_entry);
    for (long i = 1; i < r->n; ++i)
        if (key_cmp(r->vec[i - 1].key, r->vec[i].key) == 0) return -1;
    double s = 0.0;
    for (long i = 0; i < r->n; ++i) s += fabs(r->vec[i].amp);
    r->norm = s;
    r->shift = shift;
    r->step = step;
    r->n_hist = 0;
    return 0;
}

int or_run_set_reference(void *p, const okey *keys, const double *y, long n) {
    or_run *r = (or_run *)p;
    free(r->ref_key); free(r->ref_y);
    r->ref_key = (okey *)malloc(sizeof(okey) * (size_t)(n > 0 ? n : 1));
    r->ref_y = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    memcpy(r->ref_key, keys, sizeof(okey) * (size_t)n);
    memcpy(r->ref_y, y, sizeof(double) * (size_t)n);
    r->n_ref = n;
    return 0;
}

void or_run_set(void *p, double dt, double shift, double target) {
    or_run *r = (or_run *)p;
    if (dt > 0) r->pr.dt = dt;
    r->shift = shift;
    if (target > 0) r->pr.target = target;
}

void or_run_record_spawns(void *p, int on) { ((or_run *)p)->record = on; }

/* One step c^(n+1) = Pi[1 + dt (S^(n) - H~)] c^(n), then the shift update
 * S^(n+1) = S^(n) - (zeta/dt) ln(N^(n+1)/N^(n)) - (xi/dt) ln(N^(n+1)/N_t)
 * (Eq. shift-update).  Contributions to an address are summed diagonal term
 * first, then spawns by (source address, attempt).  Returns -5 when the
 * population dies (norm 0). */
typedef struct { int64_t n_exact, n_inexact, n_spawns; } step_counts;

/* The new vector of one step (spawning, annihilation, compression). */
static void step_vector(or_run *r, step_counts *sc) {
    uint32_t step = (uint32_t)(r->step + 1);
    clist cl = {0};
    int64_t n_exact = 0, n_inexact = 0, n_spawns = 0;
    for (long i = 0; i < r->n; ++i)
        source_contribs(&r->md, &r->pr, step, r->shift, r->vec[i].key, r->vec[i].amp, &cl,
                        &n_exact, &n_inexact, &n_spawns);
    if (r->record) {
        r->n_sp = 0;
        for (long i = 0; i < cl.n; ++i) {
            if (!cl.c[i].is_spawn) continue;
            if (r->n_sp == r->cap_sp) {
                r->cap_sp = r->cap_sp ? 2 * r->cap_sp : 1024;
                r->sp_key = (okey *)realloc(r->sp_key, sizeof(okey) * (size_t)r->cap_sp);
                r->sp_src = (okey *)realloc(r->sp_src, sizeof(okey) * (size_t)r->cap_sp);
                r->sp_val = (double *)realloc(r->sp_val, sizeof(double) * (size_t)r->cap_sp);
            }
            r->sp_key[r->n_sp] = cl.c[i].dest;
            r->sp_src[r->n_sp] = cl.c[i].src;
            r->sp_val[r->n_sp] = cl.c[i].val;
            r->n_sp++;
        }
    }
    qsort(cl.c, (size_t)cl.n, sizeof(contrib), cmp_contrib);
    entry *nv = (entry *)malloc(sizeof(entry) * (size_t)(cl.n > 0 ? cl.n : 1));
    long nn = 0;
    for (long i = 0; i < cl.n;) {
        long j = i;
        double w = 0.0;
        float wf = 0.0f;
        while (j < cl.n && key_cmp(cl.c[j].dest, cl.c[i].dest) == 0) {
            w += cl.c[j].val;
            wf += (float)cl.c[j].val;
            j++;
        }
        if (r->pr.mode == OR_REAL32) w = (double)wf;
        double out;
        if (early(&r->pr) ? (out = w) != 0.0
                                   : compress(&r->md, &r->pr, step, cl.c[i].dest, w, &out)) {
            nv[nn].key = cl.c[i].dest;
            nv[nn].amp = out;
            nn++;
        }
        i = j;
    }
    free(cl.c);
    free(r->vec);
    r->vec = nv; r->n = nn; r->cap = cl.n;
    sc->n_exact = n_exact; sc->n_inexact = n_inexact; sc->n_spawns = n_spawns;
}

/* The end of a step: the norm of the new vector, the shift update and the
 * history row.  Returns -5 when the population died. */
static int step_finish(or_run *r, const step_counts *sc) {
    uint32_t step = (uint32_t)(r->step + 1);
    double norm = exact_norm(r);
    r->step = step;
    if (norm == 0.0) { r->norm = 0.0; return -5; }
    r->shift = or_shift_update(r->shift, r->norm, norm, r->pr.dt, r->pr.zeta, r->pr.xi,
                               r->pr.target);
    r->norm = norm;

    or_stats st;
    st.step = r->step; st.len = r->n;
    st.exact_steps = sc->n_exact; st.inexact_steps = sc->n_inexact; st.n_spawns = sc->n_spawns;
    st.shift = r->shift; st.norm = norm;
    projections(r, &st.hproj, &st.vproj);
    if (r->n_hist == r->cap_hist) {
        r->cap_hist = r->cap_hist ? 2 * r->cap_hist : 256;
        r->hist = (or_stats *)realloc(r->hist, sizeof(or_stats) * (size_t)r->cap_hist);
    }
    r->hist[r->n_hist++] = st;
    return 0;
}

static int one_step(or_run *r) {
    step_counts sc;
    step_vector(r, &sc);
    return step_finish(r, &sc);
}

int or_run_step(void *p, long nsteps) {
    or_run *r = (or_run *)p;
    for (long i = 0; i < nsteps; ++i) {
        int rc = one_step(r);
        if (rc) return rc;
    }
    return 0;
}

long or_run_len(const void *p) { return ((const or_run *)p)->n; }

long or_run_export(const void *p, okey *keys, double *amps, long cap) {
    const or_run *r = (const or_run *)p;
    for (long i = 0; i < r->n && i < cap; ++i) { keys[i] = r->vec[i].key; amps[i] = r->vec[i].amp; }
    return r->n;
}

void or_run_state(const void *p, double *shift, double *norm, int64_t *step) {
    const or_run *r = (const or_run *)p;
    *shift = r->shift; *norm = r->norm; *step = r->step;
}

long or_run_history(const void *p, or_stats *rows, long cap) {
    const or_run *r = (const or_run *)p;
    for (long i = 0; i < r->n_hist && i < cap; ++i) rows[i] = r->hist[i];
    return r->n_hist;
}

long or_run_spawns(const void *p, okey *dest, okey *src, double *val, long cap) {
    const or_run *r = (const or_run *)p;
    for (long i = 0; i < r->n_sp && i < cap; ++i) { dest[i] = r->sp_key[i]; src[i] = r->sp_src[i]; val[i] = r->sp_val[i]; }
    return r->n_sp;
}

/* The value one address j takes in the next step, computed from j alone:
 * its diagonal term plus the spawns that land on j from every source i in
 * the column of j (H is real symmetric, so those are the only sources),
 * summed in the order one_step uses; then Pi.  *pre = merged value,
 * *post = value after compression (0 if dropped).  The stored vector is not
 * changed.  This is how a single output of a very large step is checked. */
int or_point(const void *p, const okey *jkey, double *pre, double *post) {
    const or_run *r = (const or_run *)p;
    uint32_t step = (uint32_t)(r->step + 1);
    uint8_t occ[OR_MAXM];
    decode_key(&r->md, *jkey, occ);
    long m = column(&r->md, occ, NULL, 0);
    colent *col = (colent *)malloc(sizeof(colent) * (size_t)(m > 0 ? m : 1));
    column(&r->md, occ, col, m);
    clist cl = {0};
    int64_t a = 0, b = 0, c = 0;
    double cj = lookup(r, *jkey);
    if (cj != 0.0) source_contribs(&r->md, &r->pr, step, r->shift, *jkey, cj, &cl, &a, &b, &c);
    for (long k = 0; k < m; ++k) {
        double ci = lookup(r, col[k].key);
        if (ci != 0.0)
            source_contribs(&r->md, &r->pr, step, r->shift, col[k].key, ci, &cl, &a, &b, &c);
    }
    free(col);
    long keep = 0;
    for (long i = 0; i < cl.n; ++i)
        if (key_cmp(cl.c[i].dest, *jkey) == 0) cl.c[keep++] = cl.c[i];
    cl.n = keep;
    qsort(cl.c, (size_t)cl.n, sizeof(contrib), cmp_contrib);
    double w = 0.0;
    float wf = 0.0f;
    for (long i = 0; i < cl.n; ++i) {
        w += cl.c[i].val;
        wf += (float)cl.c[i].val;
    }
    if (r->pr.mode == OR_REAL32) w = (double)wf;
    free(cl.c);
    *pre = w;
    double out = 0.0;
    if (early(&r->pr)) out = w;
    else if (!compress(&r->md, &r->pr, step, *jkey, w, &out)) out = 0.0;
    *post = out;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* replica overlaps (Sec. 4.3)                                              */

/* Eq. g2: G2(d) = (1/M) sum_i n_i (n_{i+d} - delta_{d,0}) is diagonal in the
 * real-space occupation basis; sites i + d are taken around the periodic
 * ring of M sites (1D real space). */
static double g2_diag(const or_model *md, const uint8_t *occ, int d) {
    long long s = 0;
    for (int i = 0; i < md->M; ++i)
        s += (long long)occ[i] * ((long long)occ[(i + d) % md->M] - (d == 0 ? 1 : 0));
    return (double)s / (double)md->M;
}

/* For two stored vectors of one model: out[0] = c_A^T c_B and
 * out[1 + k] = c_A^T G2(d_k) c_B (k < nd; 1D real space only), the
 * vector-vector and vector-operator-vector products of Sec. 4.3 that
 * Eq. RayleighQuotientReplica averages.  Both vectors are sorted by
 * address, so the common addresses are found by walking the two lists
 * together; the terms c_A,j c_B,j and G2(d)_jj c_A,j c_B,j are added in
 * ascending address order.  Returns -1 for G2 requested outside 1D real
 * space or d outside [0, M). */
int or_overlap(const void *pa, const void *pb, const int *d, int nd, double *out) {
    const or_run *a = (const or_run *)pa, *b = (const or_run *)pb;
    if (nd > 0 && a->md.kind != OR_REAL_1D) return -1;
    for (int k = 0; k < nd; ++k)
        if (d[k] < 0 || d[k] >= a->md.M) return -1;
    for (int k = 0; k <= nd; ++k) out[k] = 0.0;
    long i = 0, j = 0;
    while (i < a->n && j < b->n) {
        int c = key_cmp(a->vec[i].key, b->vec[j].key);
        if (c < 0) { ++i; continue; }
        if (c > 0) { ++j; continue; }
        double p = a->vec[i].amp * b->vec[j].amp;
        out[0] += p;
        if (nd > 0) {
            uint8_t occ[OR_MAXM];
            decode_key(&a->md, a->vec[i].key, occ);
            for (int k = 0; k < nd; ++k) out[1 + k] += g2_diag(&a->md, occ, d[k]) * p;
        }
        ++i; ++j;
    }
    return 0;
}

/* G2(d)_jj of one address (for pins against the definition). */
double or_g2_diag(const void *pm, const okey *k, int d) {
    const or_model *md = (const or_model *)pm;
    uint8_t occ[OR_MAXM];
    decode_key(md, *k, occ);
    return g2_diag(md, occ, d);
}

/* ------------------------------------------------------------------------ */
/* excited states (Sec. 2.2): K step-synchronised runs, the k-th
 * orthogonalised to the ones before it after every step (Gram-Schmidt)      */

static double dot_sorted(const or_run *a, const or_run *b) {
    double s = 0.0;
    long i = 0, j = 0;
    while (i < a->n && j < b->n) {
        int c = key_cmp(a->vec[i].key, b->vec[j].key);
        if (c < 0) { ++i; continue; }
        if (c > 0) { ++j; continue; }
        s += a->vec[i].amp * b->vec[j].amp;
        ++i; ++j;
    }
    return s;
}

/* c_k <- c_k - sum_{j<k} alpha_j c_j with alpha_j = (c_j^T c_k) / (c_j^T c_j)
 * (classical Gram-Schmidt: every alpha_j from the same c_k, the c_j already
 * orthogonalised this step).  Readings (the paper names the method only):
 * (i) the dot products are FP64 sums in ascending address order; (ii) per
 * address the terms are subtracted in order j = 0, 1, ..., each as
 * v - alpha_j c_j (FP32 arithmetic with FP32 alpha for REAL32 runs); (iii) a
 * value that changed is then compressed by Pi (Eq. vec-compression, the
 * draw of stream 0xFFFFFFFC of its address and run), so the vector stays
 * as sparse as a step leaves it; the deterministic limit compresses
 * nothing.  Integer walkers are not supported (returns -1). */
static int orthogonalise(or_run **runs, int k) {
    or_run *rk = runs[k];
    if (rk->pr.mode == OR_INT) return -1;
    double alpha[8];
    for (int j = 0; j < k; ++j) {
        double djj = dot_sorted(runs[j], runs[j]);
        alpha[j] = djj != 0.0 ? dot_sorted(runs[j], rk) / djj : 0.0;
    }
    long cap = rk->n;
    for (int j = 0; j < k; ++j) cap += runs[j]->n;
    entry *nv = (entry *)malloc(sizeof(entry) * (size_t)(cap > 0 ? cap : 1));
    long *pos = (long *)calloc((size_t)(k + 1), sizeof(long));
    long nn = 0;
    uint32_t step = (uint32_t)(rk->step + 1);
    const int f32 = rk->pr.mode == OR_REAL32;
    for (;;) {
        /* the smallest address not yet taken from any of the k + 1 lists */
        int have = 0;
        okey a = {0, 0};
        for (int j = 0; j <= k; ++j) {
            const or_run *rj = j < k ? runs[j] : rk;
            if (pos[j] < rj->n && (!have || key_cmp(rj->vec[pos[j]].key, a) < 0)) {
                a = rj->vec[pos[j]].key;
                have = 1;
            }
        }
        if (!have) break;
        double v = 0.0;
        if (pos[k] < rk->n && key_cmp(rk->vec[pos[k]].key, a) == 0) v = rk->vec[pos[k]++].amp;
        int changed = 0;
        for (int j = 0; j < k; ++j) {
            const or_run *rj = runs[j];
            if (pos[j] < rj->n && key_cmp(rj->vec[pos[j]].key, a) == 0) {
                double cj = rj->vec[pos[j]++].amp;
                if (f32) v = (double)((float)v - (float)alpha[j] * (float)cj);
                else v = v - alpha[j] * cj;
                changed = 1;
            }
        }
        double out = v;
        if (changed && rk->pr.mode != OR_DETERMINISTIC) {
            if (v == 0.0) continue;
            if (fabs(v) < rk->pr.threshold) {
                uint32_t w[4];
                draw(&rk->pr, step, 0xFFFFFFFCu, rng_h(&rk->md, a), w);
                if (!(uniform53(w) < fabs(v) / rk->pr.threshold)) continue;
                out = store_round(rk->pr.mode, copysign(rk->pr.threshold, v));
            }
        }
        if (out == 0.0) continue;
        nv[nn].key = a;
        nv[nn].amp = out;
        nn++;
    }
    free(pos);
    free(rk->vec);
    rk->vec = nv; rk->n = nn; rk->cap = cap;
    return 0;
}

/* nsteps steps of K runs (one model, K <= 8): every run's new vector, then
 * runs 1..K-1 orthogonalised in order, then each run's norm, shift update
 * and history row.  Returns -1 for integer walkers, -5 when a population
 * died. */
int or_spectral_step(void **pruns, int K, long nsteps) {
    or_run *runs[8];
    if (K < 1 || K > 8) return -1;
    for (int k = 0; k < K; ++k) runs[k] = (or_run *)pruns[k];
    for (long n = 0; n < nsteps; ++n) {
        step_counts sc[8];
        for (int k = 0; k < K; ++k) step_vector(runs[k], &sc[k]);
        for (int k = 1; k < K; ++k)
            if (orthogonalise(runs, k)) return -1;
        for (int k = 0; k < K; ++k) {
            int rc = step_finish(runs[k], &sc[k]);
            if (rc) return rc;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* exact diagonalisation support: breadth-first search over the column graph
 * from a start address (Sec. 5), collecting every matrix element.          */

typedef struct { okey *k; long *v; long cap; } omap;

static uint64_t mapkey_hash(okey k) { return splitmix64(k.lo ^ splitmix64(k.hi)); }

static long map_find(const omap *m, okey k) {
    uint64_t i = mapkey_hash(k) & (uint64_t)(m->cap - 1);
    while (m->v[i] >= 0) {
        if (key_cmp(m->k[i], k) == 0) return m->v[i];
        i = (i + 1) & (uint64_t)(m->cap - 1);
    }
    return -1;
}

static void map_put(omap *m, okey k, long v) {
    uint64_t i = mapkey_hash(k) & (uint64_t)(m->cap - 1);
    while (m->v[i] >= 0) i = (i + 1) & (uint64_t)(m->cap - 1);
    m->k[i] = k; m->v[i] = v;
}

/* Writes the basis (BFS order) into basis[] and the nonzeros (row, col, val)
 * of H, diagonal included.  Returns the dimension, or -1 if max_dim or
 * nnz_cap is exceeded. */
long or_build_sparse(const void *pm, const okey *start, long max_dim, okey *basis, long nnz_cap,
                     int64_t *rows, int64_t *cols, double *vals, int64_t *nnz_out) {
    const or_model *md = (const or_model *)pm;
    long cap = 16;
    while (cap < 2 * max_dim) cap *= 2;
    omap mp;
    mp.cap = cap;
    mp.k = (okey *)malloc(sizeof(okey) * (size_t)cap);
    mp.v = (long *)malloc(sizeof(long) * (size_t)cap);
    for (long i = 0; i < cap; ++i) mp.v[i] = -1;
    long dim = 0, head = 0;
    int64_t nnz = 0;
    basis[dim] = *start; map_put(&mp, *start, dim); dim++;
    uint8_t occ[OR_MAXM];
    colent *col = NULL;
    long colcap = 0;
    while (head < dim) {
        okey k = basis[head];
        decode_key(md, k, occ);
        long m = column(md, occ, NULL, 0);
        if (m > colcap) { colcap = m; col = (colent *)realloc(col, sizeof(colent) * (size_t)colcap); }
        column(md, occ, col, m);
        if (nnz + m + 1 > nnz_cap) { dim = -1; break; }
        rows[nnz] = head; cols[nnz] = head; vals[nnz] = diagonal(md, occ); nnz++;
        for (long i = 0; i < m; ++i) {
            long j = map_find(&mp, col[i].key);
            if (j < 0) {
                if (dim >= max_dim) { dim = -1; break; }
                j = dim; basis[dim] = col[i].key; map_put(&mp, col[i].key, dim); dim++;
            }
            /* column of `head`: H[j][head] */
            rows[nnz] = j; cols[nnz] = head; vals[nnz] = col[i].val; nnz++;
        }
        if (dim < 0) break;
        head++;
    }
    free(col); free(mp.k); free(mp.v);
    *nnz_out = nnz;
    return dim;
}
