// fq_api.cu -- host side of libfciqmc: the C ABI declared in fciqmc.h.
//
// A run owns its device buffers (hash-segmented walker vector, double
// buffered; spawn buckets; per-segment partial sums; state and history ring)
// and a one-run batch.  A batch owns a device table of run descriptors, the
// segment -> run map and CUDA graphs of 1 and 16 steps; each step is three
// launches whatever the number of runs (k_spawn, k_merge, k_shift).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fciqmc.h"
#include "fq_kernels.cuh"
#include "fq_launch.h"
#include "fq_shared.h"

using namespace fq;

// ---------------------------------------------------------------------------
// kernel table

namespace fq {
void register_k64_int(KernelSet*);
void register_k64_f64(KernelSet*);
void register_k64_f32(KernelSet*);
void register_k128_int(KernelSet*);
void register_k128_f64(KernelSet*);
void register_k128_f32(KernelSet*);

static KernelSet g_sets[2][3][3];
static std::once_flag g_sets_once;

const KernelSet* kernel_set(int kw, int amp, int kind) {
    std::call_once(g_sets_once, [] {
        register_k64_int(g_sets[0][FQ_AMP_INT]);
        register_k64_f64(g_sets[0][FQ_AMP_F64]);
        register_k64_f32(g_sets[0][FQ_AMP_F32]);
        register_k128_int(g_sets[1][FQ_AMP_INT]);
        register_k128_f64(g_sets[1][FQ_AMP_F64]);
        register_k128_f32(g_sets[1][FQ_AMP_F32]);
    });
    if (kw < 1 || kw > 2 || amp < 0 || amp > 2 || kind < 1 || kind > 3) return nullptr;
    return &g_sets[kw - 1][amp][kind - 1];
}

void launch_shift(const RunDesc* runs, int nruns, cudaStream_t s) {
    k_shift<256><<<nruns, 256, 0, s>>>(runs);
}

static void launch_factors(const RunDesc* runs, int nruns, cudaStream_t s) {
    k_factors<<<nruns, 256, 0, s>>>(runs);
}

// tables of sqrt(k), hop values and m / n for a model (device memory)
struct Tables {
    double *sq, *hop, *r64;
    float *hop32, *r32;
    int kmax, mmax;
};
}  // namespace fq

// ---------------------------------------------------------------------------
// handles

struct fq_ham {
    ModelParams mp;
    int kw;  // 64-bit words per address
};

struct Alloc {
    void* p;
    size_t bytes;
};

struct fq_run {
    fq_ham ham;
    fq_params prm;
    cudaStream_t stream;
    fq_allocator alloc;
    bool has_alloc;
    int amp, det;
    const KernelSet* ks;
    int log2B;
    unsigned B, Cv, Cs, slots;  // slots: on-chip table slots per merge warp
    unsigned Cp;                // spawn slots per bucket in the dense primary region
    bool no_spawn_buf;          // a failed growth left no spawn buffers: the run cannot step
    RunState* st;
    StatsRow* hist;
    unsigned* vcount[2];
    void* vkeys[2];
    void* vamps[2];
    void* skeys;
    void* samps;
    unsigned* sfill;
    double *part_h, *part_v;
    Tables tab;
    int smax;
    double* fac64;
    float* del32;
    RunDesc* d_self;       // this run's descriptor in device memory
    unsigned* ref_bkt;
    unsigned n_ref_bkt;
    void* ref_keys;
    double *ref_h, *ref_v;
    unsigned* ref_off;
    size_t ref_cap;
    unsigned long long hist_read;
    bool seeded;
    std::vector<Alloc> allocs;
    fq_batch* single;
    LaunchCfg tuned;
    bool has_tuned;
    unsigned scratch_slots;  // global scratch table size for buckets too big for SW
    unsigned forced_slots, forced_scratch;  // fq_run_set_tables overrides (0 = none)
    unsigned sort_elems;   // global sort workspace per merge warp (elements)
    unsigned gen;  // bumped whenever a device pointer of the run changes
    unsigned last_err_bits;  // device error bits reported by the last check
    double* pinned;        // host staging slot for parameter updates
    cudaEvent_t staged;    // completes when the staged value has been copied
};

struct fq_batch {
    std::vector<fq_run*> runs;
    const KernelSet* ks;
    cudaStream_t stream;
    RunDesc* d_desc;
    unsigned* d_seg_run;
    unsigned G;
    LaunchCfg cfg;
    cudaGraphExec_t g1, g16;
    bool owned_by_run;
    std::vector<unsigned> gens;  // run generations the descriptors were built from
    unsigned char* scratch;      // merge scratch tables (from runs[0]'s allocator)
    size_t scratch_bytes;
    unsigned scratch_ss;         // table size the scratch was last cleared for
    unsigned char* sort_scratch;  // sort workspaces (from runs[0]'s allocator)
    size_t sort_scratch_bytes;
    std::vector<LaunchCfg> shapes;  // launch shapes the scratch was sized for
    float arm_ms[2];             // the autotuner's best mean merge time per arm (0: untimed)
    // replica overlaps (fq_batch_set_overlaps)
    bool ov_on;
    int ov_nq;
    int ov_d[FQ_MAX_G2];
    OverlapDesc* d_ov;
    double* ov_part;
    size_t ov_part_n;
    double* ov_ring;
    unsigned long long* ov_head;
    unsigned ov_cap, ov_table;
    int ov_grid, ov_wpb;
    unsigned long long ov_read;  // rows handed out so far
    // excited states (fq_batch_set_spectral)
    int gs_K;
    GsDesc* d_gs;
    double* gs_part;
    double* gs_alpha;
    size_t gs_part_n;
    unsigned gs_table;
    int gs_grid, gs_wpb;
};

// ---------------------------------------------------------------------------
// small helpers

static int cuda_err(cudaError_t e) {
    if (e == cudaSuccess) return FQ_OK;
    if (e == cudaErrorMemoryAllocation) return FQ_ERR_NOMEM;
    return FQ_ERR_CUDA;
}
#define CK(x)                                      \
    do {                                           \
        cudaError_t _e = (x);                      \
        if (_e != cudaSuccess) return cuda_err(_e); \
    } while (0)

static void* dev_alloc(fq_run* r, size_t bytes) {
    if (!bytes) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (r->has_alloc) {
        p = r->alloc.alloc(r->alloc.ctx, bytes, (void*)r->stream);
    } else if (cudaMallocAsync(&p, bytes, r->stream) != cudaSuccess) {
        p = nullptr;
    }
    if (p) r->allocs.push_back({p, bytes});
    return p;
}

static void dev_free(fq_run* r, void* p) {
    for (size_t i = 0; i < r->allocs.size(); ++i)
        if (r->allocs[i].p == p) {
            if (r->has_alloc) r->alloc.free(r->alloc.ctx, p, r->allocs[i].bytes, (void*)r->stream);
            else cudaFreeAsync(p, r->stream);
            r->allocs.erase(r->allocs.begin() + (long)i);
            return;
        }
}

static void dev_free_all(fq_run* r) {
    for (auto& a : r->allocs) {
        if (r->has_alloc) r->alloc.free(r->alloc.ctx, a.p, a.bytes, (void*)r->stream);
        else cudaFreeAsync(a.p, r->stream);
    }
    r->allocs.clear();
}

static unsigned next_pow2(unsigned long long x) {
    unsigned p = 1;
    while (p < x) p <<= 1;
    return p;
}

static int ilog2(unsigned x) {
    int l = 0;
    while ((1u << l) < x) ++l;
    return l;
}

static int num_sms() {
    static int n = -1;
    if (n < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 1;
    }
    return n;
}

// ---------------------------------------------------------------------------
// host-side address codec (Sec. 6.1)

static bool key_bit(const fq_key& k, int p) { return p < 64 ? (k.lo >> p) & 1u : (k.hi >> (p - 64)) & 1u; }
static void key_set(fq_key& k, int p) {
    if (p < 64) k.lo |= 1ull << p; else k.hi |= 1ull << (p - 64);
}
static bool key_less(const fq_key& a, const fq_key& b) { return a.hi != b.hi ? a.hi < b.hi : a.lo < b.lo; }
static bool key_same(const fq_key& a, const fq_key& b) { return a.hi == b.hi && a.lo == b.lo; }

static bool key_valid(const fq_ham* h, const fq_key& k) {
    int ones = 0;
    for (int p = 0; p < 128; ++p)
        if (key_bit(k, p)) {
            if (p >= h->mp.nbits) return false;
            ++ones;
        }
    return ones == h->mp.N;
}

// ---------------------------------------------------------------------------
// C ABI: misc

extern "C" const char* fq_version(void) { return "fciqmc-gb300 0.1 (sm_103a)"; }

extern "C" const char* fq_strerror(int code) {
    switch (code) {
    case FQ_OK: return "ok";
    case FQ_ERR_INVALID: return "invalid argument";
    case FQ_ERR_NOMEM: return "device allocation failed";
    case FQ_ERR_CAPACITY: return "capacity exceeded (step rolled back)";
    case FQ_ERR_TIMEOUT: return "device wait timed out (step rolled back)";
    case FQ_ERR_EMPTY: return "population died (step rolled back)";
    case FQ_ERR_CUDA: return "CUDA error or no usable device";
    default: return "unknown error";
    }
}

extern "C" int fq_params_default(fq_params* p) {
    if (!p) return FQ_ERR_INVALID;
    memset(p, 0, sizeof *p);
    p->dt = 0.01;
    p->target = 1000.0;
    p->zeta = 0.08;
    p->xi = 0.08 * 0.08 / 4.0;  // zeta^2 / 4, as fq_params_set_zeta
    p->threshold = 1.0;
    p->t_rel = 1.0;
    p->mode = FQ_MODE_REAL64;
    p->annihilation = FQ_ANN_AUTO;
    p->seed = 1;
    p->run_id = 0;
    return FQ_OK;
}

extern "C" int fq_params_set_zeta(fq_params* p, double zeta) {
    if (!p || !std::isfinite(zeta) || !(zeta >= 0)) return FQ_ERR_INVALID;
    p->zeta = zeta;
    p->xi = zeta * zeta / 4.0;
    return FQ_OK;
}

// ---------------------------------------------------------------------------
// C ABI: Hamiltonians

extern "C" int fq_ham_create(fq_ham** out, int kind, int Lx, int Ly, int N, double t, double u) {
    if (!out) return FQ_ERR_INVALID;
    *out = nullptr;
    if (N < 1 || N > 255) return FQ_ERR_INVALID;
    int M;
    if (kind == FQ_BH_REAL_2D) {
        if (Lx < 3 || Ly < 3) return FQ_ERR_INVALID;
        M = Lx * Ly;
    } else if (kind == FQ_BH_REAL_1D) {
        if (Lx < 3 || Ly != 1) return FQ_ERR_INVALID;
        M = Lx;
    } else if (kind == FQ_BH_MOM_1D) {
        if (Lx < 2 || Lx > FQ_MAX_MOM_MODES || Ly != 1) return FQ_ERR_INVALID;
        M = Lx;
    } else {
        return FQ_ERR_INVALID;
    }
    if (N + M - 1 > 128 || !std::isfinite(t) || !std::isfinite(u)) return FQ_ERR_INVALID;
    fq_ham* h = new (std::nothrow) fq_ham;
    if (!h) return FQ_ERR_NOMEM;
    memset(h, 0, sizeof *h);
    ModelParams& mp = h->mp;
    mp.kind = kind; mp.M = M; mp.N = N; mp.Lx = Lx; mp.Ly = Ly; mp.nbits = N + M - 1;
    mp.t = t; mp.u = u;
    mp.g = u / (double)(2 * M);
    if (kind != FQ_BH_MOM_1D) {
        // directions (+x, -x, +y, -y) on the periodic lattice, site x + Lx y
        for (int s2 = 0; s2 < M; ++s2) {
            const int x = s2 % Lx, y = s2 / Lx;
            mp.nbr[0][s2] = (unsigned char)((x + 1) % Lx + Lx * y);
            mp.nbr[1][s2] = (unsigned char)((x + Lx - 1) % Lx + Lx * y);
            mp.nbr[2][s2] = (unsigned char)(x + Lx * ((y + 1) % Ly));
            mp.nbr[3][s2] = (unsigned char)(x + Lx * ((y + Ly - 1) % Ly));
        }
    }
    if (kind == FQ_BH_MOM_1D) {
        // mode j (1-based) carries k_j = 2 pi (j - floor(M/2)) / M
        for (int m = 0; m < M; ++m) {
            double k = (2.0 * M_PI * (double)(m + 1 - M / 2)) / (double)M;
            mp.eps[m] = (-2.0 * t) * cos(k);
        }
    }
    h->kw = mp.nbits <= 64 ? 1 : 2;
    *out = h;
    return FQ_OK;
}

extern "C" void fq_ham_destroy(fq_ham* h) { delete h; }

extern "C" int fq_ham_info(const fq_ham* h, int* M, int* nbits, int* key_words) {
    if (!h) return FQ_ERR_INVALID;
    if (M) *M = h->mp.M;
    if (nbits) *nbits = h->mp.nbits;
    if (key_words) *key_words = h->kw;
    return FQ_OK;
}

extern "C" int fq_ham_dimension(const fq_ham* h, double* dim) {
    if (!h || !dim) return FQ_ERR_INVALID;
    // C(N + M - 1, N): exact in 128-bit integers while it fits, else FP64
    unsigned __int128 c = 1;
    bool exact = true;
    for (int i = 1; i <= h->mp.N && exact; ++i) {
        const unsigned __int128 f = (unsigned __int128)(h->mp.M - 1 + i);
        if (c > (~(unsigned __int128)0) / f) exact = false;
        else c = c * f / (unsigned __int128)i;
    }
    if (exact) {
        *dim = (double)c;
    } else {
        double d = 1.0;
        for (int i = 1; i <= h->mp.N; ++i) d = d * (double)(h->mp.M - 1 + i) / (double)i;
        *dim = d;
    }
    return FQ_OK;
}

extern "C" int fq_encode(const fq_ham* h, const uint8_t* occ, fq_key* out) {
    if (!h || !occ || !out) return FQ_ERR_INVALID;
    int s = 0;
    for (int m = 0; m < h->mp.M; ++m) s += occ[m];
    if (s != h->mp.N) return FQ_ERR_INVALID;
    fq_key k = {0, 0};
    int pos = 0;
    for (int m = 0; m < h->mp.M; ++m) {
        for (int j = 0; j < occ[m]; ++j) key_set(k, pos++);
        if (m < h->mp.M - 1) ++pos;
    }
    *out = k;
    return FQ_OK;
}

extern "C" int fq_decode(const fq_ham* h, fq_key key, uint8_t* occ) {
    if (!h || !occ || !key_valid(h, key)) return FQ_ERR_INVALID;
    memset(occ, 0, (size_t)h->mp.M);
    int m = 0;
    for (int p = 0; p < h->mp.nbits; ++p) {
        if (key_bit(key, p)) occ[m]++;
        else ++m;
    }
    return FQ_OK;
}

extern "C" int fq_ham_starting_address(const fq_ham* h, fq_key* out) {
    if (!h || !out) return FQ_ERR_INVALID;
    std::vector<uint8_t> occ((size_t)h->mp.M, 0);
    if (h->mp.kind == FQ_BH_MOM_1D) {
        occ[(size_t)(h->mp.M / 2 - 1)] = (uint8_t)h->mp.N;
    } else {
        for (int m = 0; m < h->mp.M; ++m)
            occ[(size_t)m] = (uint8_t)(h->mp.N / h->mp.M + (m < h->mp.N % h->mp.M ? 1 : 0));
    }
    return fq_encode(h, occ.data(), out);
}

// device buffers of one call, released on every return path
struct CallBufs {
    std::vector<void*> p;
    ~CallBufs() {
        for (void* q : p) cudaFree(q);
    }
    template <class T> cudaError_t get(T** out, size_t bytes) {
        void* q = nullptr;
        const cudaError_t e = cudaMalloc(&q, bytes);
        if (e == cudaSuccess) p.push_back(q);
        *out = (T*)q;
        return e;
    }
};

static int ham_column_dev(const fq_ham* h, int amp, fq_key key, double* diag, fq_key* dest,
                          double* val, size_t cap, size_t* m_out, cudaStream_t s) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return FQ_ERR_CUDA;
    const KernelSet* ks = kernel_set(h->kw, amp, h->mp.kind);
    const size_t kb = ks->key_bytes;
    const unsigned ccap = (unsigned)std::min<size_t>(cap, 1u << 20);
    CallBufs bufs;
    void* d_dest = nullptr;
    double *d_val = nullptr, *d_diag = nullptr;
    unsigned* d_m = nullptr;
    CK(bufs.get(&d_dest, kb * (ccap ? ccap : 1)));
    CK(bufs.get(&d_val, sizeof(double) * (ccap ? ccap : 1)));
    CK(bufs.get(&d_diag, sizeof(double)));
    CK(bufs.get(&d_m, sizeof(unsigned)));
    unsigned char kbuf[16];
    memcpy(kbuf, &key, 16);
    ModelParams mp = h->mp;
    mp.kmax = (mp.N + 1) * (mp.N + 2);
    double *d_sq = nullptr, *d_hop = nullptr;
    float* d_hop32 = nullptr;
    CK(bufs.get(&d_sq, sizeof(double) * (mp.kmax + 1)));
    CK(bufs.get(&d_hop, sizeof(double) * (mp.kmax + 1)));
    CK(bufs.get(&d_hop32, sizeof(float) * (mp.kmax + 1)));
    k_tables<<<(unsigned)((mp.kmax + 256) / 256), 256, 0, s>>>(mp.t, mp.kmax, d_sq, d_hop, d_hop32);
    mp.sqrt_tab = d_sq;
    mp.hop_tab = d_hop;
    mp.hop32_tab = d_hop32;
    ks->column(mp, kbuf, d_dest, d_val, ccap, d_diag, d_m, s);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    unsigned m = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&m, d_m, sizeof m, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && diag) e = cudaMemcpy(diag, d_diag, sizeof(double), cudaMemcpyDeviceToHost);
    const size_t nw = std::min<size_t>(m, ccap);
    if (e == cudaSuccess && nw && val) e = cudaMemcpy(val, d_val, sizeof(double) * nw, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && nw && dest) {
        std::vector<unsigned char> tmp(kb * nw);
        e = cudaMemcpy(tmp.data(), d_dest, kb * nw, cudaMemcpyDeviceToHost);
        for (size_t i = 0; i < nw; ++i) {
            fq_key k = {0, 0};
            memcpy(&k, tmp.data() + i * kb, kb);
            dest[i] = k;
        }
    }
    if (m_out) *m_out = m;
    return cuda_err(e);
}

extern "C" int fq_ham_column(const fq_ham* h, fq_key key, double* diag, fq_key* dest, double* val,
                             size_t cap, size_t* m) {
    if (!h || !key_valid(h, key)) return FQ_ERR_INVALID;
    return ham_column_dev(h, FQ_AMP_F64, key, diag, dest, val, cap, m, 0);
}

// ---------------------------------------------------------------------------
// runs: sizing and creation

static size_t max_offdiag(const ModelParams& mp) {
    const size_t nocc = (size_t)std::min(mp.N, mp.M);
    if (mp.kind == FQ_BH_REAL_1D) return 2 * nocc;
    if (mp.kind == FQ_BH_REAL_2D) return 4 * nocc;
    return (nocc * (nocc + 1) / 2) * (size_t)(mp.M / 2 + 1);
}

// the run's model with its device tables: every kernel that evaluates
// matrix elements of the run gets this copy
static ModelParams run_mp(const fq_run* r) {
    ModelParams mp = r->ham.mp;
    mp.kmax = r->tab.kmax;
    mp.sqrt_tab = r->tab.sq;
    mp.hop_tab = r->tab.hop;
    mp.hop32_tab = r->tab.hop32;
    return mp;
}

static void fill_desc(const fq_run* r, RunDesc& d, unsigned seg_base) {
    memset(&d, 0, sizeof d);
    d.mp = run_mp(r);
    d.amp = r->amp;
    d.mode_det = r->det;
    d.theta = r->prm.threshold;
    d.theta32 = (float)r->prm.threshold;
    d.t_rel = r->prm.t_rel;
    d.trel_one = r->prm.t_rel == 1.0;
    d.early = r->prm.compression == FQ_COMPRESS_EARLY && !r->det && r->amp != FQ_AMP_INT;
    {
        int e = 0;
        const double fr = r->det || r->amp == FQ_AMP_INT ? 0.0 : std::frexp(r->prm.threshold, &e);
        d.theta_pow2 = fr == 0.5;
        d.theta_exp = e - 1;  // threshold = 2^(e-1) when fr == 1/2
        d.norm_q = r->amp == FQ_AMP_INT || r->det ? 0 : std::ilogb(r->prm.threshold) - 52;
    }
    d.mmax = r->tab.mmax;
    d.coef64 = r->tab.r64;
    d.coef32 = r->tab.r32;
    d.smax = r->smax;
    d.fac64 = r->fac64;
    d.del32 = r->del32;
    d.ref_bkt = r->ref_bkt;
    d.n_ref_bkt = r->n_ref_bkt;
    d.key_x = (unsigned)r->prm.seed;
    d.key_y = (unsigned)(r->prm.seed >> 32) ^ (unsigned)(r->prm.run_id * 0x9E3779B9u);
    d.log2B = r->log2B;
    d.B = r->B;
    d.seg_base = seg_base;
    d.Cv = r->Cv;
    d.Cs = r->Cs;
    d.Cp = r->Cp;
    for (int i = 0; i < 2; ++i) {
        d.vkeys[i] = r->vkeys[i];
        d.vamps[i] = r->vamps[i];
        d.vcount[i] = r->vcount[i];
    }
    d.skeys = r->skeys;
    d.samps = r->samps;
    d.sfill = r->sfill;
    d.st = r->st;
    d.hist = r->hist;
    d.ref_keys = r->ref_keys;
    d.ref_h = r->ref_h;
    d.ref_v = r->ref_v;
    d.ref_off = r->ref_off;
    d.part_h = r->part_h;
    d.part_v = r->part_v;
}

static cudaError_t sync_self(fq_run* r) {
    RunDesc hd;
    fill_desc(r, hd, 0);
    cudaError_t e = cudaMemcpyAsync(r->d_self, &hd, sizeof hd, cudaMemcpyHostToDevice, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    return e;
}

// a launch shape: persistent grids of one (spawn) or a few (merge) blocks per
// SM, sized by occupancy; at most one warp per segment
static LaunchCfg make_cfg(const KernelSet* ks, int spawn_var, int spawn_waves, int merge_var,
                          unsigned slots, unsigned G, int ann) {
    LaunchCfg c;
    memset(&c, 0, sizeof c);
    const int spawn_wpb = variant_wpb(spawn_var), merge_wpb = variant_wpb(merge_var);
    c.ann = ann;
    c.spawn_var = spawn_var;
    c.spawn_wpb = spawn_wpb;
    c.merge_var = merge_var;
    c.merge_wpb = merge_wpb;
    c.slots = slots;
    c.scratch_slots = 0;
    c.scratch = nullptr;
    const int sms = num_sms();
    int occ_s = ks->spawn_occupancy(spawn_var);
    const size_t smem = ks->merge_smem(ann, merge_wpb, slots);
    int occ_m = ks->merge_occupancy(ann, merge_var, smem);
    if (occ_s < 1) occ_s = 1;
    if (occ_m < 1) occ_m = 1;
    const long long ws = ((long long)G + spawn_wpb - 1) / spawn_wpb;
    const long long wm = ((long long)G + merge_wpb - 1) / merge_wpb;
    c.spawn_grid = (int)std::max<long long>(1, std::min<long long>((long long)sms * occ_s * spawn_waves, ws));
    c.merge_grid = (int)std::max<long long>(1, std::min<long long>((long long)sms * occ_m, wm));
    return c;
}

// on-chip table slots per merge warp: 512, fewer if a warp's share of
// shared memory would not allow two 8-warp blocks per SM (2 x (112 KB +
// the 1 KB the SM reserves per block) within its 228 KB).  The bucket count
// follows (a bucket's spawns fill about a third of the table), so the
// larger table also means fewer, fuller buckets: on the 127-bit c5
// workload 512 slots and 2^22 buckets stepped 12 % faster than 256 slots
// and 2^23 buckets (fewer per-bucket costs in the merge; fewer counters
// and a denser primary region for the spawn stores).
static unsigned warp_slots(const KernelSet* ks) {
    unsigned sw = 512;
    while (sw > 128 && 8ull * sw * ks->slot_bytes > 112u * 1024u) sw >>= 1;
    return sw;
}

// the merge's table sizes of a run: on-chip slots per warp, and the global
// scratch table, which holds any bucket within the run's capacities
// (Cv + Cs <= 0.9 of its slots), unless fq_run_set_tables overrode them
static void table_sizes(fq_run* r) {
    r->slots = r->forced_slots ? r->forced_slots : warp_slots(r->ks);
    r->scratch_slots =
        r->forced_scratch
            ? r->forced_scratch
            : std::max(r->slots, next_pow2((unsigned long long)std::ceil((r->Cv + r->Cs) / 0.9)));
    // the sort arm's workspace holds a bucket's entries and spawns (16-bit
    // indices: at most 32768 elements; a larger bucket fails the step)
    r->sort_elems = (unsigned)std::min<unsigned long long>(
        32768, next_pow2((unsigned long long)r->Cv + r->Cs));
}

// per-segment capacities for totals lcap, scap over B segments (spawns
// arrive in clumps of up to k, see fq_run_create)
static void segment_caps(double lcap, double scap, unsigned B, double k, unsigned& Cv, unsigned& Cs) {
    const double mv = lcap / B, ms = scap / B;
    Cv = (unsigned)((mv + 4.0 * std::sqrt(mv) + 16.0 + 31.0) / 32.0) * 32u;
    Cs = (unsigned)((ms + 4.0 * std::sqrt(ms * k) + k + 16.0 + 31.0) / 32.0) * 32u;
}

// Spawn slots per bucket in the dense primary region: the steady-state fill
// plus three standard deviations of its compound-Poisson count (a multiple
// of 32, at most the bucket's capacity), so that nearly every spawn of an
// equilibrated run is stored there.
static unsigned primary_slots(double s_ss, unsigned B, double k, unsigned Cs) {
    const double m = s_ss / B;
    const unsigned p = (unsigned)((m + 3.0 * std::sqrt(m * k) + 16.0 + 31.0) / 32.0) * 32u;
    return std::min(p, Cs);
}

static void batch_free(fq_batch* b);
static int batch_build(fq_batch* b);

extern "C" int fq_run_create(fq_run** out, const fq_ham* h, const fq_params* p, void* stream,
                             const fq_allocator* alloc) {
    if (!out || !h || !p) return FQ_ERR_INVALID;
    *out = nullptr;
    if (!(p->dt > 0) || !(p->target > 0) || !(p->zeta >= 0) || !(p->xi >= 0) || !(p->t_rel > 0))
        return FQ_ERR_INVALID;
    if (p->mode < FQ_MODE_INT || p->mode > FQ_MODE_DETERMINISTIC) return FQ_ERR_INVALID;
    if (p->mode != FQ_MODE_DETERMINISTIC && p->mode != FQ_MODE_INT && !(p->threshold > 0))
        return FQ_ERR_INVALID;
    if (p->annihilation != FQ_ANN_AUTO && p->annihilation != FQ_ANN_HASH &&
        p->annihilation != FQ_ANN_SORT)
        return FQ_ERR_INVALID;
    if (p->compression != FQ_COMPRESS_LATE && p->compression != FQ_COMPRESS_EARLY)
        return FQ_ERR_INVALID;
    if (p->mode == FQ_MODE_INT && p->target > 1e12) return FQ_ERR_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return FQ_ERR_CUDA;

    fq_run* r = new (std::nothrow) fq_run();
    if (!r) return FQ_ERR_NOMEM;
    r->ham = *h;
    r->prm = *p;
    r->stream = (cudaStream_t)stream;
    r->has_alloc = alloc && alloc->alloc && alloc->free;
    if (r->has_alloc) r->alloc = *alloc;
    r->amp = p->mode == FQ_MODE_INT ? FQ_AMP_INT : p->mode == FQ_MODE_REAL32 ? FQ_AMP_F32 : FQ_AMP_F64;
    r->det = p->mode == FQ_MODE_DETERMINISTIC;
    r->ks = kernel_set(h->kw, r->amp, h->mp.kind);

    // capacities: after compression every entry has |c| >= threshold, so
    // len <= norm / threshold; spawns per step <= norm * max(1, t_rel) + len
    double dim = 0;
    fq_ham_dimension(h, &dim);
    const double th = r->det ? 1.0 : (p->mode == FQ_MODE_INT ? 1.0 : std::min(1.0, p->threshold));
    // the spawn count follows the norm, not the occupied count: when the
    // vector fills a small Hilbert space its entries grow and spawn more
    const double lnorm = p->capacity_vec ? (double)p->capacity_vec : 2.0 * p->target / th + 1024.0;
    double lcap = lnorm;
    if (r->det && !p->capacity_vec) lcap = std::min(dim * 1.05 + 1024.0, 1.0e9);
    lcap = std::min(lcap, dim * 1.05 + 1024.0);
    double scap = p->capacity_spawn ? (double)p->capacity_spawn
                                    : 1.5 * lnorm * std::max(1.0, p->t_rel) + 4096.0;
    if (r->det && !p->capacity_spawn) scap = lcap * (double)max_offdiag(h->mp) + 4096.0;
    if (lcap > 4.0e9 || scap > 8.0e9) {
        delete r;
        return FQ_ERR_INVALID;
    }
    const size_t kb = r->ks->key_bytes, ab = r->ks->amp_bytes, sb = r->ks->spawn_bytes;
    // segments: at the expected steady state (len ~ target / threshold,
    // spawns ~ len) the spawns into a bucket fill about a third of one merge
    // warp's on-chip table (the table holds spawned addresses only)
    r->slots = warp_slots(r->ks);
    double l_ss = std::min(p->target / th, dim), s_ss = 1.1 * p->target / th;
    if (r->det) {
        l_ss = std::min(lcap, dim);
        s_ss = l_ss * (double)max_offdiag(h->mp);
    }
    const unsigned long long want =
        (unsigned long long)std::ceil(s_ss / (r->slots / 3.0));
    r->B = next_pow2(std::max<unsigned long long>(1, std::min<unsigned long long>(want, 1ull << 28)));
    {
        // spawns arrive in clumps (one address receives spawns from many
        // sources; every neighbour's in the deterministic limit), so the
        // bucket count fluctuates like a compound Poisson sum with clump size k
        const double k = r->det ? (double)max_offdiag(h->mp) : 8.0;
        segment_caps(lcap, scap, r->B, k, r->Cv, r->Cs);
        r->Cp = primary_slots(s_ss, r->B, k, r->Cs);
        table_sizes(r);
    }
    r->log2B = ilog2(r->B);
    const unsigned B = r->B;

    bool ok = true;
    auto A = [&](size_t bytes) {
        void* q = dev_alloc(r, bytes);
        if (!q) ok = false;
        return q;
    };
    r->st = (RunState*)A(sizeof(RunState));
    r->hist = (StatsRow*)A(sizeof(StatsRow) * FQ_HIST_CAP);
    for (int i = 0; i < 2; ++i) {
        r->vcount[i] = (unsigned*)A(sizeof(unsigned) * B);
        r->vkeys[i] = A(kb * (size_t)B * r->Cv);
        r->vamps[i] = A(ab * (size_t)B * r->Cv);
    }
    r->skeys = A(r->ks->spawn_key_stride * (size_t)B * r->Cs);
    r->samps = A(std::max<size_t>(16, r->ks->spawn_val_stride * (size_t)B * r->Cs));
    r->sfill = (unsigned*)A(sizeof(unsigned) * B);
    r->part_h = (double*)A(sizeof(double) * B);
    r->part_v = (double*)A(sizeof(double) * B);
    r->ref_off = (unsigned*)A(sizeof(unsigned) * (B + 1));
    r->ref_bkt = (unsigned*)A(sizeof(unsigned) * 64 * 1024);
    r->n_ref_bkt = 0;
    // matrix-element tables; diagonal factors (real space)
    const ModelParams& mp0 = h->mp;
    r->tab.kmax = (mp0.N + 1) * (mp0.N + 2);
    r->tab.mmax = mp0.kind == FQ_BH_MOM_1D ? 0 : (int)max_offdiag(mp0);
    r->tab.sq = (double*)A(sizeof(double) * (r->tab.kmax + 1));
    r->tab.hop = (double*)A(sizeof(double) * (r->tab.kmax + 1));
    r->tab.hop32 = (float*)A(sizeof(float) * (r->tab.kmax + 1));
    const size_t nrat = mp0.kind == FQ_BH_MOM_1D ? 0 : (size_t)(r->tab.mmax + 1) * (r->tab.mmax + 1);
    r->tab.r64 = nrat ? (double*)A(sizeof(double) * nrat) : nullptr;
    r->tab.r32 = nrat ? (float*)A(sizeof(float) * nrat) : nullptr;
    r->smax = mp0.kind == FQ_BH_MOM_1D ? -1 : mp0.N * (mp0.N - 1);
    r->fac64 = r->smax >= 0 ? (double*)A(sizeof(double) * (r->smax + 1)) : nullptr;
    r->del32 = r->smax >= 0 ? (float*)A(sizeof(float) * (r->smax + 1)) : nullptr;
    r->d_self = (RunDesc*)A(sizeof(RunDesc));
    r->ref_cap = 0;
    r->ref_keys = nullptr;
    r->ref_h = r->ref_v = nullptr;
    if (!ok) {
        dev_free_all(r);
        cudaStreamSynchronize(r->stream);
        delete r;
        return FQ_ERR_NOMEM;
    }

    RunState s0;
    memset(&s0, 0, sizeof s0);
    s0.dt = p->dt;
    s0.target = p->target;
    s0.zeta = p->zeta;
    s0.xi = p->xi;
    s0.norm = 1.0;
    cudaError_t e = cudaMemcpyAsync(r->st, &s0, sizeof s0, cudaMemcpyHostToDevice, r->stream);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = cudaMemsetAsync(r->vcount[i], 0, sizeof(unsigned) * B, r->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->sfill, 0, sizeof(unsigned) * B, r->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->ref_off, 0, sizeof(unsigned) * (B + 1), r->stream);
    if (e == cudaSuccess) {
        const long long nt = r->tab.kmax + 1;
        k_tables<<<(unsigned)((nt + 255) / 256), 256, 0, r->stream>>>(
            h->mp.t, r->tab.kmax, r->tab.sq, r->tab.hop, r->tab.hop32);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        RunDesc hd;
        fill_desc(r, hd, 0);
        e = cudaMemcpyAsync(r->d_self, &hd, sizeof hd, cudaMemcpyHostToDevice, r->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) {
        dev_free_all(r);
        delete r;
        return cuda_err(e);
    }
    r->seeded = false;
    r->hist_read = 0;
    r->single = nullptr;
    r->has_tuned = false;
    r->gen = 0;
    if (cudaMallocHost((void**)&r->pinned, sizeof(double)) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->staged, cudaEventDisableTiming) != cudaSuccess) {
        dev_free_all(r);
        cudaStreamSynchronize(r->stream);
        delete r;
        return FQ_ERR_NOMEM;
    }
    cudaEventRecord(r->staged, r->stream);
    *out = r;
    return FQ_OK;
}

extern "C" void fq_run_destroy(fq_run* r) {
    if (!r) return;
    cudaStreamSynchronize(r->stream);
    if (r->single) batch_free(r->single);
    dev_free_all(r);
    cudaStreamSynchronize(r->stream);
    cudaEventDestroy(r->staged);
    cudaFreeHost(r->pinned);
    delete r;
}

// ---------------------------------------------------------------------------
// runs: seeding and reference

static void pack_keys(const fq_key* keys, size_t n, size_t kb, std::vector<unsigned char>& out) {
    out.resize(kb * n);
    for (size_t i = 0; i < n; ++i) memcpy(out.data() + i * kb, &keys[i], kb);
}

extern "C" int fq_run_seed(fq_run* r, const fq_key* keys, const double* amps, size_t n,
                           double shift, int64_t step) {
    if (!r || (n && (!keys || !amps)) || !std::isfinite(shift)) return FQ_ERR_INVALID;
    std::vector<size_t> idx;
    idx.reserve(n);
    for (size_t i = 0; i < n; ++i) {
        if (!key_valid(&r->ham, keys[i]) || !std::isfinite(amps[i])) return FQ_ERR_INVALID;
        if (r->amp == FQ_AMP_INT && (amps[i] != std::floor(amps[i]) || std::fabs(amps[i]) > 9.0e15))
            return FQ_ERR_INVALID;
        if (amps[i] != 0.0) idx.push_back(i);
    }
    std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return key_less(keys[a], keys[b]); });
    for (size_t i = 1; i < idx.size(); ++i)
        if (key_same(keys[idx[i - 1]], keys[idx[i]])) return FQ_ERR_INVALID;
    const size_t m = idx.size();
    std::vector<fq_key> sk(m);
    std::vector<double> sa(m);
    double norm = 0.0;
    for (size_t i = 0; i < m; ++i) {
        sk[i] = keys[idx[i]];
        double a = amps[idx[i]];
        if (r->amp == FQ_AMP_F32) a = (double)(float)a;
        sa[i] = a;
        norm += std::fabs(a);
    }
    if (m > (size_t)r->B * r->Cv) return FQ_ERR_CAPACITY;
    CK(cudaStreamSynchronize(r->stream));
    const size_t kb = r->ks->key_bytes;
    std::vector<unsigned char> kbuf;
    pack_keys(sk.data(), m, kb, kbuf);
    void* d_k = nullptr;
    double* d_a = nullptr;
    CallBufs bufs;  // released on every return
    CK(bufs.get(&d_k, kb * (m ? m : 1)));
    CK(bufs.get(&d_a, sizeof(double) * (m ? m : 1)));
    RunState s0;
    memset(&s0, 0, sizeof s0);
    CK(cudaMemcpy(&s0, r->st, sizeof s0, cudaMemcpyDeviceToHost));
    s0.shift = shift;
    s0.norm = norm;
    s0.step = step;
    s0.len = (long long)m;
    s0.cur = 0;
    s0.err = 0;
    s0.n_exact = s0.n_inexact = s0.n_spawns = 0;
    s0.hist_head = 0;
    s0.last_hproj = s0.last_vproj = 0.0;
    s0.last_exact = s0.last_inexact = s0.last_spawns = 0;
    s0.norm_lo = s0.norm_hi = 0;
    s0.norm_fp = 0.0;
    s0.len_acc = 0;
    s0.merged_onchip = s0.merged_scratch = 0;
    cudaError_t e = cudaMemcpyAsync(r->st, &s0, sizeof s0, cudaMemcpyHostToDevice, r->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->vcount[0], 0, sizeof(unsigned) * r->B, r->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->vcount[1], 0, sizeof(unsigned) * r->B, r->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->sfill, 0, sizeof(unsigned) * r->B, r->stream);
    if (e == cudaSuccess && m) e = cudaMemcpyAsync(d_k, kbuf.data(), kb * m, cudaMemcpyHostToDevice, r->stream);
    if (e == cudaSuccess && m) e = cudaMemcpyAsync(d_a, sa.data(), sizeof(double) * m, cudaMemcpyHostToDevice, r->stream);
    if (e == cudaSuccess) {
        r->ks->seed(r->d_self, d_k, d_a, m, r->stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && r->smax >= 0) {
        launch_factors(r->d_self, 1, r->stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    unsigned err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, &r->st->err, sizeof err, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e);
    if (err) {
        unsigned z = 0;
        cudaMemset(r->vcount[0], 0, sizeof(unsigned) * r->B);
        cudaMemcpy(&r->st->err, &z, sizeof z, cudaMemcpyHostToDevice);
        r->seeded = false;
        return FQ_ERR_CAPACITY;
    }
    r->seeded = true;
    r->hist_read = 0;
    return FQ_OK;
}

extern "C" int fq_run_set_reference(fq_run* r, const fq_key* keys, const double* y, size_t n) {
    if (!r || n > 64 || (n && (!keys || !y))) return FQ_ERR_INVALID;
    for (size_t i = 0; i < n; ++i) {
        if (!key_valid(&r->ham, keys[i]) || !std::isfinite(y[i])) return FQ_ERR_INVALID;
        for (size_t j = 0; j < i; ++j)
            if (key_same(keys[i], keys[j])) return FQ_ERR_INVALID;
    }
    CK(cudaStreamSynchronize(r->stream));
    const size_t kb = r->ks->key_bytes;
    const unsigned B = r->B;
    if (n == 0) {
        CK(cudaMemset(r->ref_off, 0, sizeof(unsigned) * (B + 1)));
        r->n_ref_bkt = 0;
        r->gen++;
        CK(sync_self(r));
        return FQ_OK;
    }
    std::vector<unsigned char> kbuf;
    pack_keys(keys, n, kb, kbuf);
    void *d_refs = nullptr, *d_tk = nullptr;
    double *d_y = nullptr, *d_th = nullptr, *d_tv = nullptr;
    unsigned *d_cnt = nullptr, *d_off = nullptr, *d_tseg = nullptr;
    CallBufs bufs;  // released on every return
    CK(bufs.get(&d_refs, kb * n));
    CK(bufs.get(&d_y, sizeof(double) * n));
    CK(bufs.get(&d_cnt, sizeof(unsigned) * n));
    CK(cudaMemcpy(d_refs, kbuf.data(), kb * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_y, y, sizeof(double) * n, cudaMemcpyHostToDevice));
    const ModelParams mp = run_mp(r);
    r->ks->ref_count(mp, d_refs, (int)n, d_cnt, 0);
    std::vector<unsigned> cnt(n), off(n + 1, 0);
    CK(cudaMemcpy(cnt.data(), d_cnt, sizeof(unsigned) * n, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) off[i + 1] = off[i] + cnt[i];
    const size_t T = off[n];
    CK(bufs.get(&d_off, sizeof(unsigned) * (n + 1)));
    CK(bufs.get(&d_tk, kb * T));
    CK(bufs.get(&d_th, sizeof(double) * T));
    CK(bufs.get(&d_tv, sizeof(double) * T));
    CK(bufs.get(&d_tseg, sizeof(unsigned) * T));
    CK(cudaMemcpy(d_off, off.data(), sizeof(unsigned) * (n + 1), cudaMemcpyHostToDevice));
    r->ks->ref_terms(mp, d_refs, d_y, (int)n, d_off, d_tk, d_th, d_tv, d_tseg, r->log2B, 0);
    CK(cudaDeviceSynchronize());
    std::vector<unsigned char> tk(kb * T);
    std::vector<double> th(T), tv(T);
    std::vector<unsigned> tseg(T);
    CK(cudaMemcpy(tk.data(), d_tk, kb * T, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(th.data(), d_th, sizeof(double) * T, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(tv.data(), d_tv, sizeof(double) * T, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(tseg.data(), d_tseg, sizeof(unsigned) * T, cudaMemcpyDeviceToHost));
    // group the terms by segment (stable), so each merge block finds its own
    std::vector<size_t> order(T);
    for (size_t i = 0; i < T; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return tseg[a] < tseg[b]; });
    std::vector<unsigned char> sk(kb * T);
    std::vector<double> sh(T), sv(T);
    std::vector<unsigned> soff(B + 1, 0);
    for (size_t i = 0; i < T; ++i) {
        memcpy(sk.data() + i * kb, tk.data() + order[i] * kb, kb);
        sh[i] = th[order[i]];
        sv[i] = tv[order[i]];
        soff[tseg[order[i]] + 1]++;
    }
    for (unsigned b = 0; b < B; ++b) soff[b + 1] += soff[b];
    if (T > r->ref_cap) {
        // the reference arrays are rarely resized; they live as long as the run
        r->ref_keys = dev_alloc(r, kb * T);
        r->ref_h = (double*)dev_alloc(r, sizeof(double) * T);
        r->ref_v = (double*)dev_alloc(r, sizeof(double) * T);
        if (!r->ref_keys || !r->ref_h || !r->ref_v) return FQ_ERR_NOMEM;
        r->ref_cap = T;
        r->gen++;
    }
    CK(cudaMemcpy(r->ref_keys, sk.data(), kb * T, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(r->ref_h, sh.data(), sizeof(double) * T, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(r->ref_v, sv.data(), sizeof(double) * T, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(r->ref_off, soff.data(), sizeof(unsigned) * (B + 1), cudaMemcpyHostToDevice));
    std::vector<unsigned> bk;
    for (unsigned b = 0; b < B; ++b)
        if (soff[b + 1] > soff[b]) bk.push_back(b);
    if (bk.size() > 64 * 1024) return FQ_ERR_INVALID;
    CK(cudaMemcpy(r->ref_bkt, bk.data(), sizeof(unsigned) * bk.size(), cudaMemcpyHostToDevice));
    r->n_ref_bkt = (unsigned)bk.size();
    r->gen++;
    CK(sync_self(r));
    return FQ_OK;
}

extern "C" int fq_run_seed_default(fq_run* r, double weight) {
    if (!r || !(weight != 0.0) || !std::isfinite(weight)) return FQ_ERR_INVALID;
    fq_key s;
    int rc = fq_ham_starting_address(&r->ham, &s);
    if (rc) return rc;
    double diag = 0;
    size_t m = 0;
    rc = ham_column_dev(&r->ham, r->amp, s, &diag, nullptr, nullptr, 0, &m, r->stream);
    if (rc) return rc;
    rc = fq_run_seed(r, &s, &weight, 1, diag, 0);
    if (rc) return rc;
    return fq_run_set_reference(r, &s, &weight, 1);
}

static int set_state_field(fq_run* r, size_t offset, double v) {
    if (!r || !std::isfinite(v)) return FQ_ERR_INVALID;
    // ordered with queued steps: the value is staged in the run's pinned slot,
    // which is reused only after the copy has completed
    CK(cudaEventSynchronize(r->staged));
    *r->pinned = v;
    CK(cudaMemcpyAsync((char*)r->st + offset, r->pinned, sizeof(double), cudaMemcpyHostToDevice,
                       r->stream));
    CK(cudaEventRecord(r->staged, r->stream));
    if (r->smax >= 0 && (offset == offsetof(RunState, shift) || offset == offsetof(RunState, dt))) {
        launch_factors(r->d_self, 1, r->stream);
        CK(cudaGetLastError());
    }
    return FQ_OK;
}

extern "C" int fq_run_set_dt(fq_run* r, double dt) {
    if (!(dt > 0)) return FQ_ERR_INVALID;
    return set_state_field(r, offsetof(RunState, dt), dt);
}
extern "C" int fq_run_set_shift(fq_run* r, double s) { return set_state_field(r, offsetof(RunState, shift), s); }
extern "C" int fq_run_set_target(fq_run* r, double t) {
    if (!(t > 0)) return FQ_ERR_INVALID;
    return set_state_field(r, offsetof(RunState, target), t);
}

// ---------------------------------------------------------------------------
// batches: descriptor table, graphs, stepping

static void launch_overlaps(fq_batch* b, cudaStream_t s) {
    if (b->ov_on) b->ks->overlap(b->d_desc, b->d_ov, b->ov_grid, b->ov_wpb, b->ov_table, s);
}

// Gram-Schmidt of the spectral states, between the merge and the shift update
static void launch_gs(fq_batch* b, cudaStream_t s) {
    for (int k = 1; k < b->gs_K; ++k)
        b->ks->gs(b->d_desc, b->d_gs, k, b->gs_grid, b->gs_wpb, b->gs_table, s);
}

static void enqueue_steps(fq_batch* b, int n, cudaStream_t s) {
    const int nr = (int)b->runs.size();
    for (int i = 0; i < n; ++i) {
        b->ks->spawn(b->cfg, b->d_desc, b->d_seg_run, b->G, s);
        b->ks->merge(b->cfg, b->d_desc, b->d_seg_run, b->G, s);
        launch_gs(b, s);
        launch_shift(b->d_desc, nr, s);
        launch_overlaps(b, s);
    }
}

static void batch_release(fq_batch* b) {
    if (b->g1) cudaGraphExecDestroy(b->g1);
    if (b->g16) cudaGraphExecDestroy(b->g16);
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_seg_run) cudaFree(b->d_seg_run);
    b->g1 = b->g16 = nullptr;
    b->d_desc = nullptr;
    b->d_seg_run = nullptr;
}

static void overlaps_free(fq_batch* b) {
    if (b->d_ov) cudaFree(b->d_ov);
    if (b->ov_part) cudaFree(b->ov_part);
    if (b->ov_ring) cudaFree(b->ov_ring);
    if (b->ov_head) cudaFree(b->ov_head);
    b->d_ov = nullptr;
    b->ov_part = b->ov_ring = nullptr;
    b->ov_head = nullptr;
    b->ov_part_n = 0;
    b->ov_on = false;
}

// blocks per SM for a join kernel with `smem` bytes of tables per block:
// as many as the SM's 228 KB hold (1 KB of it reserved per block), at most 8
static unsigned long long join_blocks_per_sm(size_t smem) {
    return std::max<size_t>(1, std::min<size_t>(8, (228u * 1024u) / (smem + 1024u)));
}

// the overlap launch for the batch's current sizes: one table per warp with
// more slots than the largest segment capacity, so an insert always finds
// one (a segment's typical fill keeps the load near a third)
static int overlaps_build(fq_batch* b) {
    if (!b->ov_on) return FQ_OK;
    unsigned cv = 0;
    for (fq_run* r : b->runs) cv = std::max(cv, r->Cv);
    const unsigned T = std::max(64u, next_pow2(cv + 1ull));
    const size_t slot = b->ks->overlap_slot_bytes;
    int wpb = 4;
    while (wpb > 1 && (size_t)wpb * T * slot > 200u * 1024u) wpb >>= 1;
    if ((size_t)T * slot > 200u * 1024u) return FQ_ERR_INVALID;  // segments too large
    const size_t smem = (size_t)wpb * T * slot;
    CK(b->ks->prepare_overlap(smem));
    const int R = (int)b->runs.size(), P = R * (R - 1) / 2;
    const unsigned long long items = (unsigned long long)P * b->runs[0]->B;
    b->ov_wpb = wpb;
    b->ov_grid = (int)std::max<unsigned long long>(
        1, std::min<unsigned long long>((unsigned long long)num_sms() * join_blocks_per_sm(smem),
                                        (items + wpb - 1) / wpb));
    b->ov_table = T;
    const size_t need = (size_t)b->ov_grid * wpb * P * (1 + b->ov_nq);
    if (need > b->ov_part_n) {
        if (b->ov_part) cudaFree(b->ov_part);
        b->ov_part = nullptr;
        b->ov_part_n = 0;
        CK(cudaMalloc((void**)&b->ov_part, sizeof(double) * need));
        b->ov_part_n = need;
    }
    OverlapDesc od;
    memset(&od, 0, sizeof od);
    od.R = R;
    od.P = P;
    od.nq = b->ov_nq;
    for (int k = 0; k < b->ov_nq; ++k) od.d[k] = b->ov_d[k];
    int p = 0;
    for (int a = 0; a < R; ++a)
        for (int c = a + 1; c < R; ++c, ++p) {
            od.pa[p] = a;
            od.pb[p] = c;
        }
    od.B = b->runs[0]->B;
    od.table = T;
    od.part = b->ov_part;
    od.ring = b->ov_ring;
    od.head = b->ov_head;
    od.cap = b->ov_cap;
    CK(cudaMemcpy(b->d_ov, &od, sizeof od, cudaMemcpyHostToDevice));
    return FQ_OK;
}

static void gs_free(fq_batch* b) {
    if (b->d_gs) cudaFree(b->d_gs);
    if (b->gs_part) cudaFree(b->gs_part);
    if (b->gs_alpha) cudaFree(b->gs_alpha);
    b->d_gs = nullptr;
    b->gs_part = b->gs_alpha = nullptr;
    b->gs_part_n = 0;
    b->gs_K = 0;
}

// the Gram-Schmidt launches for the batch's current sizes: one table per
// warp with more slots than K segments' capacities (an insert always finds one)
static int gs_build(fq_batch* b) {
    if (b->gs_K < 2) return FQ_OK;
    unsigned cv = 0;
    for (int k = 0; k < b->gs_K; ++k) cv = std::max(cv, b->runs[k]->Cv);
    const unsigned T = std::max(64u, next_pow2((unsigned long long)b->gs_K * cv + 1ull));
    const size_t slot = b->ks->gs_slot_bytes;
    if ((size_t)T * slot > 200u * 1024u) return FQ_ERR_INVALID;  // segments too large
    int wpb = 4;
    while (wpb > 1 && (size_t)wpb * T * slot > 200u * 1024u) wpb >>= 1;
    CK(b->ks->prepare_gs((size_t)wpb * T * slot));
    const unsigned B = b->runs[0]->B;
    b->gs_wpb = wpb;
    b->gs_grid = (int)std::max<unsigned long long>(
        1, std::min<unsigned long long>(
               (unsigned long long)num_sms() * join_blocks_per_sm((size_t)wpb * T * slot),
               ((unsigned long long)B + wpb - 1) / wpb));
    b->gs_table = T;
    const size_t need = (size_t)b->gs_grid * wpb * 2 * FQ_MAX_SPECTRAL;
    if (need > b->gs_part_n) {
        if (b->gs_part) cudaFree(b->gs_part);
        b->gs_part = nullptr;
        b->gs_part_n = 0;
        CK(cudaMalloc((void**)&b->gs_part, sizeof(double) * need));
        b->gs_part_n = need;
    }
    GsDesc g;
    memset(&g, 0, sizeof g);
    g.K = b->gs_K;
    g.B = B;
    g.table = T;
    g.part = b->gs_part;
    g.alpha = b->gs_alpha;
    CK(cudaMemcpy(b->d_gs, &g, sizeof g, cudaMemcpyHostToDevice));
    return FQ_OK;
}

static void batch_free(fq_batch* b) {
    if (!b) return;
    batch_release(b);
    overlaps_free(b);
    gs_free(b);
    fq_run* r0 = b->runs[0];
    if (b->scratch) {
        if (r0->has_alloc) r0->alloc.free(r0->alloc.ctx, b->scratch, b->scratch_bytes, (void*)r0->stream);
        else cudaFreeAsync(b->scratch, r0->stream);
    }
    if (b->sort_scratch) {
        if (r0->has_alloc)
            r0->alloc.free(r0->alloc.ctx, b->sort_scratch, b->sort_scratch_bytes, (void*)r0->stream);
        else cudaFreeAsync(b->sort_scratch, r0->stream);
    }
    delete b;
}

static int capture(fq_batch* b, int n, cudaGraphExec_t* out) {
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        enqueue_steps(b, n, cs);
        e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return cuda_err(e);
}

// the launch shapes a batch may use: the default first, then the ones the
// autotuner tries
// the annihilation arms a batch may use: the runs' choice, both for AUTO
static std::vector<int> batch_arms(const fq_batch* b) {
    const int a = b->runs[0]->prm.annihilation;
    if (a == FQ_ANN_HASH) return {FQ_ANN_HASH_ARM};
    if (a == FQ_ANN_SORT) return {FQ_ANN_SORT_ARM};
    return {FQ_ANN_HASH_ARM, FQ_ANN_SORT_ARM};
}

static std::vector<LaunchCfg> batch_shapes(fq_batch* b, unsigned slots) {
    std::vector<LaunchCfg> v;
    const size_t limit = 200u * 1024u;
    const std::vector<int> arms = batch_arms(b);
    v.push_back(make_cfg(b->ks, 0, 1, 0, slots, b->G, arms[0]));
    for (int ann : arms)
        for (int sv = 0; sv < kKernelVariants; ++sv)
            for (int waves : {1, 2})
                for (int mv = 0; mv < kKernelVariants; ++mv)
                    for (unsigned sl : {slots / 2, slots, slots * 2}) {
                        if (sl < 64 || b->ks->merge_smem(ann, variant_wpb(mv), sl) > limit) continue;
                        v.push_back(make_cfg(b->ks, sv, waves, mv, sl, b->G, ann));
                    }
    return v;
}

static int batch_build(fq_batch* b) {
    const size_t nr = b->runs.size();
    b->gens.resize(nr);
    for (size_t i = 0; i < nr; ++i) b->gens[i] = b->runs[i]->gen;
    std::vector<RunDesc> desc(nr);
    std::vector<unsigned> seg_run;
    unsigned base = 0, slots = 0, ss = 0, se = 0;
    for (size_t i = 0; i < nr; ++i) {
        fq_run* r = b->runs[i];
        fill_desc(r, desc[i], base);
        for (unsigned s = 0; s < r->B; ++s) seg_run.push_back((unsigned)i);
        base += r->B;
        slots = std::max(slots, r->slots);
        ss = std::max(ss, r->scratch_slots);
        se = std::max(se, r->sort_elems);
    }
    b->G = base;
    CK(cudaMalloc((void**)&b->d_desc, sizeof(RunDesc) * nr));
    CK(cudaMalloc((void**)&b->d_seg_run, sizeof(unsigned) * base));
    CK(cudaMemcpy(b->d_desc, desc.data(), sizeof(RunDesc) * nr, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_seg_run, seg_run.data(), sizeof(unsigned) * base, cudaMemcpyHostToDevice));
    CK(b->ks->prepare(200u * 1024u));
    b->shapes = batch_shapes(b, slots);
    // scratch tables for the largest number of merge warps of any shape
    size_t warps = 0;
    for (const LaunchCfg& c : b->shapes) warps = std::max(warps, (size_t)c.merge_grid * c.merge_wpb);
    const size_t bytes = warps * ss * b->ks->slot_bytes;
    if (!b->scratch || b->scratch_bytes < bytes || b->scratch_ss != ss) {
        fq_run* r0 = b->runs[0];
        if (b->scratch) {
            CK(cudaStreamSynchronize(b->stream));
            if (r0->has_alloc) r0->alloc.free(r0->alloc.ctx, b->scratch, b->scratch_bytes, (void*)r0->stream);
            else cudaFreeAsync(b->scratch, r0->stream);
            b->scratch = nullptr;
        }
        void* p = nullptr;
        if (r0->has_alloc) p = r0->alloc.alloc(r0->alloc.ctx, bytes, (void*)r0->stream);
        else if (cudaMallocAsync(&p, bytes, r0->stream) != cudaSuccess) p = nullptr;
        if (!p) return FQ_ERR_NOMEM;
        b->scratch = (unsigned char*)p;
        b->scratch_bytes = bytes;
        // each merge warp's table is laid out for `ss` slots: cleared for it
        b->scratch_ss = ss;
        b->ks->scratch_init(b->scratch, ss, (unsigned)warps, r0->stream);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(r0->stream));
    }
    // sort workspaces in device memory, when a sort shape may run (no
    // clearing needed: each use writes before it reads)
    bool sort_shapes = false;
    for (const LaunchCfg& c : b->shapes) sort_shapes |= c.ann == FQ_ANN_SORT_ARM;
    const size_t sbytes = sort_shapes ? warps * b->ks->sort_ws_bytes(se) : 0;
    if (sbytes > b->sort_scratch_bytes) {
        fq_run* r0 = b->runs[0];
        if (b->sort_scratch) {
            CK(cudaStreamSynchronize(b->stream));
            if (r0->has_alloc)
                r0->alloc.free(r0->alloc.ctx, b->sort_scratch, b->sort_scratch_bytes, (void*)r0->stream);
            else cudaFreeAsync(b->sort_scratch, r0->stream);
            b->sort_scratch = nullptr;
            b->sort_scratch_bytes = 0;
        }
        void* p = nullptr;
        if (r0->has_alloc) p = r0->alloc.alloc(r0->alloc.ctx, sbytes, (void*)r0->stream);
        else if (cudaMallocAsync(&p, sbytes, r0->stream) != cudaSuccess) p = nullptr;
        if (!p) return FQ_ERR_NOMEM;
        b->sort_scratch = (unsigned char*)p;
        b->sort_scratch_bytes = sbytes;
    }
    for (LaunchCfg& c : b->shapes) {
        c.scratch = b->scratch;
        c.scratch_slots = ss;
        c.sort_scratch = b->sort_scratch;
        c.sort_elems = se;
    }
    {
        int rc = overlaps_build(b);
        if (!rc) rc = gs_build(b);
        if (rc) return rc;
    }
    b->cfg = b->shapes[0];
    if (nr == 1 && b->runs[0]->has_tuned) {
        const LaunchCfg& t = b->runs[0]->tuned;
        for (const LaunchCfg& c : b->shapes)
            if (c.spawn_var == t.spawn_var && c.spawn_grid == t.spawn_grid &&
                c.merge_var == t.merge_var && c.merge_grid == t.merge_grid && c.slots == t.slots &&
                c.ann == t.ann)
                b->cfg = c;
    }
    int rc = capture(b, 1, &b->g1);
    if (!rc) rc = capture(b, 16, &b->g16);
    return rc;
}

static int batch_new(fq_run* const* runs, int n, bool owned, fq_batch** out) {
    fq_batch* b = new (std::nothrow) fq_batch();
    if (!b) return FQ_ERR_NOMEM;
    b->runs.assign(runs, runs + n);
    b->ks = runs[0]->ks;
    b->stream = runs[0]->stream;
    b->owned_by_run = owned;
    b->d_desc = nullptr;
    b->d_seg_run = nullptr;
    b->g1 = b->g16 = nullptr;
    b->scratch = nullptr;
    b->scratch_bytes = 0;
    b->scratch_ss = 0;
    int rc = batch_build(b);
    if (rc) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return FQ_OK;
}

static int batch_refresh(fq_batch* b) {
    bool stale = false;
    for (size_t i = 0; i < b->runs.size(); ++i) stale |= b->gens[i] != b->runs[i]->gen;
    if (!stale) return FQ_OK;
    CK(cudaStreamSynchronize(b->stream));
    batch_release(b);
    return batch_build(b);
}

static int batch_launch(fq_batch* b, int64_t n) {
    if (n < 0) return FQ_ERR_INVALID;
    int rc = batch_refresh(b);
    if (rc) return rc;
    while (n >= 16) {
        CK(cudaGraphLaunch(b->g16, b->stream));
        n -= 16;
    }
    while (n-- > 0) CK(cudaGraphLaunch(b->g1, b->stream));
    return FQ_OK;
}

static int single_batch(fq_run* r) {
    if (r->single) return FQ_OK;
    fq_run* one[1] = {r};
    return batch_new(one, 1, true, &r->single);
}

extern "C" int fq_run_step(fq_run* r, int64_t n) {
    if (!r || n < 0) return FQ_ERR_INVALID;
    if (!r->seeded) return FQ_ERR_INVALID;
    if (r->no_spawn_buf) return FQ_ERR_NOMEM;
    int rc = single_batch(r);
    if (rc) return rc;
    return batch_launch(r->single, n);
}

// read the device error; on error roll the run back to its last completed
// step (the current buffer and state are untouched by a failed step)
static int run_check(fq_run* r) {
    if (r->no_spawn_buf) return FQ_ERR_NOMEM;
    CK(cudaStreamSynchronize(r->stream));
    unsigned err = 0;
    CK(cudaMemcpy(&err, &r->st->err, sizeof err, cudaMemcpyDeviceToHost));
    if (!err) return FQ_OK;
    r->last_err_bits = err;
    RunState s;
    CK(cudaMemcpy(&s, r->st, sizeof s, cudaMemcpyDeviceToHost));
    s.err = 0;
    s.n_exact = s.n_inexact = s.n_spawns = 0;
    s.norm_lo = s.norm_hi = 0;
    s.norm_fp = 0.0;
    s.len_acc = 0;
    CK(cudaMemcpy(r->st, &s, sizeof s, cudaMemcpyHostToDevice));
    CK(cudaMemset(r->sfill, 0, sizeof(unsigned) * r->B));
    if (err & FQ_DERR_EMPTY) return FQ_ERR_EMPTY;
    if (err & FQ_DERR_TIMEOUT) return FQ_ERR_TIMEOUT;
    return FQ_ERR_CAPACITY;
}

extern "C" int fq_run_error_bits(const fq_run* r, unsigned* bits) {
    if (!r || !bits) return FQ_ERR_INVALID;
    *bits = r->last_err_bits;
    return FQ_OK;
}

extern "C" int fq_run_sync(fq_run* r) {
    if (!r) return FQ_ERR_INVALID;
    return run_check(r);
}

extern "C" int fq_run_stats(fq_run* r, fq_stats* out) {
    if (!r || !out) return FQ_ERR_INVALID;
    const int rc = run_check(r);
    RunState s;
    CK(cudaMemcpy(&s, r->st, sizeof s, cudaMemcpyDeviceToHost));
    out->step = s.step;
    out->len = s.len;
    out->exact_steps = s.last_exact;
    out->inexact_steps = s.last_inexact;
    out->n_spawns = s.last_spawns;
    out->shift = s.shift;
    out->norm = s.norm;
    out->hproj = s.last_hproj;
    out->vproj = s.last_vproj;
    return rc;
}

extern "C" int fq_run_history(fq_run* r, fq_stats* out, size_t cap, size_t* n) {
    if (!r || !n || (cap && !out)) return FQ_ERR_INVALID;
    *n = 0;
    const int rc = run_check(r);
    unsigned long long head = 0;
    CK(cudaMemcpy(&head, &r->st->hist_head, sizeof head, cudaMemcpyDeviceToHost));
    unsigned long long first = r->hist_read;
    if (head > FQ_HIST_CAP && first < head - FQ_HIST_CAP) first = head - FQ_HIST_CAP;
    size_t cnt = (size_t)std::min<unsigned long long>(head - first, cap);
    static_assert(sizeof(StatsRow) == sizeof(fq_stats), "row layout");
    for (size_t i = 0; i < cnt;) {
        const unsigned pos = (unsigned)((first + i) % FQ_HIST_CAP);
        const size_t chunk = std::min<size_t>(cnt - i, FQ_HIST_CAP - pos);
        CK(cudaMemcpy(out + i, r->hist + pos, sizeof(StatsRow) * chunk, cudaMemcpyDeviceToHost));
        i += chunk;
    }
    r->hist_read = first + cnt;
    *n = cnt;
    return rc;
}

// gather the segmented arrays (counts `cnt_dev`, capacity `cap`) to the host
static int gather(fq_run* r, const void* keys, const void* vals, unsigned cap, const unsigned* cnt_dev,
                  bool spawns, std::vector<fq_key>& ok, std::vector<double>& ov) {
    const unsigned B = r->B;
    std::vector<unsigned> cnt(B), off(B + 1, 0);
    CK(cudaMemcpy(cnt.data(), cnt_dev, sizeof(unsigned) * B, cudaMemcpyDeviceToHost));
    for (unsigned b = 0; b < B; ++b) off[b + 1] = off[b] + std::min(cnt[b], cap);
    const size_t T = off[B];
    const size_t kb = r->ks->key_bytes;
    ok.assign(T, fq_key{0, 0});
    ov.assign(T, 0.0);
    if (!T) return FQ_OK;
    unsigned* d_off = nullptr;
    void* d_k = nullptr;
    double* d_v = nullptr;
    CallBufs bufs;  // released on every return
    CK(bufs.get(&d_off, sizeof(unsigned) * (B + 1)));
    CK(bufs.get(&d_k, kb * T));
    CK(bufs.get(&d_v, sizeof(double) * T));
    CK(cudaMemcpy(d_off, off.data(), sizeof(unsigned) * (B + 1), cudaMemcpyHostToDevice));
    if (spawns) r->ks->gather_spawns(keys, vals, cap, r->Cp, cnt_dev, d_off, B, d_k, d_v, 0);
    else r->ks->gather_vec(keys, vals, cap, cnt_dev, d_off, B, d_k, d_v, nullptr, 0);
    CK(cudaDeviceSynchronize());
    std::vector<unsigned char> kbuf(kb * T);
    CK(cudaMemcpy(kbuf.data(), d_k, kb * T, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(ov.data(), d_v, sizeof(double) * T, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < T; ++i) memcpy(&ok[i], kbuf.data() + i * kb, kb);
    return FQ_OK;
}

extern "C" int fq_run_export(fq_run* r, fq_key* keys, double* amps, size_t cap, size_t* n) {
    if (!r || !n || (cap && (!keys || !amps))) return FQ_ERR_INVALID;
    *n = 0;
    const int rc = run_check(r);
    int cur = 0;
    CK(cudaMemcpy(&cur, &r->st->cur, sizeof cur, cudaMemcpyDeviceToHost));
    std::vector<fq_key> k;
    std::vector<double> v;
    int g = gather(r, r->vkeys[cur], r->vamps[cur], r->Cv, r->vcount[cur], false, k, v);
    if (g) return g;
    std::vector<size_t> order(k.size());
    for (size_t i = 0; i < k.size(); ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return key_less(k[a], k[b]); });
    const size_t w = std::min(cap, k.size());
    for (size_t i = 0; i < w; ++i) {
        keys[i] = k[order[i]];
        amps[i] = v[order[i]];
    }
    *n = k.size();
    return rc;
}

extern "C" int fq_run_reserve(fq_run* r, size_t capacity_vec, size_t capacity_spawn) {
    if (!r) return FQ_ERR_INVALID;
    int rc = run_check(r);
    if (rc) return rc;
    const double k = r->det ? (double)max_offdiag(r->ham.mp) : 8.0;
    unsigned Cv, Cs;
    segment_caps((double)capacity_vec, (double)capacity_spawn, r->B, k, Cv, Cs);
    Cv = std::max(Cv, r->Cv);
    Cs = std::max(Cs, r->Cs);
    if (Cv == r->Cv && Cs == r->Cs) return FQ_OK;
    const size_t kb = r->ks->key_bytes, ab = r->ks->amp_bytes, sb = r->ks->spawn_bytes;
    int cur = 0;
    CK(cudaMemcpy(&cur, &r->st->cur, sizeof cur, cudaMemcpyDeviceToHost));
    if (Cv > r->Cv) {
        void* nk[2] = {dev_alloc(r, kb * (size_t)r->B * Cv), dev_alloc(r, kb * (size_t)r->B * Cv)};
        void* na[2] = {dev_alloc(r, ab * (size_t)r->B * Cv), dev_alloc(r, ab * (size_t)r->B * Cv)};
        if (!nk[0] || !nk[1] || !na[0] || !na[1]) {
            for (int i = 0; i < 2; ++i) {
                if (nk[i]) dev_free(r, nk[i]);
                if (na[i]) dev_free(r, na[i]);
            }
            return FQ_ERR_NOMEM;
        }
        r->ks->restride(r->vkeys[cur], r->vamps[cur], r->Cv, r->vcount[cur], r->B, nk[cur], na[cur],
                        Cv, r->stream);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(r->stream));
        for (int i = 0; i < 2; ++i) {
            dev_free(r, r->vkeys[i]);
            dev_free(r, r->vamps[i]);
            r->vkeys[i] = nk[i];
            r->vamps[i] = na[i];
        }
        r->Cv = Cv;
    }
    int out = FQ_OK;
    if (Cs > r->Cs) {
        // the spawn buffers hold nothing between steps: the old ones are
        // released first, so growing them needs no room for both
        auto spawn_alloc = [&](unsigned cs, void** k, void** v) {
            *k = dev_alloc(r, r->ks->spawn_key_stride * (size_t)r->B * cs);
            *v = dev_alloc(r, std::max<size_t>(16, r->ks->spawn_val_stride * (size_t)r->B * cs));
            if (*k && *v) return true;
            if (*k) dev_free(r, *k);
            if (*v) dev_free(r, *v);
            *k = *v = nullptr;
            return false;
        };
        dev_free(r, r->skeys);
        dev_free(r, r->samps);
        void *nk, *nv;
        if (spawn_alloc(Cs, &nk, &nv)) {
            r->Cs = Cs;
        } else {
            out = FQ_ERR_NOMEM;  // back to the old size, which fitted before
            if (!spawn_alloc(r->Cs, &nk, &nv)) r->no_spawn_buf = true;
        }
        r->skeys = nk;
        r->samps = nv;
    }
    table_sizes(r);
    r->gen++;
    CK(sync_self(r));
    return out;
}

extern "C" int fq_run_capacity(const fq_run* r, size_t* capacity_vec, size_t* capacity_spawn) {
    if (!r) return FQ_ERR_INVALID;
    if (capacity_vec) *capacity_vec = (size_t)r->B * r->Cv;
    if (capacity_spawn) *capacity_spawn = (size_t)r->B * r->Cs;
    return FQ_OK;
}

extern "C" int fq_run_set_tables(fq_run* r, unsigned slots, unsigned scratch_slots) {
    if (!r) return FQ_ERR_INVALID;
    auto pow2 = [](unsigned x) { return x && !(x & (x - 1)); };
    if (slots && (!pow2(slots) || slots < 64 || 8ull * slots * r->ks->slot_bytes > 200u * 1024u))
        return FQ_ERR_INVALID;
    if (scratch_slots && (!pow2(scratch_slots) || scratch_slots < 64 || scratch_slots > (1u << 26)))
        return FQ_ERR_INVALID;
    int rc = run_check(r);
    if (rc) return rc;
    r->forced_slots = slots;
    r->forced_scratch = scratch_slots;
    table_sizes(r);
    r->has_tuned = false;  // a tuned shape was timed with the old tables
    r->gen++;
    return FQ_OK;
}

extern "C" int fq_run_set_spawn_split(fq_run* r, unsigned primary) {
    if (!r) return FQ_ERR_INVALID;
    int rc = run_check(r);
    if (rc) return rc;
    if (primary % 32u || primary > r->Cs) return FQ_ERR_INVALID;
    r->Cp = primary;
    r->gen++;
    CK(sync_self(r));
    return FQ_OK;
}

extern "C" int fq_run_merge_paths(fq_run* r, uint64_t* onchip, uint64_t* scratch) {
    if (!r || !onchip || !scratch) return FQ_ERR_INVALID;
    const int rc = run_check(r);
    RunState s;
    CK(cudaMemcpy(&s, r->st, sizeof s, cudaMemcpyDeviceToHost));
    *onchip = s.merged_onchip;
    *scratch = s.merged_scratch;
    return rc;
}

extern "C" int fq_run_lookup(fq_run* r, const fq_key* keys, size_t n, double* amps) {
    if (!r || (n && (!keys || !amps))) return FQ_ERR_INVALID;
    int rc = run_check(r);
    if (rc) return rc;
    if (!n) return FQ_OK;
    const size_t kb = r->ks->key_bytes;
    std::vector<unsigned char> kbuf;
    pack_keys(keys, n, kb, kbuf);
    void* d_k = nullptr;
    double* d_a = nullptr;
    CallBufs bufs;  // released on every return
    CK(bufs.get(&d_k, kb * n));
    CK(bufs.get(&d_a, sizeof(double) * n));
    cudaError_t e = cudaMemcpy(d_k, kbuf.data(), kb * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        r->ks->lookup(r->d_self, d_k, n, d_a, r->stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e == cudaSuccess) e = cudaMemcpy(amps, d_a, sizeof(double) * n, cudaMemcpyDeviceToHost);
    return cuda_err(e);
}

extern "C" int fq_run_sample(fq_run* r, uint64_t seed, size_t want, fq_key* keys, double* amps,
                             size_t cap, size_t* n) {
    if (!r || !n || (cap && (!keys || !amps))) return FQ_ERR_INVALID;
    *n = 0;
    int rc = run_check(r);
    if (rc) return rc;
    int cur = 0;
    CK(cudaMemcpy(&cur, &r->st->cur, sizeof cur, cudaMemcpyDeviceToHost));
    const unsigned B = r->B;
    std::vector<unsigned> cnt(B);
    CK(cudaMemcpy(cnt.data(), r->vcount[cur], sizeof(unsigned) * B, cudaMemcpyDeviceToHost));
    // whole segments in a seeded random order until `want` entries
    std::vector<unsigned> order(B);
    for (unsigned b = 0; b < B; ++b) order[b] = b;
    uint64_t x = seed;
    for (unsigned b = B; b > 1; --b) {
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        std::swap(order[b - 1], order[(unsigned)(z % b)]);
    }
    std::vector<unsigned> segs, off(1, 0);
    size_t tot = 0;
    for (unsigned b = 0; b < B && tot < want; ++b) {
        const unsigned s = order[b];
        if (!cnt[s]) continue;
        segs.push_back(s);
        tot += std::min(cnt[s], r->Cv);
        off.push_back((unsigned)tot);
    }
    const size_t kb = r->ks->key_bytes;
    if (tot) {
        unsigned *d_off = nullptr, *d_segs = nullptr;
        void* d_k = nullptr;
        double* d_v = nullptr;
        CallBufs bufs;  // released on every return
        CK(bufs.get(&d_off, sizeof(unsigned) * off.size()));
        CK(bufs.get(&d_segs, sizeof(unsigned) * segs.size()));
        CK(bufs.get(&d_k, kb * tot));
        CK(bufs.get(&d_v, sizeof(double) * tot));
        CK(cudaMemcpy(d_off, off.data(), sizeof(unsigned) * off.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_segs, segs.data(), sizeof(unsigned) * segs.size(), cudaMemcpyHostToDevice));
        r->ks->gather_vec(r->vkeys[cur], r->vamps[cur], r->Cv, r->vcount[cur], d_off,
                          (unsigned)segs.size(), d_k, d_v, d_segs, 0);
        CK(cudaDeviceSynchronize());
        std::vector<unsigned char> kbuf(kb * tot);
        std::vector<double> v(tot);
        CK(cudaMemcpy(kbuf.data(), d_k, kb * tot, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(v.data(), d_v, sizeof(double) * tot, cudaMemcpyDeviceToHost));
        const size_t w = std::min(cap, tot);
        for (size_t i = 0; i < w; ++i) {
            fq_key k = {0, 0};
            memcpy(&k, kbuf.data() + i * kb, kb);
            keys[i] = k;
            amps[i] = v[i];
        }
    }
    *n = tot;
    return FQ_OK;
}

extern "C" int fq_run_spawns(fq_run* r, fq_key* dest, double* val, size_t cap, size_t* n) {
    if (!r || !n || (cap && (!dest || !val))) return FQ_ERR_INVALID;
    *n = 0;
    int rc = run_check(r);
    if (rc) return rc;
    if (!r->seeded) return FQ_ERR_INVALID;
    rc = single_batch(r);
    if (!rc) rc = batch_refresh(r->single);
    if (rc) return rc;
    fq_batch* b = r->single;
    b->ks->spawn(b->cfg, b->d_desc, b->d_seg_run, b->G, r->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(r->stream));
    unsigned err = 0;
    CK(cudaMemcpy(&err, &r->st->err, sizeof err, cudaMemcpyDeviceToHost));
    std::vector<fq_key> k;
    std::vector<double> v;
    if (!err) {
        int g = gather(r, r->skeys, r->samps, r->Cs, r->sfill, true, k, v);
        if (g) return g;
    }
    rc = run_check(r);  // clears the error flag if one was set
    CK(cudaMemset(r->sfill, 0, sizeof(unsigned) * r->B));
    RunState s;
    CK(cudaMemcpy(&s, r->st, sizeof s, cudaMemcpyDeviceToHost));
    s.n_exact = s.n_inexact = s.n_spawns = 0;
    CK(cudaMemcpy(r->st, &s, sizeof s, cudaMemcpyHostToDevice));
    if (err) return FQ_ERR_CAPACITY;
    const size_t w = std::min(cap, k.size());
    for (size_t i = 0; i < w; ++i) {
        dest[i] = k[i];
        val[i] = v[i];
    }
    *n = k.size();
    return rc;
}

// ---------------------------------------------------------------------------
// autotuning: time each launch shape over real steps, keep the fastest

static int autotune(fq_batch* b, int steps) {
    if (steps < 1) return FQ_ERR_INVALID;
    // the spawn and merge kernels are independent launches: their shapes are
    // timed separately (CUDA events around each kernel) and chosen separately
    std::vector<LaunchCfg> sc, mc;
    for (const LaunchCfg& c : b->shapes) {
        bool seen_s = false, seen_m = false;
        for (const LaunchCfg& x : sc) seen_s |= x.spawn_var == c.spawn_var && x.spawn_grid == c.spawn_grid;
        for (const LaunchCfg& x : mc)
            seen_m |= x.merge_var == c.merge_var && x.merge_grid == c.merge_grid &&
                      x.slots == c.slots && x.ann == c.ann;
        if (!seen_s) sc.push_back(c);
        if (!seen_m) mc.push_back(c);
    }
    const size_t nc = std::max(sc.size(), mc.size());
    const size_t total = nc * (size_t)steps;
    std::vector<cudaEvent_t> ev(3 * total, nullptr);
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < ev.size() && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
    const int nr = (int)b->runs.size();
    auto shape = [&](size_t i) {
        LaunchCfg c = mc[i % mc.size()];
        const LaunchCfg& s2 = sc[i % sc.size()];
        c.spawn_var = s2.spawn_var;
        c.spawn_wpb = s2.spawn_wpb;
        c.spawn_grid = s2.spawn_grid;
        return c;
    };
    if (e == cudaSuccess) enqueue_steps(b, 1, b->stream);  // warm
    for (size_t t = 0; t < total && e == cudaSuccess; ++t) {
        const LaunchCfg c = shape(t % nc);
        cudaEventRecord(ev[3 * t], b->stream);
        b->ks->spawn(c, b->d_desc, b->d_seg_run, b->G, b->stream);
        cudaEventRecord(ev[3 * t + 1], b->stream);
        b->ks->merge(c, b->d_desc, b->d_seg_run, b->G, b->stream);
        e = cudaEventRecord(ev[3 * t + 2], b->stream);
        launch_gs(b, b->stream);
        launch_shift(b->d_desc, nr, b->stream);
        launch_overlaps(b, b->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    std::vector<double> ts(sc.size(), 0.0), tm(mc.size(), 0.0);
    std::vector<int> ns(sc.size(), 0), nm(mc.size(), 0);
    for (size_t t = 0; t < total && e == cudaSuccess; ++t) {
        float a = 0, m = 0;
        e = cudaEventElapsedTime(&a, ev[3 * t], ev[3 * t + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&m, ev[3 * t + 1], ev[3 * t + 2]);
        const size_t i = t % nc;
        ts[i % sc.size()] += a;
        ns[i % sc.size()] += 1;
        tm[i % mc.size()] += m;
        nm[i % mc.size()] += 1;
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return cuda_err(e);
    size_t bs = 0, bm = 0;
    for (size_t i = 1; i < sc.size(); ++i)
        if (ts[i] / ns[i] < ts[bs] / ns[bs]) bs = i;
    for (size_t i = 1; i < mc.size(); ++i)
        if (tm[i] / nm[i] < tm[bm] / nm[bm]) bm = i;
    b->arm_ms[0] = b->arm_ms[1] = 0.0f;
    for (size_t i = 0; i < mc.size(); ++i) {
        float& a = b->arm_ms[mc[i].ann == FQ_ANN_SORT_ARM ? 1 : 0];
        const float t = (float)(tm[i] / nm[i]);
        if (a == 0.0f || t < a) a = t;
    }
    LaunchCfg best = mc[bm];
    best.spawn_var = sc[bs].spawn_var;
    best.spawn_wpb = sc[bs].spawn_wpb;
    best.spawn_grid = sc[bs].spawn_grid;
    b->cfg = best;
    if (b->g1) cudaGraphExecDestroy(b->g1);
    if (b->g16) cudaGraphExecDestroy(b->g16);
    b->g1 = b->g16 = nullptr;
    int rc = capture(b, 1, &b->g1);
    if (!rc) rc = capture(b, 16, &b->g16);
    return rc;
}

extern "C" int fq_run_autotune(fq_run* r, int steps) {
    if (!r || !r->seeded) return FQ_ERR_INVALID;
    int rc = single_batch(r);
    if (!rc) rc = batch_refresh(r->single);
    if (rc) return rc;
    rc = autotune(r->single, steps);
    if (rc) return rc;
    r->tuned = r->single->cfg;
    r->has_tuned = true;
    return run_check(r);
}

extern "C" int fq_run_arm_times(fq_run* r, float* hash_ms, float* sort_ms) {
    if (!r || !hash_ms || !sort_ms) return FQ_ERR_INVALID;
    *hash_ms = r->single ? r->single->arm_ms[0] : 0.0f;
    *sort_ms = r->single ? r->single->arm_ms[1] : 0.0f;
    return FQ_OK;
}

extern "C" int fq_run_shape(fq_run* r, int* shape) {
    if (!r || !shape || !r->seeded) return FQ_ERR_INVALID;
    int rc = single_batch(r);
    if (!rc) rc = batch_refresh(r->single);
    if (rc) return rc;
    const LaunchCfg& c = r->single->cfg;
    shape[0] = c.spawn_wpb;
    shape[1] = c.spawn_grid;
    shape[2] = c.merge_wpb;
    shape[3] = c.merge_grid;
    shape[4] = (int)c.slots;
    shape[5] = (int)(c.ann == FQ_ANN_SORT_ARM ? c.sort_elems : c.scratch_slots);
    shape[6] = c.ann == FQ_ANN_SORT_ARM ? FQ_ANN_SORT : FQ_ANN_HASH;
    return FQ_OK;
}

extern "C" int fq_run_profile(fq_run* r, int n, float* ms) {
    if (!r || !ms || n < 1 || n > 4096 || !r->seeded) return FQ_ERR_INVALID;
    int rc = single_batch(r);
    if (!rc) rc = batch_refresh(r->single);
    if (rc) return rc;
    fq_batch* b = r->single;
    std::vector<cudaEvent_t> ev((size_t)4 * n, nullptr);
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < ev.size() && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        cudaEventRecord(ev[4 * i], r->stream);
        b->ks->spawn(b->cfg, b->d_desc, b->d_seg_run, b->G, r->stream);
        cudaEventRecord(ev[4 * i + 1], r->stream);
        b->ks->merge(b->cfg, b->d_desc, b->d_seg_run, b->G, r->stream);
        cudaEventRecord(ev[4 * i + 2], r->stream);
        launch_shift(b->d_desc, 1, r->stream);
        e = cudaEventRecord(ev[4 * i + 3], r->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    double acc[3] = {0, 0, 0};
    for (int i = 0; i < n && e == cudaSuccess; ++i)
        for (int k = 0; k < 3; ++k) {
            float t = 0;
            e = cudaEventElapsedTime(&t, ev[4 * i + k], ev[4 * i + k + 1]);
            acc[k] += t;
        }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return cuda_err(e);
    for (int k = 0; k < 3; ++k) ms[k] = (float)(acc[k] / n);
    return run_check(r);
}

// ---------------------------------------------------------------------------
// C ABI: batches

extern "C" int fq_batch_create(fq_batch** out, fq_run* const* runs, int B) {
    if (!out || !runs || B < 1) return FQ_ERR_INVALID;
    *out = nullptr;
    for (int i = 0; i < B; ++i) {
        if (!runs[i] || !runs[i]->seeded) return FQ_ERR_INVALID;
        if (runs[i]->ks != runs[0]->ks || runs[i]->stream != runs[0]->stream ||
            runs[i]->prm.annihilation != runs[0]->prm.annihilation)
            return FQ_ERR_INVALID;
        for (int j = 0; j < i; ++j)
            if (runs[j] == runs[i]) return FQ_ERR_INVALID;
    }
    return batch_new(runs, B, false, out);
}

extern "C" void fq_batch_destroy(fq_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
}

extern "C" int fq_batch_step(fq_batch* b, int64_t n) {
    if (!b) return FQ_ERR_INVALID;
    for (fq_run* r : b->runs)
        if (r->no_spawn_buf) return FQ_ERR_NOMEM;
    return batch_launch(b, n);
}

extern "C" int fq_batch_sync(fq_batch* b) {
    if (!b) return FQ_ERR_INVALID;
    int rc = FQ_OK;
    for (fq_run* r : b->runs) {
        int e = run_check(r);
        if (e && !rc) rc = e;
    }
    return rc;
}

extern "C" int fq_batch_set_overlaps(fq_batch* b, const int* g2_d, int n_g2) {
    if (!b || n_g2 < 0 || n_g2 > FQ_MAX_G2 || (n_g2 && !g2_d)) return FQ_ERR_INVALID;
    const int R = (int)b->runs.size();
    if (R < 2 || R > FQ_MAX_REPLICAS) return FQ_ERR_INVALID;
    const fq_run* r0 = b->runs[0];
    for (const fq_run* r : b->runs)
        if (r->B != r0->B || r->ham.mp.kind != r0->ham.mp.kind || r->ham.mp.M != r0->ham.mp.M ||
            r->ham.mp.N != r0->ham.mp.N || r->ham.mp.Lx != r0->ham.mp.Lx)
            return FQ_ERR_INVALID;
    if (n_g2 && r0->ham.mp.kind != FQ_BH_REAL_1D) return FQ_ERR_INVALID;
    for (int k = 0; k < n_g2; ++k)
        if (g2_d[k] < 0 || g2_d[k] >= r0->ham.mp.M) return FQ_ERR_INVALID;
    CK(cudaStreamSynchronize(b->stream));
    overlaps_free(b);
    const int P = R * (R - 1) / 2;
    const size_t width = 1 + (size_t)P * (1 + n_g2);
    b->ov_cap = (unsigned)std::min<size_t>(65536, std::max<size_t>(1024, (8u << 20) / width));
    CK(cudaMalloc((void**)&b->d_ov, sizeof(OverlapDesc)));
    CK(cudaMalloc((void**)&b->ov_ring, sizeof(double) * width * b->ov_cap));
    CK(cudaMalloc((void**)&b->ov_head, sizeof(unsigned long long)));
    CK(cudaMemset(b->ov_head, 0, sizeof(unsigned long long)));
    b->ov_read = 0;
    b->ov_nq = n_g2;
    for (int k = 0; k < n_g2; ++k) b->ov_d[k] = g2_d[k];
    b->ov_on = true;
    // rebuild the descriptors and graphs with the overlap launch in each step
    batch_release(b);
    int rc = batch_build(b);
    if (rc) overlaps_free(b);
    return rc;
}

extern "C" int fq_batch_set_spectral(fq_batch* b, int K) {
    if (!b || K < 0 || K > FQ_MAX_SPECTRAL || K > (int)b->runs.size()) return FQ_ERR_INVALID;
    if (K >= 2) {
        const fq_run* r0 = b->runs[0];
        for (int k = 0; k < K; ++k) {
            const fq_run* r = b->runs[k];
            if (r->B != r0->B || r->amp == FQ_AMP_INT || r->ham.mp.M != r0->ham.mp.M ||
                r->ham.mp.N != r0->ham.mp.N || r->ham.mp.kind != r0->ham.mp.kind ||
                r->ham.mp.Lx != r0->ham.mp.Lx)
                return FQ_ERR_INVALID;
        }
    }
    CK(cudaStreamSynchronize(b->stream));
    gs_free(b);
    if (K >= 2) {
        CK(cudaMalloc((void**)&b->d_gs, sizeof(GsDesc)));
        CK(cudaMalloc((void**)&b->gs_alpha, sizeof(double) * FQ_MAX_SPECTRAL));
        b->gs_K = K;
    }
    batch_release(b);
    int rc = batch_build(b);
    if (rc) {
        gs_free(b);
        batch_release(b);
        const int rc2 = batch_build(b);
        (void)rc2;
    }
    return rc;
}

extern "C" int fq_batch_overlaps(fq_batch* b, double* rows, size_t cap, size_t* n, int* width) {
    if (!b || !n || (cap && !rows)) return FQ_ERR_INVALID;
    *n = 0;
    if (!b->ov_on) return FQ_ERR_INVALID;
    const int R = (int)b->runs.size(), P = R * (R - 1) / 2;
    const size_t w = 1 + (size_t)P * (1 + b->ov_nq);
    if (width) *width = (int)w;
    CK(cudaStreamSynchronize(b->stream));
    unsigned long long head = 0;
    CK(cudaMemcpy(&head, b->ov_head, sizeof head, cudaMemcpyDeviceToHost));
    unsigned long long first = b->ov_read;
    if (head > b->ov_cap && first < head - b->ov_cap) first = head - b->ov_cap;
    const size_t cnt = (size_t)std::min<unsigned long long>(head - first, cap);
    for (size_t i = 0; i < cnt;) {
        const unsigned pos = (unsigned)((first + i) % b->ov_cap);
        const size_t chunk = std::min<size_t>(cnt - i, b->ov_cap - pos);
        CK(cudaMemcpy(rows + i * w, b->ov_ring + (size_t)pos * w, sizeof(double) * w * chunk,
                      cudaMemcpyDeviceToHost));
        i += chunk;
    }
    b->ov_read = first + cnt;
    *n = cnt;
    return FQ_OK;
}

extern "C" int fq_batch_autotune(fq_batch* b, int steps) {
    if (!b) return FQ_ERR_INVALID;
    int rc = autotune(b, steps);
    if (rc) return rc;
    return fq_batch_sync(b);
}


// ---------------------------------------------------------------------------
// fq_ham_column_noalloc: the column of H without allocating anything.
//
// fq_ham_column allocates its device buffers with cudaMalloc and releases
// them with cudaFree on every call.  Two kinds of caller cannot afford that:
// a caller whose device memory is all taken (a large run plus a caching
// allocator that keeps its freed blocks can leave cudaMalloc nothing), and a
// caller with steps queued on other streams, because cudaFree waits for the
// whole device and so stalls them.  This variant evaluates the column into
// one fixed device array that exists from the moment the library is loaded.
//
// Limits and rules of use:
//  - The array holds the matrix-element tables for N <= 128 and at most
//    FQ_COLUMN_NOALLOC_MAX (16384) off-diagonal entries; a longer column is
//    rejected with FQ_ERR_CAPACITY (its length is still reported).
//  - Nothing in the array has to start at zero: every call writes the
//    tables, the diagonal, the count and the entries before reading them.
//  - The array is shared by every caller on a device.  Calls that overlap in
//    time (from several host threads) race on it; callers must serialise.
//  - Work runs on a stream the library creates once per device with
//    cudaStreamNonBlocking, so it neither waits for nor holds up the legacy
//    default stream or any other stream of the caller.
//  - The first call on a device looks up the array's device address
//    (cudaGetSymbolAddress, which may load the module) and creates that
//    stream: make that first call outside any stream capture.

namespace {
constexpr unsigned kNaMax = FQ_COLUMN_NOALLOC_MAX;  // column entries
constexpr size_t kNaTab = 129u * 130u + 1u;                   // (N+1)(N+2)+1, N <= 128
constexpr size_t na_round(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kNaOffSq = 0;
constexpr size_t kNaOffHop = kNaOffSq + na_round(sizeof(double) * kNaTab);
constexpr size_t kNaOffHop32 = kNaOffHop + na_round(sizeof(double) * kNaTab);
constexpr size_t kNaOffHead = kNaOffHop32 + na_round(sizeof(float) * kNaTab);  // diag, m
constexpr size_t kNaOffDest = kNaOffHead + 256;
constexpr size_t kNaOffVal = kNaOffDest + na_round(sizeof(fq_key) * kNaMax);
constexpr size_t kNaBytes = kNaOffVal + na_round(sizeof(double) * kNaMax);  // 729,600 B
constexpr int kNaDevices = 64;

struct NaDevice {
    unsigned char* base;  // device address of g_na_scratch on this device
    cudaStream_t stream;  // non-blocking stream of this device's calls
};
NaDevice g_na[kNaDevices];
std::atomic<bool> g_na_ready[kNaDevices];
std::mutex g_na_setup;
}  // namespace

static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

// the column at `key`, with the tables k_tables wrote into the fixed array by
// an earlier launch on the same stream; written in fq_key layout (one thread)
template <class K, int KIND>
__global__ void k_column_fixed(ModelParams mp, K key, unsigned char* base) {
    if (threadIdx.x || blockIdx.x) return;
    mp.sqrt_tab = (const double*)(base + kNaOffSq);
    mp.hop_tab = (const double*)(base + kNaOffHop);
    mp.hop32_tab = (const float*)(base + kNaOffHop32);
    typedef Model<KIND> MD;
    typename MD::Col col;
    const unsigned m = MD::num_offdiag(mp, key, col);
    *(double*)(base + kNaOffHead) = MD::diagonal(mp, key);
    *(unsigned*)(base + kNaOffHead + 8) = m;
    unsigned long long* dest = (unsigned long long*)(base + kNaOffDest);
    double* val = (double*)(base + kNaOffVal);
    for (unsigned k = 0; k < m && k < kNaMax; ++k) {
        const K d = MD::offdiag(mp, key, col, k, val[k]);
        dest[2 * k] = (unsigned long long)d;
        dest[2 * k + 1] = sizeof(K) > 8 ? (unsigned long long)(d >> 32 >> 32) : 0ull;
    }
}

template <class K>
static void launch_column_fixed(int kind, const ModelParams& mp, K key, unsigned char* base,
                                cudaStream_t s) {
    if (kind == FQ_BH_REAL_1D) k_column_fixed<K, FQ_KIND_REAL_1D><<<1, 32, 0, s>>>(mp, key, base);
    else if (kind == FQ_BH_REAL_2D) k_column_fixed<K, FQ_KIND_REAL_2D><<<1, 32, 0, s>>>(mp, key, base);
    else k_column_fixed<K, FQ_KIND_MOM_1D><<<1, 32, 0, s>>>(mp, key, base);
}

// set-up of the current device, once: the array's address and the stream
static int na_device(NaDevice** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_err(e);
    if (dev < 0 || dev >= kNaDevices) return FQ_ERR_INVALID;
    if (!g_na_ready[dev].load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> lock(g_na_setup);
        if (!g_na_ready[dev].load(std::memory_order_relaxed)) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_na_scratch);
            if (e != cudaSuccess) return cuda_err(e);
            cudaStream_t s = nullptr;
            e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_err(e);
            g_na[dev].base = (unsigned char*)p;
            g_na[dev].stream = s;
            g_na_ready[dev].store(true, std::memory_order_release);
        }
    }
    *out = &g_na[dev];
    return FQ_OK;
}

extern "C" int fq_ham_column_noalloc(const fq_ham* h, fq_key key, double* diag, fq_key* dest,
                                     double* val, size_t cap, size_t* m_out) {
    if (!h || !key_valid(h, key)) return FQ_ERR_INVALID;
    ModelParams mp = h->mp;
    mp.kmax = (mp.N + 1) * (mp.N + 2);
    if ((size_t)mp.kmax + 1 > kNaTab) return FQ_ERR_INVALID;
    NaDevice* nd = nullptr;
    int rc = na_device(&nd);
    if (rc) return rc;
    unsigned char* base = nd->base;
    const cudaStream_t s = nd->stream;
    // the tables first, in their own launch: the column kernel reads them
    // through the read-only cache, which is only valid for data that no
    // thread of the same launch writes
    k_tables<<<(unsigned)((mp.kmax + 256) / 256), 256, 0, s>>>(
        mp.t, mp.kmax, (double*)(base + kNaOffSq), (double*)(base + kNaOffHop),
        (float*)(base + kNaOffHop32));
    if (h->kw == 1) launch_column_fixed<uint64_t>(mp.kind, mp, (uint64_t)key.lo, base, s);
    else launch_column_fixed<u128>(mp.kind, mp, ((u128)key.hi << 64) | (u128)key.lo, base, s);
    cudaError_t e = cudaGetLastError();
    unsigned char head[16];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(head, base + kNaOffHead, sizeof head, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(e);
    double d;
    unsigned m;
    memcpy(&d, head, sizeof d);
    memcpy(&m, head + 8, sizeof m);
    if (m_out) *m_out = m;
    if (m > kNaMax) return FQ_ERR_CAPACITY;  // longer than the fixed array holds
    if (diag) *diag = d;
    const size_t nw = std::min<size_t>(m, cap);
    if (nw && dest)
        e = cudaMemcpyAsync(dest, base + kNaOffDest, sizeof(fq_key) * nw, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && nw && val)
        e = cudaMemcpyAsync(val, base + kNaOffVal, sizeof(double) * nw, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_err(e);
}
static_assert(kNaBytes == 729600, "fixed column array size as documented in fciqmc.h");
