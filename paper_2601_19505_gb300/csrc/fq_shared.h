// fq_shared.h -- plain structs shared by the host code (fq_api.cu) and the
// kernels: model parameters, per-run device state, the per-run descriptor
// the batched kernels read, and launch shapes.
#pragma once

#include <cstddef>
#include <cstdint>

#define FQ_KIND_REAL_1D 1
#define FQ_KIND_REAL_2D 2
#define FQ_KIND_MOM_1D 3

// amplitude representation
#define FQ_AMP_INT 0  // int64 amplitudes, int32 spawns, exact integer sums
#define FQ_AMP_F64 1  // double amplitudes and spawns, FP64 sums
#define FQ_AMP_F32 2  // float amplitudes, spawns and sums

// device-side error bits (RunState::err)
#define FQ_DERR_SPAWN_CAP 1u
#define FQ_DERR_VEC_CAP 2u
#define FQ_DERR_TABLE 4u
#define FQ_DERR_EMPTY 8u
#define FQ_DERR_TIMEOUT 16u
#define FQ_DERR_RANGE 32u  // an amplitude beyond the exact-norm range

// annihilation arms of the merge kernel
#define FQ_ANN_HASH_ARM 0
#define FQ_ANN_SORT_ARM 1

#define FQ_MAX_MOM_MODES 64
#define FQ_HIST_CAP 65536u

namespace fq {

struct ModelParams {
    int kind, M, N, Lx, Ly, nbits;
    double t, u;
    double g;                        // u / (2M), momentum space
    int kmax;                        // largest index of the sqrt/hop tables
    const double* sqrt_tab;          // sqrt((double)k), k <= kmax (device)
    const double* hop_tab;           // -(t * sqrt((double)k)), k <= kmax (device)
    const float* hop32_tab;          // (float) of hop_tab
    unsigned char nbr[4][128];       // real space: neighbour of site s in direction d
    // kept last: the spawn kernel copies the members before it for real-space
    // models and the whole struct for momentum space
    double eps[FQ_MAX_MOM_MODES];    // momentum-space single-particle energies
};

// One row of the time series; layout identical to fq_stats in fciqmc.h.
struct StatsRow {
    long long step, len, exact_steps, inexact_steps, n_spawns;
    double shift, norm, hproj, vproj;
};

// Mutable per-run state in device memory.  The kernels of step n read
// shift/step/cur/dt; the shift kernel writes the next values and clears
// the accumulators of the step.
struct RunState {
    double shift;      // S^(n)
    double norm;       // N^(n) = ||c^(n)||_1
    double dt, target, zeta, xi;
    long long step;    // n
    long long len;     // occupied entries of c^(n)
    int cur;           // vector buffer holding c^(n)
    unsigned err;      // FQ_DERR_* bits; a set bit freezes the run
    unsigned long long n_exact, n_inexact, n_spawns;  // step in flight
    unsigned long long hist_head;                     // rows written
    double last_hproj, last_vproj;
    long long last_exact, last_inexact, last_spawns;
    // norm of the step in flight: exact sum in units of 2^norm_q (128-bit),
    // or a plain FP64 sum in the deterministic limit
    unsigned long long norm_lo, norm_hi;
    double norm_fp;
    unsigned long long len_acc;
    // buckets the merge kernel summed in the on-chip table and in the global
    // scratch table, since seeding
    unsigned long long merged_onchip, merged_scratch;
};

// Everything a kernel needs to process one run's segments.  Lives in a
// device array, one entry per run of a batch.
struct RunDesc {
    ModelParams mp;
    int amp;            // FQ_AMP_*
    int mode_det;       // deterministic limit: every column exact, no compression
    double theta, t_rel;
    float theta32;      // (float)theta
    int theta_pow2;     // theta = 2^theta_exp: compression decided in integers
    int theta_exp;
    int early;          // early compression (Sec. 7.1): each spawn and diagonal term alone
    int norm_q;         // exact norm unit 2^norm_q
    int trel_one;       // t_rel == 1
    unsigned key_x, key_y;   // Philox key
    int log2B;
    unsigned B, seg_base, Cv, Cs;
    unsigned Cp;             // spawn slots per bucket in the dense primary region (<= Cs)
    void* vkeys[2];
    void* vamps[2];
    unsigned* vcount[2];
    void* skeys;
    void* samps;
    unsigned* sfill;
    RunState* st;
    StatsRow* hist;
    int mmax;                 // largest m of the coefficient tables (real space)
    double* coef64;           // (-dt) ((double)m / (double)n), index m * (mmax + 1) + n
    float* coef32;            // the same in FP32 arithmetic
    int smax;                 // largest sum n(n-1) (real space)
    double* fac64;            // 1 + dt (S - H_ii) per s = sum n(n-1), this step
    float* del32;             // (float)(dt (S - H_ii)) per s, this step
    const void* ref_keys;     // reference terms sorted by segment
    const double* ref_h;      // y_r H_{r,j}
    const double* ref_v;      // y_r on the reference address itself, else 0
    const unsigned* ref_off;  // B + 1 offsets into the reference terms
    const unsigned* ref_bkt;  // segments holding reference terms, ascending
    unsigned n_ref_bkt;
    double* part_h;           // per-segment projected-energy partial sums
    double* part_v;
};

// Replica overlaps of a batch (Sec. 4.3): for every pair (A, B) of its runs,
// c_A^T c_B and c_A^T G2(d_k) c_B (Eq. g2) after each step.  The runs share
// one segment map (equal B), so segment b of A and of B hold the same
// addresses' entries.
#define FQ_MAX_REPLICAS 8
#define FQ_MAX_G2 16
struct OverlapDesc {
    int R, P, nq;                  // runs, pairs, G2 distances
    int d[FQ_MAX_G2];
    int pa[FQ_MAX_REPLICAS * (FQ_MAX_REPLICAS - 1) / 2];
    int pb[FQ_MAX_REPLICAS * (FQ_MAX_REPLICAS - 1) / 2];
    unsigned B;                    // segments per run
    unsigned table;                // slots of a warp's table (power of 2)
    double* part;                  // per warp: P x (1 + nq) partial sums
    double* ring;                  // rows of width 1 + P (1 + nq)
    unsigned long long* head;      // rows written
    unsigned cap;                  // rows the ring holds
};

// Excited states (Sec. 2.2): runs 0..K-1 of a batch are step-synchronised
// spectral states; after every step's merge, run k >= 1 is orthogonalised to
// runs 0..k-1 (Gram-Schmidt) on the new vectors, segment by segment.
#define FQ_MAX_SPECTRAL 8
struct GsDesc {
    int K;                  // spectral states
    unsigned B;             // segments per run
    unsigned table;         // slots of a warp's table (power of 2)
    double* part;           // per warp: 2 FQ_MAX_SPECTRAL partial dot products
    double* alpha;          // FQ_MAX_SPECTRAL coefficients of the run being orthogonalised
};

struct LaunchCfg {
    int ann;              // annihilation arm of the merge kernel (FQ_ANN_*_ARM)
    int spawn_var;        // compiled variant of the spawn kernel (warps, register cap)
    int spawn_wpb;        // its warps per block
    int spawn_grid;       // persistent spawn blocks
    int merge_var;        // compiled variant of the merge kernel
    int merge_wpb;        // its warps per block
    int merge_grid;       // persistent merge blocks
    unsigned slots;       // per merge warp: on-chip hash-table slots (power of 2), or
                          // sort-workspace elements
    unsigned scratch_slots;       // global scratch table slots per merge warp
    unsigned char* scratch;       // scratch tables, merge_grid * merge_wpb of them
    unsigned sort_elems;          // global sort workspace elements per merge warp
    unsigned char* sort_scratch;  // sort workspaces, merge_grid * merge_wpb of them
};

}  // namespace fq
