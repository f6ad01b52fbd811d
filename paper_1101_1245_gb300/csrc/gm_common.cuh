// Internal definitions of the gpumcd CUDA library (sm_103a): device data
// layouts, table geometry, the Philox generator and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gpumcd.h"

namespace gm {

// ---------------------------------------------------------------------------
// Constants
// ---------------------------------------------------------------------------
constexpr double kMC2 = 0.51099895000;       // MeV
constexpr double kRE = 2.8179403262e-13;     // cm
constexpr double kALPHA = 1.0 / 137.035999084;
constexpr double kNA = 6.02214076e23;
constexpr double kPI = 3.14159265358979323846;
constexpr float kMC2f = 0.51099895f;
constexpr float kTWO_PIf = 6.283185307179586f;
constexpr double kQ = 1.0 / 67108864.0;      // energy quantum, 2^-26 MeV
constexpr float kQf = 1.4901161193847656e-08f;
constexpr float kInvQf = 67108864.0f;
constexpr float kRhoQ = 5.9604644775390625e-08f;  // density quantum, 2^-24 g/cm^3
constexpr double kMeVPerGramToGy = 1.602176634e-10;

constexpr int G = 512;      // points of each energy grid
constexpr int G_MS = 512;   // points of the multiple-scattering ln(a) table
constexpr int NMAT = GPUMCD_MAX_MATERIALS;
// the transport kernel masks a voxel's material id with NMAT - 1
static_assert((NMAT & (NMAT - 1)) == 0, "NMAT must be a power of two");
// ...and a record's plan index with GPUMCD_MAX_PLANS_PER_RUN - 1
static_assert((GPUMCD_MAX_PLANS_PER_RUN & (GPUMCD_MAX_PLANS_PER_RUN - 1)) == 0, "plan table size");
constexpr double MS_G_MIN = 1e-8;  // paths below this many transport mean free paths: no deflection
constexpr double MS_G_MAX = 20.0;  // paths above: isotropic

// Table layout in floats (global memory; a CTA stages the part it needs into
// shared memory): the multiple-scattering table, the bremsstrahlung shape
// constants, then one block per material holding its photon tables
// [mu_tot, mu_C, mu_pe][G] (cm^2/g) and its electron tables
// [L, S_hard, S_brem, l1inv][G].  The loaded materials come first, so their
// blocks and everything before them are one contiguous range.
constexpr int TAB_MS = 0;                            // [G_MS] ln a over ln G1
constexpr int TAB_BREM = TAB_MS + G_MS;              // [mat][cA, c1] bremsstrahlung shape
constexpr int TAB_MAT = TAB_BREM + 4 * NMAT;         // first material block
constexpr int TAB_MAT_FLOATS = 7 * G;                // 3 photon + 4 electron tables
constexpr int TAB_FLOATS = TAB_MAT + NMAT * TAB_MAT_FLOATS;
constexpr int TAB_BYTES = TAB_FLOATS * 4;
__host__ __device__ constexpr int tab_ph(int m) { return TAB_MAT + m * TAB_MAT_FLOATS; }          // photon tables of m
__host__ __device__ constexpr int tab_el(int m) { return TAB_MAT + m * TAB_MAT_FLOATS + 3 * G; }  // electron tables of m
// bytes of the tables of materials 0 .. n-1 and what precedes them (what a CTA stages)
__host__ __device__ constexpr uint32_t tab_bytes(int n) { return 4u * (uint32_t)(TAB_MAT + n * TAB_MAT_FLOATS); }
static_assert(tab_bytes(1) % 16 == 0 && (4 * TAB_MAT_FLOATS) % 16 == 0, "bulk copies move multiples of 16 bytes");

constexpr int MAJ_FLOATS = 2 * G;  // per phantom: photon majorant | electron majorant

// Grid geometry: a table index is x = (ln E - ln E0) / d, evaluated as
// x = log2(E) * a + b with E in energy quanta (bq) or in MeV (bm).
struct Grid {
    float ph_a, ph_bq;          // photon grid
    float el_a, el_bq, el_bm;   // electron grid
    float ms_a, ms_b;           // multiple-scattering grid, E -> G1
};

// Transport parameters in device form.
struct Phys {
    uint32_t p_cut_q, e_abs_q, two_mc2_q;
    float t_c, k_c, estepe, nudge;
    Grid grid;
};

// Particle types of the transport kernel's warps, stacks and queues.
enum { T_PH = 0, T_EL = 1, NT = 2 };

// A particle record: 48 bytes, three 16-byte words.
//   a = (x, y, z, ux), b = (uy, uz, E bits, history bits), c = (lineage lo, lineage hi, draw, plan)
struct __align__(16) Rec {
    float4 a;
    float4 b;
    uint4 c;
};

// An electron whose step ended on a hard-event candidate (§II.B.3, the
// electron Woodcock test), parked until its warp runs a converged hard pass:
// the particle after its step, the majorant Sigma_hat of the step and the
// step's voxel (where the candidate lies, and whose cross-section the
// majorant bounds).  64 bytes.
struct __align__(16) HardRec {
    Rec r;
    float sig_hat;
    uint32_t idx;
    uint32_t pad[2];
};
constexpr unsigned HARD_CAP = 64;  // per warp: a pass starts at 32, one step adds at most 32

// One plan inside a launch (copied to shared memory by the transport kernel).
struct __align__(16) PlanDev {
    const uint32_t *vox;           // packed voxel words
    unsigned long long *tally;     // [n_batches][nvox] energy in quanta
    unsigned long long *ledger;    // [incident, escaped, rest, spare]
    const float *maj;              // [photon G | electron G] majorants, 1/cm
    const float *spec;             // spectrum: [n_spec+1 cdf | n_spec+1 edges], or null
    int32_t nx, ny, nz, n_spec;
    float dx, dy, dz, inv_dx;
    float inv_dy, inv_dz, X, Y;
    float Z, cx, cy, field;
    uint32_t nvox, bmask, key_lo, key_hi;
    int32_t src_type, beam;
    uint32_t e_src_q, n_phsp;     // n_phsp: phase-space records (spec holds them)
    unsigned long long hist_base;  // first history of this launch
    const uint32_t *order;         // e_group: the launch's histories in claim order (offsets from hist_base)
    uint32_t e_group, n_sorted;    // e_group: a source grouped by energy; n_sorted: histories `order` covers
};
static_assert(sizeof(PlanDev) == 160, "the plan table in shared memory keeps its size");

// Queue of particle records in global memory (overflow between launches).
// For an input queue `cursor` counts records claimed; for an output queue it
// counts records written.
struct Queue {
    Rec *rec;
    unsigned long long *cursor;
    uint32_t capacity;
};

struct TransportArgs {
    const float *tables;
    Phys phys;
    const PlanDev *plans;
    int32_t n_plans;
    uint32_t n_prim_plans[2];          // plans per source type in prim_plan[]
    uint8_t prim_plan[2][GPUMCD_MAX_PLANS_PER_RUN];       // plan index, by source type
    unsigned long long prim_off[2][GPUMCD_MAX_PLANS_PER_RUN + 1];  // prefix of histories
    unsigned long long *prim_cursor;   // [2]
    Queue in[NT], out[NT];
    unsigned long long in_count[NT];   // records available in in[t]
    Rec *stacks;                       // [warp][type][stack_capacity]
    HardRec *hard;                     // [warp][HARD_CAP] parked hard-event candidates
    uint32_t stack_cap, switch_high, refill_low, chunk;
    uint32_t flags;
    uint32_t refill_period;            // 1: refill every pass; N: every N-th pass or when empty
    uint32_t phsp;                     // a plan of the launch has a phase-space source
    uint32_t tab_bytes;                // bytes of tables staged into shared memory (the loaded materials')
    unsigned long long *counters;      // run counters (see CNT_*)
    int32_t *error;                    // device status word
};

enum {
    CNT_PH_EVENTS = 0, CNT_PH_REAL, CNT_COMPTON, CNT_PHOTO, CNT_PAIR,
    CNT_E_STEPS, CNT_HARD_REAL, CNT_HARD_FICT, CNT_MOLLER, CNT_BREM,
    CNT_PHOTONS, CNT_ELECTRONS, CNT_OVERFLOW, CNT_SPILLS, CNT_SAMPLER_CAP,
    // profile counters (GPUMCD_LAUNCH_PROFILE), per particle type (photon,
    // electron): SM clock cycles of the warps' event passes, the passes, and
    // the active lanes summed over them; then cycles in refills and the number
    // of type switches
    CNT_PROF_CYC, CNT_PROF_ITER = CNT_PROF_CYC + NT, CNT_PROF_LANES = CNT_PROF_ITER + NT,
    CNT_PROF_REFILL_CYC = CNT_PROF_LANES + NT, CNT_PROF_SWITCHES,
    // converged passes over parked hard-event candidates (always counted)
    CNT_HARD_PASSES, CNT_N
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the two 32x32->64
// multiplies with the Weyl-sequence key schedule.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
        const uint64_t p0 = 0xD2511F53ull * c.x, p1 = 0xCD9E8D57ull * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Uniform in (0, 1] from the top 24 bits of a word.
__device__ __forceinline__ float u01(uint32_t w) {
    return __uint2float_rn((w >> 8) + 1u) * 5.9604644775390625e-08f;
}

// Launch helpers implemented in the .cu files (host side).
struct LaunchCfg {
    int grid, block;
    size_t smem;
};

}  // namespace gm
