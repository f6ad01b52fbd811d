// Persistent coupled photon-electron transport kernel for sm_103a.
//
// One launch runs every particle it can reach to completion.  Each warp holds
// 32 particles of ONE type (photon or electron) in registers and advances all
// of them by one event per iteration: a Woodcock flight for photons (GPUMCD
// §II.A) or one condensed-history step for electrons (§II.B.3).  Lanes whose
// particle ended are refilled, in this order, from the warp's private stack of
// that type, from the global overflow queue of the previous launch, and from
// the primaries of the launch's plans (claimed in chunks).  Secondaries go to
// the warp's private stacks (the paper's per-type particle arrays, §II.C.2)
// and spill to a global overflow queue only when a stack fills; a warp
// switches type when its own lanes run dry or when the other stack is high
// (§II.C.3's "pool" of persistent threads, with warp-uniform particle type).
// An electron step that ends on a hard-event candidate parks the particle on
// a third per-warp stack; with 32 parked, the warp runs their Woodcock tests
// and Moller/bremsstrahlung events together (a converged hard pass) instead
// of one or two lanes at a time inside every step.
//
// Randomness is a counter-based Philox keyed by the plan seed with counter
// (draw, lineage lo, lineage hi, history), and energies are integers, so the
// tally is independent of how particles are scheduled.
//
// Divisions on the event path are written __fdividef (reciprocal, then
// multiply): every divisor there is a direction cosine, an energy, a cross
// section or a sampler constant, far inside the range (|y| < 2^126) for which
// that form is specified.  There it skips the range handling of the
// approximate division this file is compiled with (-prec-div=false), and the
// tallies and event counts of every workload compared were bit-identical with
// either form.
#include "gm_common.cuh"
#include "gm_host.h"

namespace gm {

// Relative margin of the per-voxel electron hard-event majorant (2^-14).
constexpr float kHardMajorantMargin = 1.00006103515625f;
constexpr unsigned FULL = 0xffffffffu;
constexpr int MAX_WARPS = 32;

struct WarpState {
    unsigned int stk[2];
    unsigned int hc;   // parked hard-event candidates (electrons)
    unsigned int pad;
    unsigned long long p_lo[2], p_hi[2];  // claimed primaries by type (type-local index)
    unsigned long long q_lo[2], q_hi[2];  // claimed overflow-queue records by type
};

struct Lane {
    float x, y, z, ux, uy, uz;
    uint32_t E, hist, lin_lo, lin_hi, draw, plan;
    bool act;
};

// Shared-memory context of a CTA.
struct Smem {
    const float *tab;
    PlanDev *plans;
    WarpState *ws;
    unsigned long long *cnt;     // [CNT_N]
    unsigned long long *ledger;  // [n_plans][3]: incident, escaped, rest
};

__device__ __forceinline__ float interp(const float *t, float x) {
    x = fminf(fmaxf(x, 0.0f), (float)(G - 1));
    const int i = min((int)x, G - 2);
    const float f = x - (float)i;
    const float a = t[i], b = t[i + 1];
    return fmaf(f, b - a, a);
}

__device__ __forceinline__ float interp_ldg(const float *t, float x) {
    x = fminf(fmaxf(x, 0.0f), (float)(G - 1));
    const int i = min((int)x, G - 2);
    const float f = x - (float)i;
    const float a = __ldg(t + i), b = __ldg(t + i + 1);
    return fmaf(f, b - a, a);
}

__device__ __forceinline__ float interp_ms(const float *t, float x) {
    x = fminf(fmaxf(x, 0.0f), (float)(G_MS - 1));
    const int i = min((int)x, G_MS - 2);
    const float f = x - (float)i;
    return fmaf(f, t[i + 1] - t[i], t[i]);
}

__device__ __forceinline__ uint4 draw4(Lane &p, const PlanDev &P) {
    const uint4 r = philox4x32_10(make_uint4(p.draw, p.lin_lo, p.lin_hi, p.hist),
                                  make_uint2(P.key_lo, P.key_hi));
    ++p.draw;
    return r;
}

// Lineage of the j-th particle a parent creates at draw index `draw`: a 64-bit
// finalizer of (parent lineage, draw, j), never equal to the primary's lineage 1.
__device__ __forceinline__ void child_lineage(const Lane &p, uint32_t j, uint32_t &lo, uint32_t &hi) {
    unsigned long long z = ((unsigned long long)p.lin_hi << 32) | p.lin_lo;
    z ^= ((unsigned long long)p.draw << 20) ^ ((unsigned long long)(j + 1) << 52) ^ 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 33)) * 0xFF51AFD7ED558CCDull;
    z = (z ^ (z >> 33)) * 0xC4CEB9FE1A85EC53ull;
    z ^= z >> 33;
    z |= 2ull;
    lo = (uint32_t)z;
    hi = (uint32_t)(z >> 32);
}

__device__ __forceinline__ bool inside(const PlanDev &P, float x, float y, float z) {
    return x >= 0.f && y >= 0.f && z >= 0.f && x < P.X && y < P.Y && z < P.Z;
}

__device__ __forceinline__ uint32_t voxel_index(const PlanDev &P, float x, float y, float z, int &ix,
                                                int &iy, int &iz) {
    ix = min((int)(x * P.inv_dx), P.nx - 1);
    iy = min((int)(y * P.inv_dy), P.ny - 1);
    iz = min((int)(z * P.inv_dz), P.nz - 1);
    return (uint32_t)ix + (uint32_t)P.nx * ((uint32_t)iy + (uint32_t)P.ny * (uint32_t)iz);
}

// Distance along the direction to the exit face of voxel (ix, iy, iz).
__device__ __forceinline__ float exit_distance(const PlanDev &P, const Lane &p, int ix, int iy, int iz) {
    float dv = 3.0e38f;
    if (p.ux != 0.f) dv = fminf(dv, __fdividef(((p.ux > 0.f ? (float)(ix + 1) : (float)ix) - p.x * P.inv_dx) * P.dx, p.ux));
    if (p.uy != 0.f) dv = fminf(dv, __fdividef(((p.uy > 0.f ? (float)(iy + 1) : (float)iy) - p.y * P.inv_dy) * P.dy, p.uy));
    if (p.uz != 0.f) dv = fminf(dv, __fdividef(((p.uz > 0.f ? (float)(iz + 1) : (float)iz) - p.z * P.inv_dz) * P.dz, p.uz));
    return dv;
}

// One float further along a direction cosine.  An electron step ends a nudge
// past the face it aims at, but at a grazing angle nudge x cosine can fall
// below FP32 resolution and the end point rounds back onto the face; indexed
// by position, a particle crossing in the negative direction would then stay
// in the voxel it is leaving, with a zero distance to its exit, and creep on
// in nudge-sized steps (seen in thin air, where nothing deflects it).  Moving
// every end coordinate one float along its direction takes it off the face.
__device__ __forceinline__ float float_along(float x, float u) {
    const int b = __float_as_int(x);
    return u > 0.f ? __int_as_float(b + 1) : (u < 0.f ? __int_as_float(b - 1) : x);
}

// Fire-and-forget 64-bit add into the tally (no value comes back).
__device__ __forceinline__ void red_add_u64(unsigned long long *addr, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(addr), "l"(v) : "memory");
}

__device__ __forceinline__ void deposit(const PlanDev &P, uint32_t hist, uint32_t idx, uint32_t e) {
    if (e == 0u) return;
    const uint32_t b = hist & P.bmask;  // batch = history mod W
    red_add_u64(P.tally + (size_t)b * P.nvox + idx, (unsigned long long)e);
}

// Deposit at a convergent point (all 32 lanes call it): lanes that hit the
// same tally word add their energies into one atomic.  Energies are < 2^31,
// so the group sum is formed exactly from two 32-bit reductions.
__device__ __forceinline__ void deposit_aggregated(const PlanDev &P, uint32_t hist, uint32_t idx,
                                                   uint32_t e) {
    const bool on = e != 0u;
    const unsigned mask = __ballot_sync(FULL, on);
    if (!on) return;
    const uint32_t b = hist & P.bmask;  // batch = history mod W
    unsigned long long *addr = P.tally + (size_t)b * P.nvox + idx;
    const unsigned peers = __match_any_sync(mask, (unsigned long long)addr);
    const unsigned lo = __reduce_add_sync(peers, e & 0xFFFFu);
    const unsigned hi = __reduce_add_sync(peers, e >> 16);
    if ((threadIdx.x & 31) == __ffs(peers) - 1)
        red_add_u64(addr, ((unsigned long long)hi << 16) + (unsigned long long)lo);
}

__device__ __forceinline__ void ledger_add(const Smem &S, uint32_t plan, int which, uint32_t e) {
    if (e) atomicAdd(&S.ledger[plan * 3 + which], (unsigned long long)e);
}

__device__ __forceinline__ void count(const Smem &S, int which) { atomicAdd(&S.cnt[which], 1ull); }

// Rotate (ux, uy, uz) by polar angle (cos c, sin s) and azimuth (cos cp, sin sp).
__device__ __forceinline__ void rotate(float &ux, float &uy, float &uz, float c, float s, float cp,
                                       float sp) {
    const float r2 = ux * ux + uy * uy;
    float nx, ny, nz;
    if (r2 > 1e-10f) {
        const float ir = rsqrtf(r2);
        const float r = r2 * ir;
        nx = ux * c + s * (ux * uz * cp - uy * sp) * ir;
        ny = uy * c + s * (uy * uz * cp + ux * sp) * ir;
        nz = uz * c - s * cp * r;
    } else {
        nx = s * cp;
        ny = s * sp;
        nz = uz >= 0.f ? c : -c;
    }
    const float n = rsqrtf(nx * nx + ny * ny + nz * nz);
    ux = nx * n;
    uy = ny * n;
    uz = nz * n;
}

// Push a new particle onto the warp's private stack of its type (headroom is
// guaranteed by the caller before each step).
__device__ __forceinline__ void push(const TransportArgs &A, const Smem &S, int gw, int w, int type,
                                     float x, float y, float z, float ux, float uy, float uz,
                                     uint32_t E, const Lane &parent, uint32_t j) {
    uint32_t lo, hi;
    child_lineage(parent, j, lo, hi);
    const unsigned slot = atomicAdd(&S.ws[w].stk[type], 1u);
    Rec *r = A.stacks + ((size_t)gw * 2 + type) * A.stack_cap + slot;
    r->a = make_float4(x, y, z, ux);
    r->b = make_float4(uy, uz, __uint_as_float(E), __uint_as_float(parent.hist));
    r->c = make_uint4(lo, hi, 0u, parent.plan);
    count(S, type == 0 ? CNT_PHOTONS : CNT_ELECTRONS);
}

// An electron set in motion by a photon: pushed for transport, or, in the
// photon-only mode (GPUMCD_LAUNCH_KERMA), deposited in the voxel `idx` of the
// photon's interaction.
template <bool KERMA>
__device__ __forceinline__ void emit_electron(const TransportArgs &A, const Smem &S, int gw, int w,
                                              const PlanDev &P, uint32_t idx, float vx, float vy, float vz,
                                              uint32_t E, const Lane &parent, uint32_t j) {
    if (KERMA)
        deposit(P, parent.hist, idx, E);
    else
        push(A, S, gw, w, 1, parent.x, parent.y, parent.z, vx, vy, vz, E, parent, j);
}

__device__ __forceinline__ void load_rec(Lane &p, const Rec &r) {
    const float4 a = r.a;
    const float4 b = r.b;
    const uint4 c = r.c;
    p.x = a.x; p.y = a.y; p.z = a.z; p.ux = a.w;
    p.uy = b.x; p.uz = b.y; p.E = __float_as_uint(b.z); p.hist = __float_as_uint(b.w);
    // the plan field indexes the CTA's 64-entry plan table, all of whose
    // entries are set at launch: masked, it stays in range by construction
    p.lin_lo = c.x; p.lin_hi = c.y; p.draw = c.z; p.plan = c.w & (GPUMCD_MAX_PLANS_PER_RUN - 1);
    p.act = true;
}

__device__ __forceinline__ Rec make_rec(const Lane &p) {
    Rec r;
    r.a = make_float4(p.x, p.y, p.z, p.ux);
    r.b = make_float4(p.uy, p.uz, __uint_as_float(p.E), __uint_as_float(p.hist));
    r.c = make_uint4(p.lin_lo, p.lin_hi, p.draw, p.plan);
    return r;
}

// ---------------------------------------------------------------------------
// Samplers (exact, FP32)
// ---------------------------------------------------------------------------

// Klein-Nishina (GPUMCD §II.A, Compton): composition-rejection on eps = k'/k
// in [1/(1+2k), 1]: choose 1/eps or eps by their integrals, accept with
// 1 - eps sin^2 / (1 + eps^2).  Returns eps, with cos theta in *c and the
// fourth word of the last draw in *w4.
constexpr int SAMPLER_CAP = 4096;  // proposals before a sampler gives up (counted, never expected)

__device__ float sample_kn(Lane &p, const PlanDev &P, float k, float *c, uint32_t *w4, unsigned *capped) {
    const float e0 = __fdividef(1.0f, 1.0f + 2.0f * k);
    const float a1 = __logf(1.0f + 2.0f * k);
    const float a2 = 0.5f * (1.0f - e0 * e0);
    for (int it = 0;; ++it) {
        const uint4 r = draw4(p, P);
        float eps;
        if (u01(r.x) * (a1 + a2) < a1)
            eps = __expf(-a1 * u01(r.y));
        else
            eps = sqrtf(fmaf(1.0f - e0 * e0, u01(r.y), e0 * e0));
        const float t = __fdividef(1.0f - eps, k * eps);
        const float s2 = t * (2.0f - t);
        const bool ok = u01(r.z) <= 1.0f - __fdividef(eps * s2, 1.0f + eps * eps);
        if (ok || it >= SAMPLER_CAP) {
            if (!ok) ++*capped;
            *c = 1.0f - t;
            *w4 = r.w;
            return eps;
        }
    }
}

// Sauter photo-electron polar angle (§II.A): nu = 1 - cos drawn from
// nu/(A+nu)^3 and accepted with (2-nu)(1/(A+nu)+B) / (2(1/A+B)).
__device__ float sample_sauter(Lane &p, const PlanDev &P, float T, uint32_t *w3, unsigned *capped) {
    const float g = 1.0f + T / kMC2f;
    const float b2 = 1.0f - __fdividef(1.0f, g * g);
    const float beta = sqrtf(b2);
    const float A = __fdividef(__fdividef(1.0f, g * g * (1.0f + beta)), beta);
    const float B = 0.5f * beta * g * (g - 1.0f) * (g - 2.0f);
    const float gmax = 2.0f * (__fdividef(1.0f, A) + B);
    for (int it = 0;; ++it) {
        const uint4 r = draw4(p, P);
        const float sq = sqrtf(u01(r.x));
        const float nu = __fdividef(2.0f * A * sq, A + 2.0f - 2.0f * sq);
        const bool ok = u01(r.y) * gmax <= (2.0f - nu) * (__fdividef(1.0f, A + nu) + B);
        if (ok || it >= SAMPLER_CAP) {
            if (!ok) ++*capped;
            *w3 = r.z;
            return 1.0f - nu;
        }
    }
}

// Moller knock-on fraction in [t_c/T, 1/2] (§II.B.1): 1/eps^2 proposal.
__device__ float sample_moller(Lane &p, const PlanDev &P, float T, float t_c, uint32_t *w3, unsigned *capped) {
    const float g = T / kMC2f + 1.0f;
    const float c1 = __fdividef((g - 1.0f) * (g - 1.0f), g * g);
    const float c2 = __fdividef(2.0f * g - 1.0f, g * g);
    const float ec = __fdividef(t_c, T);
    const float bound = 2.0f + 0.25f * c1;
    for (int it = 0;; ++it) {
        const uint4 r = draw4(p, P);
        const float eps = __fdividef(ec, 1.0f - u01(r.x) * (1.0f - 2.0f * ec));
        const float q = __fdividef(eps, 1.0f - eps);
        const float f = 1.0f + q * q + c1 * eps * eps - c2 * q;
        const bool ok = u01(r.y) * bound <= f;
        if (ok || it >= SAMPLER_CAP) {
            if (!ok) ++*capped;
            *w3 = r.z;
            return eps;
        }
    }
}

// Bremsstrahlung photon energy in [k_c, T] (§II.B.1): 1/k proposal, accepted
// with the normalised shape (4/3 - 4y/3 + y^2) cA + (1 - y) c1.
__device__ float sample_brem(Lane &p, const PlanDev &P, float T, float k_c, float cA, float c1,
                             uint32_t *w3, unsigned *capped) {
    const float E = T + kMC2f;
    const float lr = __logf(__fdividef(T, k_c));
    for (int it = 0;; ++it) {
        const uint4 r = draw4(p, P);
        const float k = k_c * __expf(u01(r.x) * lr);
        const float y = __fdividef(k, E);
        const float gy = fmaf(y, y - 4.0f / 3.0f, 4.0f / 3.0f) * cA + (1.0f - y) * c1;
        const bool ok = u01(r.y) <= gy;
        if (ok || it >= SAMPLER_CAP) {
            if (!ok) ++*capped;
            *w3 = r.z;
            return k;
        }
    }
}

// Multiple-scattering mu = (1 - cos)/2 after G1 transport mean free paths
// (§II.B.2 substitute): f(mu) ~ (mu + a)^-2 with a from the ln(a) table.
__device__ __forceinline__ float ms_mu(const float *tab, const Grid &gr, float g1, float z) {
    if (g1 < (float)MS_G_MIN) return 0.0f;
    if (g1 > (float)MS_G_MAX) return z;
    const float a = __expf(interp_ms(tab + TAB_MS, fmaf(__log2f(g1), gr.ms_a, gr.ms_b)));
    // at z = 1 the exact value is 1; in FP32, 1 + a rounds to 1 when a < 2^-24
    // and the quotient would be a / 0
    return fminf(__fdividef(a * z, 1.0f + a - z), 1.0f);
}

__device__ __forceinline__ float sample_spectrum(const PlanDev &P, float z) {
    const float *cdf = P.spec;
    const float *edges = P.spec + P.n_spec + 1;
    int lo = 0, hi = P.n_spec - 1;  // first bin with cdf[i+1] >= z
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(cdf + mid + 1) >= z) hi = mid; else lo = mid + 1;
    }
    const float c0 = __ldg(cdf + lo), c1 = __ldg(cdf + lo + 1);
    const float f = c1 > c0 ? fminf(fmaxf((z - c0) / (c1 - c0), 0.f), 1.f) : 0.5f;
    const float e0 = __ldg(edges + lo), e1 = __ldg(edges + lo + 1);
    return fmaf(f, e1 - e0, e0);
}

// Primary of history h of plan P (§II.C.2 initParticle): pencil or square
// parallel beam entering through z = 0 along +z; with PHSP, a phase-space
// plan's primary is record h mod n as listed (the first draw is still taken,
// so the draw counter starts where the beams' does).  A source grouped by
// energy starts each history as an ungrouped one does: the grouping orders the
// claims (refill), not the sample.
template <bool PHSP>
__device__ __forceinline__ uint32_t make_primary(Lane &p, const PlanDev &P, uint32_t plan, uint64_t h) {
    p.hist = (uint32_t)h;
    p.lin_lo = 1u;
    p.lin_hi = 0u;
    p.draw = 0u;
    p.plan = plan;
    const uint4 r = draw4(p, P);
    if (PHSP && P.beam == GPUMCD_BEAM_PHASE_SPACE) {
        const float4 *ps = reinterpret_cast<const float4 *>(P.spec);
        const uint32_t k = (uint32_t)(h % (unsigned long long)P.n_phsp);
        const float4 a = __ldg(ps + 2 * (size_t)k), b = __ldg(ps + 2 * (size_t)k + 1);
        p.x = a.x;
        p.y = a.y;
        p.z = a.z;
        p.ux = b.x;
        p.uy = b.y;
        p.uz = b.z;
        p.E = __float2uint_rn(a.w * kInvQf);
        p.act = true;
        return p.E;
    }
    p.x = P.cx;
    p.y = P.cy;
    if (P.beam == GPUMCD_BEAM_SQUARE) {
        p.x = fmaf(u01(r.x) - 0.5f, P.field, P.cx);
        p.y = fmaf(u01(r.y) - 0.5f, P.field, P.cy);
    }
    p.z = 0.0f;
    p.ux = 0.0f;
    p.uy = 0.0f;
    p.uz = 1.0f;
    const float zq = u01(r.z);
    p.E = P.n_spec > 0 ? __float2uint_rn(sample_spectrum(P, zq) * kInvQf) : P.e_src_q;
    p.act = true;
    return p.E;
}

// ---------------------------------------------------------------------------
// Photon transport
// ---------------------------------------------------------------------------
// Photon (GPUMCD §II.A).  photon_flight: one Woodcock flight; true when it
// ends on a real event, with its voxel, the word that picks the interaction,
// and the voxel's material, density and attenuation coefficient.  xp (the
// energy's grid coordinate) and mu_hat (the majorant) are the caller's, taken
// once for all flights of a pass: the energy does not change on a fictitious
// event.  photon_interact: that interaction (Compton, photoelectric or pair,
// by the partial attenuation coefficients of the voxel's material).
__device__ __forceinline__ bool photon_flight(const TransportArgs &A, const Smem &S, Lane &p, float xp,
                                              float mu_hat, uint32_t &idx_out, uint32_t &rz, int &m_out,
                                              float &rho_out, float &mu_out) {
    const PlanDev &P = S.plans[p.plan];
    const Phys &ph = A.phys;
    const uint4 r = draw4(p, P);
    const float s = __fdividef(-__logf(u01(r.x)), mu_hat);
    p.x = fmaf(s, p.ux, p.x);
    p.y = fmaf(s, p.uy, p.y);
    p.z = fmaf(s, p.uz, p.z);
    if (!inside(P, p.x, p.y, p.z)) {
        ledger_add(S, p.plan, 1, p.E);
        p.act = false;
        return false;
    }
    int ix, iy, iz;
    const uint32_t idx = voxel_index(P, p.x, p.y, p.z, ix, iy, iz);
    const uint32_t vw = __ldg(P.vox + idx);
    const int m = vw & (NMAT - 1);  // ids < NMAT (checked when packed): in range by construction
    const float rho = (float)(vw >> 4) * kRhoQ;
    const float *tp = S.tab + tab_ph(m);
    const bool pair_open = p.E > ph.two_mc2_q;
    float mu = rho * interp(tp, xp);
    if (!pair_open) mu = rho * (interp(tp + G, xp) + interp(tp + 2 * G, xp));
    if (u01(r.y) * mu_hat > mu) return false;  // fictitious: direction and energy unchanged
    count(S, CNT_PH_REAL);
    idx_out = idx;
    rz = r.z;
    m_out = m;
    rho_out = rho;
    mu_out = mu;
    return true;
}

template <bool KERMA>
__device__ __forceinline__ void photon_interact(const TransportArgs &A, const Smem &S, Lane &p, uint32_t idx,
                                                uint32_t rz, float xp, int m, float rho, float mu, int gw,
                                                int w) {
    const PlanDev &P = S.plans[p.plan];
    const Phys &ph = A.phys;
    const float *tp = S.tab + tab_ph(m);
    const bool pair_open = p.E > ph.two_mc2_q;
    const float muC = rho * interp(tp + G, xp);
    const float mupe = rho * interp(tp + 2 * G, xp);
    const float q = u01(rz) * mu;
    const float E = (float)p.E * kQf;
    if (q < muC) {
        // Compton scattering on a free electron (Klein-Nishina).
        count(S, CNT_COMPTON);
        float c;
        uint32_t w4;
        unsigned capped = 0;
        const float eps = sample_kn(p, P, E / kMC2f, &c, &w4, &capped);
        if (capped) atomicAdd(&S.cnt[CNT_SAMPLER_CAP], 1ull);
        float sp, cp;
        __sincosf(kTWO_PIf * u01(w4), &sp, &cp);
        const float sn = sqrtf(fmaxf(0.0f, (1.0f - c) * (1.0f + c)));
        const uint32_t e1 = min(p.E, __float2uint_rn(eps * (float)p.E));
        const uint32_t te = p.E - e1;
        float vx = p.ux, vy = p.uy, vz = p.uz;
        rotate(vx, vy, vz, c, sn, cp, sp);
        if (te >= ph.e_abs_q) {
            // recoil direction from momentum balance: E u - E' u'
            const float e1f = (float)e1 * kQf;
            float ex = E * p.ux - e1f * vx, ey = E * p.uy - e1f * vy, ez = E * p.uz - e1f * vz;
            const float n = rsqrtf(fmaxf(ex * ex + ey * ey + ez * ez, 1e-30f));
            emit_electron<KERMA>(A, S, gw, w, P, idx, ex * n, ey * n, ez * n, te, p, 0);
        } else {
            deposit(P, p.hist, idx, te);
        }
        p.ux = vx;
        p.uy = vy;
        p.uz = vz;
        p.E = e1;
        if (e1 < ph.p_cut_q) {
            deposit(P, p.hist, idx, e1);
            p.act = false;
        }
    } else if (q < muC + mupe || !pair_open) {
        // Photoelectric: one K-shell electron carrying all of E (no binding).
        count(S, CNT_PHOTO);
        if (p.E >= ph.e_abs_q) {
            uint32_t w3;
            unsigned capped = 0;
            const float c = sample_sauter(p, P, E, &w3, &capped);
            if (capped) atomicAdd(&S.cnt[CNT_SAMPLER_CAP], 1ull);
            float sp, cp;
            __sincosf(kTWO_PIf * u01(w3), &sp, &cp);
            const float sn = sqrtf(fmaxf(0.0f, (1.0f - c) * (1.0f + c)));
            float vx = p.ux, vy = p.uy, vz = p.uz;
            rotate(vx, vy, vz, c, sn, cp, sp);
            emit_electron<KERMA>(A, S, gw, w, P, idx, vx, vy, vz, p.E, p, 0);
        } else {
            deposit(P, p.hist, idx, p.E);
        }
        p.act = false;
    } else {
        // Pair production without positrons: two electrons share E - 2mc^2
        // uniformly, the rest energy goes to its own ledger.
        count(S, CNT_PAIR);
        const uint32_t tt = p.E - ph.two_mc2_q;
        ledger_add(S, p.plan, 2, ph.two_mc2_q);
        const uint4 r2 = draw4(p, P);
        const uint32_t t1 = min(tt, __float2uint_rn(u01(r2.x) * (float)tt));
        const uint32_t t2 = tt - t1;
        float sp, cp;
        __sincosf(kTWO_PIf * u01(r2.y), &sp, &cp);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const uint32_t te = j == 0 ? t1 : t2;
            if (te >= ph.e_abs_q) {
                const float th = __fdividef(kMC2f, (float)te * kQf + kMC2f);
                float st, ct;
                __sincosf(th, &st, &ct);
                float vx = p.ux, vy = p.uy, vz = p.uz;
                rotate(vx, vy, vz, ct, st, j == 0 ? cp : -cp, j == 0 ? sp : -sp);
                emit_electron<KERMA>(A, S, gw, w, P, idx, vx, vy, vz, te, p, (uint32_t)j);
            } else {
                deposit(P, p.hist, idx, te);
            }
        }
        p.act = false;
    }
}

// ---------------------------------------------------------------------------
// Electron: one condensed-history step (GPUMCD §II.B.3)
// ---------------------------------------------------------------------------
// The energy lost along the step is not deposited here: its voxel and amount
// come back in dep_idx / dep_e so the caller can deposit it at a convergent
// point.  Returns true when a step was taken.  The particle starts inside the
// phantom, so its voxel index is in range: electron primaries are tested when
// they are claimed, secondaries start at interaction points inside, and a
// step that ends outside escapes there.
__device__ bool electron_step(const TransportArgs &A, const Smem &S, Lane &p, int gw, int w,
                              uint32_t &dep_idx, uint32_t &dep_e) {
    const PlanDev &P = S.plans[p.plan];
    const Phys &ph = A.phys;
    int ix, iy, iz;
    const uint32_t idx0 = voxel_index(P, p.x, p.y, p.z, ix, iy, iz);
    const uint32_t vw = __ldg(P.vox + idx0);
    // the step's draw, taken while the voxel word is on its way
    const uint4 r = draw4(p, P);
    const int m0 = vw & (NMAT - 1);
    const float rho0 = (float)(vw >> 4) * kRhoQ;
    if (p.E < ph.e_abs_q) {
        deposit(P, p.hist, idx0, p.E);
        p.act = false;
        return false;
    }
    const float *te = S.tab + tab_el(m0);
    const float T = (float)p.E * kQf;
    const float xe = fmaf(__log2f((float)p.E), ph.grid.el_a, ph.grid.el_bq);
    const float L0 = rho0 * interp(te, xe);
    const float smax = __fdividef(ph.estepe * T, L0);
    // distance to the voxel faces along u, plus the nudge
    float dv = exit_distance(P, p, ix, iy, iz);
    dv = fmaxf(dv, 0.0f) + ph.nudge;
    // The step stays in its voxel (it ends at the exit face, plus the nudge),
    // so the voxel's own hard cross-section at the start energy bounds it over
    // the step: Sigma_hard,m rises with T, and T only falls along the step.
    // The margin covers the rounding of the two interpolations.
    const float sig_hat = rho0 * interp(te + G, xe) * kHardMajorantMargin;
    const float ehard = __fdividef(-__logf(u01(r.x)), sig_hat);
    float es = fminf(dv, smax);
    const bool hard = ehard < es;
    es = fminf(es, ehard);
    // Delta E = e_s L(E0 - L(E0) e_s / 2)
    const float tm = fmaxf(T - 0.5f * L0 * es, 1e-6f);
    const float dE = es * rho0 * interp(te, fmaf(__log2f(tm), ph.grid.el_a, ph.grid.el_bm));
    const uint32_t dq = min(p.E, __float2uint_rn(dE * kInvQf));
    const uint32_t e1 = p.E - dq;
    // random hinge: move z e_s, deflect with the energy before or after the
    // loss (coin from the low bit of the first word), deposit, move (1 - z) e_s
    const float zh = u01(r.y);
    const float l1 = zh * es;
    float x = fmaf(l1, p.ux, p.x), y = fmaf(l1, p.uy, p.y), z = fmaf(l1, p.uz, p.z);
    const float tms = fmaxf((r.x & 1u) ? T : (float)e1 * kQf, 1e-6f);
    const float g1 = es * rho0 * interp(te + 3 * G, fmaf(__log2f(tms), ph.grid.el_a, ph.grid.el_bm));
    const float mu = ms_mu(S.tab, ph.grid, g1, u01(r.z));
    if (mu > 0.0f) {
        float sp, cp;
        __sincosf(kTWO_PIf * u01(r.w), &sp, &cp);
        rotate(p.ux, p.uy, p.uz, 1.0f - 2.0f * mu, 2.0f * sqrtf(mu * (1.0f - mu)), cp, sp);
    }
    dep_idx = idx0;  // the hinge lies in the step-start voxel
    dep_e = dq;
    const float l2 = es - l1;
    // each coordinate one float further along the direction (float_along)
    p.x = float_along(fmaf(l2, p.ux, x), p.ux);
    p.y = float_along(fmaf(l2, p.uy, y), p.uy);
    p.z = float_along(fmaf(l2, p.uz, z), p.uz);
    p.E = e1;
    if (!inside(P, p.x, p.y, p.z)) {
        ledger_add(S, p.plan, 1, e1);
        p.act = false;
        return true;
    }
    int jx, jy, jz;
    const uint32_t idx1 = voxel_index(P, p.x, p.y, p.z, jx, jy, jz);
    if (e1 < ph.e_abs_q) {
        deposit(P, p.hist, idx1, e1);
        p.act = false;
        return true;
    }
    if (!hard) return true;
    // A hard-event candidate: park the particle for a converged hard pass of
    // its warp (the candidate test and the event follow there, with the same
    // random draws in the same order, so the result does not change).
    {
        const unsigned slot = atomicAdd(&S.ws[w].hc, 1u);
        HardRec &h = A.hard[(size_t)gw * HARD_CAP + slot];
        h.r = make_rec(p);
        h.sig_hat = sig_hat;
        h.idx = idx0;
        p.act = false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Electron hard event (GPUMCD §II.B.3): the electron Woodcock test at the end
// of a step whose sampled hard distance was the shortest, then Moller or
// bremsstrahlung.  Runs in the warp's hard pass with the parked candidate in
// the lane: p after its step, sig_hat = the step's majorant, idx1 = the step's
// voxel, which holds the candidate point (the step ends inside it, or at most
// the nudge past its face) and so the event and its sub-cut-off deposits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void hard_event(const TransportArgs &A, const Smem &S, Lane &p, float sig_hat,
                                        uint32_t idx1, int gw, int w) {
    const PlanDev &P = S.plans[p.plan];
    const Phys &ph = A.phys;
    const uint32_t e1 = p.E;
    // electron Woodcock: accept a real hard event with Sigma(T_end)/Sigma_hat
    const uint32_t vw1 = __ldg(P.vox + idx1);
    const uint4 r2 = draw4(p, P);  // the event's draw, taken while the voxel word loads
    const int m1 = vw1 & (NMAT - 1);
    const float rho1 = (float)(vw1 >> 4) * kRhoQ;
    const float *t1 = S.tab + tab_el(m1);
    const float xe1 = fmaf(__log2f((float)e1), ph.grid.el_a, ph.grid.el_bq);
    const float T1 = (float)e1 * kQf;
    // Moller needs T > 2 t_c and bremsstrahlung T > k_c (zero below, as in the
    // closed forms; the interpolated tables are not exactly zero there)
    const float sb = T1 > ph.k_c ? rho1 * interp(t1 + 2 * G, xe1) : 0.0f;
    const float sm = T1 > 2.0f * ph.t_c ? fmaxf(rho1 * interp(t1 + G, xe1) - sb, 0.0f) : 0.0f;
    const float sig = sm + sb;
    if (u01(r2.x) * sig_hat >= sig) {
        count(S, CNT_HARD_FICT);
        return;
    }
    count(S, CNT_HARD_REAL);
    if (u01(r2.y) * sig < sm) {
        // Moller: knock-on and scattered electron, azimuths phi and phi + pi
        count(S, CNT_MOLLER);
        uint32_t w3;
        unsigned capped = 0;
        const float eps = sample_moller(p, P, T1, ph.t_c, &w3, &capped);
        if (capped) atomicAdd(&S.cnt[CNT_SAMPLER_CAP], 1ull);
        const uint32_t tk = min(e1, __float2uint_rn(eps * (float)e1));
        const uint32_t tp = e1 - tk;
        const float tkf = (float)tk * kQf, tpf = (float)tp * kQf;
        const float ck = sqrtf(fminf(1.0f, __fdividef(tkf * (T1 + 2.0f * kMC2f), T1 * (tkf + 2.0f * kMC2f))));
        const float cpp = sqrtf(fminf(1.0f, __fdividef(tpf * (T1 + 2.0f * kMC2f), T1 * (tpf + 2.0f * kMC2f))));
        float sp, cp;
        __sincosf(kTWO_PIf * u01(w3), &sp, &cp);
        float vx = p.ux, vy = p.uy, vz = p.uz;
        rotate(vx, vy, vz, ck, sqrtf(fmaxf(0.f, 1.f - ck * ck)), cp, sp);
        rotate(p.ux, p.uy, p.uz, cpp, sqrtf(fmaxf(0.f, 1.f - cpp * cpp)), -cp, -sp);
        if (tk >= ph.e_abs_q)
            push(A, S, gw, w, 1, p.x, p.y, p.z, vx, vy, vz, tk, p, 0);
        else
            deposit(P, p.hist, idx1, tk);
        p.E = tp;
    } else {
        // bremsstrahlung: electron direction kept, photon at theta = mc^2/E
        count(S, CNT_BREM);
        uint32_t w3;
        unsigned capped = 0;
        const float k = sample_brem(p, P, T1, ph.k_c, S.tab[TAB_BREM + 2 * m1], S.tab[TAB_BREM + 2 * m1 + 1], &w3,
                                    &capped);
        if (capped) atomicAdd(&S.cnt[CNT_SAMPLER_CAP], 1ull);
        const uint32_t kq = min(e1, __float2uint_rn(k * kInvQf));
        const float th = __fdividef(kMC2f, T1 + kMC2f);
        float st, ct, sp, cp;
        __sincosf(th, &st, &ct);
        __sincosf(kTWO_PIf * u01(w3), &sp, &cp);
        float vx = p.ux, vy = p.uy, vz = p.uz;
        rotate(vx, vy, vz, ct, st, cp, sp);
        if (kq >= ph.p_cut_q)
            push(A, S, gw, w, 0, p.x, p.y, p.z, vx, vy, vz, kq, p, 0);
        else
            deposit(P, p.hist, idx1, kq);
        p.E = e1 - kq;
    }
}

// ---------------------------------------------------------------------------
// Warp scheduling helpers (all called by the whole warp, convergent)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Claim `want` records of a global source with a cursor and a fixed count.
__device__ __forceinline__ void claim(unsigned long long *cursor, unsigned long long total, uint32_t want,
                                      unsigned long long &lo, unsigned long long &hi) {
    const unsigned long long base = atomicAdd(cursor, (unsigned long long)want);
    lo = base < total ? base : total;
    hi = base + want < total ? base + want : total;
}

// Per-CTA flags that remember exhausted global sources, so a warp does not
// re-read global counters once a source is known to be empty.
struct CtaFlags {
    int in_done[2];
    int prim_done[2];
};

// Shared memory of a CTA: the plan table, warp states, counters, ledgers, the
// mbarrier and the source flags (fixed size, rounded up to 128 bytes), then the
// tables staged by the bulk copy.
constexpr size_t SMEM_FIXED = (sizeof(PlanDev) * GPUMCD_MAX_PLANS_PER_RUN + sizeof(WarpState) * MAX_WARPS +
                               sizeof(unsigned long long) * (CNT_N + 3 * GPUMCD_MAX_PLANS_PER_RUN + 1) +
                               sizeof(CtaFlags) + 127) / 128 * 128;

// Move the top n records of stack `t` to the global overflow queue.  A full
// queue sets GPUMCD_ERR_QUEUE_OVERFLOW: the run is then invalid and reported,
// never silently truncated.
__device__ void spill_to_queue(const TransportArgs &A, const Smem &S, int gw, int w, int t, unsigned n) {
    const int lane = threadIdx.x & 31;
    const unsigned top = S.ws[w].stk[t];
    n = min(n, top);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(A.out[t].cursor, (unsigned long long)n);
    base = __shfl_sync(FULL, base, 0);
    const Rec *src = A.stacks + ((size_t)gw * 2 + t) * A.stack_cap + (top - n);
    for (unsigned i = lane; i < n; i += 32)
        if (base + i < A.out[t].capacity) A.out[t].rec[base + i] = src[i];
    if (lane == 0) {
        if (base + n > A.out[t].capacity) {
            atomicExch(A.error, GPUMCD_ERR_QUEUE_OVERFLOW);
            atomicAdd(&S.cnt[CNT_OVERFLOW], 1ull);
        }
        S.ws[w].stk[t] = top - n;
        atomicAdd(&S.cnt[CNT_SPILLS], (unsigned long long)n);
    }
    __syncwarp();
}

// Fill empty lanes with particles of type t.  Returns the number of lanes
// that hold a particle afterwards.
template <bool KERMA, bool PHSP>
__device__ int refill(const TransportArgs &A, const Smem &S, CtaFlags &F, Lane &p, int gw, int w, int t) {
    const int lane = threadIdx.x & 31;
    WarpState &ws = S.ws[w];
    unsigned empty = __ballot_sync(FULL, !p.act);
    if (empty == 0u) return 32;
    const unsigned lt = lanemask_lt();
    // 1) the warp's private stack (newest first)
    {
        const unsigned sc = ws.stk[t];
        const unsigned take = min((unsigned)__popc(empty), sc);
        if (take) {
            const unsigned rank = __popc(empty & lt);
            if (!p.act && rank < take)
                load_rec(p, A.stacks[((size_t)gw * 2 + t) * A.stack_cap + (sc - 1u - rank)]);
            __syncwarp();
            if (lane == 0) ws.stk[t] = sc - take;
            __syncwarp();
            empty = __ballot_sync(FULL, !p.act);
            if (empty == 0u) return 32;
        }
    }
    // 2) the overflow queue of the previous launch, in chunks
    for (int pass = 0; pass < 2; ++pass) {
        unsigned long long lo = ws.q_lo[t], hi = ws.q_hi[t];
        if (lo == hi) {
            if (__shfl_sync(FULL, lane == 0 ? *(volatile int *)&F.in_done[t] : 0, 0)) break;
            if (lane == 0) claim(A.in[t].cursor, A.in_count[t], A.chunk, lo, hi);
            lo = __shfl_sync(FULL, lo, 0);
            hi = __shfl_sync(FULL, hi, 0);
            if (lo == hi) {
                if (lane == 0) F.in_done[t] = 1;
                break;
            }
        }
        const unsigned take = (unsigned)min((unsigned long long)__popc(empty), hi - lo);
        const unsigned rank = __popc(empty & lt);
        if (!p.act && rank < take) load_rec(p, A.in[t].rec[lo + rank]);
        __syncwarp();
        if (lane == 0) {
            ws.q_lo[t] = lo + take;
            ws.q_hi[t] = hi;
        }
        __syncwarp();
        empty = __ballot_sync(FULL, !p.act);
        if (empty == 0u) return 32;
    }
    // 3) primaries of this type, in chunks
    for (int pass = 0; pass < 2; ++pass) {
        unsigned long long lo = ws.p_lo[t], hi = ws.p_hi[t];
        if (lo == hi) {
            if (__shfl_sync(FULL, lane == 0 ? *(volatile int *)&F.prim_done[t] : 0, 0)) break;
            if (lane == 0) claim(&A.prim_cursor[t], A.prim_off[t][A.n_prim_plans[t]], A.chunk, lo, hi);
            lo = __shfl_sync(FULL, lo, 0);
            hi = __shfl_sync(FULL, hi, 0);
            if (lo == hi) {
                if (lane == 0) F.prim_done[t] = 1;
                break;
            }
        }
        const unsigned take = (unsigned)min((unsigned long long)__popc(empty), hi - lo);
        const unsigned rank = __popc(empty & lt);
        if (!p.act && rank < take) {
            const unsigned long long g = lo + rank;
            int a = 0, b = (int)A.n_prim_plans[t] - 1;  // last plan with prim_off <= g
            while (a < b) {
                const int mid = (a + b + 1) >> 1;
                if (A.prim_off[t][mid] <= g) a = mid; else b = mid - 1;
            }
            const uint32_t plan = A.prim_plan[t][a];
            const PlanDev &P = S.plans[plan];
            unsigned long long j = g - A.prim_off[t][a];
            // a source grouped by energy: its histories are claimed in
            // decreasing order of their energy (the order its launch sorted)
            if (PHSP && P.e_group && j < P.n_sorted) j = __ldg(P.order + j);
            ledger_add(S, plan, 0, make_primary<PHSP>(p, P, plan, P.hist_base + j));
            if (t == 0 && p.E < A.phys.p_cut_q) {
                // a photon primary below the photon cut-off deposits where it
                // starts, or escapes from outside (every other photon flies
                // above the cut-off)
                if (inside(P, p.x, p.y, p.z)) {
                    int ix, iy, iz;
                    deposit(P, p.hist, voxel_index(P, p.x, p.y, p.z, ix, iy, iz), p.E);
                } else {
                    ledger_add(S, plan, 1, p.E);
                }
                p.act = false;
            }
            if (!KERMA && t == 1 && !inside(P, p.x, p.y, p.z)) {
                // an electron primary aimed outside the phantom escapes at once
                // (every other electron starts its steps inside)
                ledger_add(S, plan, 1, p.E);
                p.act = false;
            }
            if (KERMA && t == 1) {
                // photon-only mode: a primary electron deposits where it enters
                if (inside(P, p.x, p.y, p.z)) {
                    int ix, iy, iz;
                    deposit(P, p.hist, voxel_index(P, p.x, p.y, p.z, ix, iy, iz), p.E);
                } else {
                    ledger_add(S, plan, 1, p.E);
                }
                p.act = false;
            }
        }
        __syncwarp();
        if (lane == 0) {
            ws.p_lo[t] = lo + take;
            ws.p_hi[t] = hi;
            atomicAdd(&S.cnt[t == 0 ? CNT_PHOTONS : CNT_ELECTRONS], (unsigned long long)take);
        }
        __syncwarp();
        empty = __ballot_sync(FULL, !p.act);
        if (empty == 0u) return 32;
    }
    return 32 - __popc(empty);
}

// Particles of type t the warp could still take (a global source counts 32).
// Evaluated by lane 0 and broadcast, so the whole warp takes the same branch.
__device__ __forceinline__ unsigned available(const TransportArgs &A, const Smem &S, CtaFlags &F, int w,
                                              int t) {
    unsigned n = 0;
    if ((threadIdx.x & 31) == 0) {
        const WarpState &ws = S.ws[w];
        n = ws.stk[t] + (t == 1 ? ws.hc : 0u);  // parked hard candidates are electrons
        if (ws.q_lo[t] < ws.q_hi[t]) n += 32;
        else if (!*(volatile int *)&F.in_done[t]) {
            if (*(volatile unsigned long long *)A.in[t].cursor < A.in_count[t]) n += 32;
            else F.in_done[t] = 1;
        }
        if (ws.p_lo[t] < ws.p_hi[t]) n += 32;
        else if (!*(volatile int *)&F.prim_done[t]) {
            if (*(volatile unsigned long long *)&A.prim_cursor[t] < A.prim_off[t][A.n_prim_plans[t]]) n += 32;
            else F.prim_done[t] = 1;
        }
    }
    return __shfl_sync(FULL, n, 0);
}

// The warp's hard pass: park its stepping electrons on their stack, take up
// to 32 parked hard-event candidates into the lanes and run their events
// together.  The lanes then hold electrons again (after their events), so
// the warp goes on stepping electrons.
__device__ __forceinline__ void hard_pass(const TransportArgs &A, const Smem &S, Lane &p, int gw, int w) {
    const int lane = threadIdx.x & 31;
    if (S.ws[w].stk[1] + 32u > A.stack_cap) spill_to_queue(A, S, gw, w, 1, 64u);
    const unsigned actm = __ballot_sync(FULL, p.act);
    const unsigned base = S.ws[w].stk[1];
    if (p.act) {
        const unsigned rank = __popc(actm & lanemask_lt());
        A.stacks[((size_t)gw * 2 + 1) * A.stack_cap + base + rank] = make_rec(p);
        p.act = false;
    }
    __syncwarp();
    const unsigned hc = S.ws[w].hc;
    const unsigned take = min(32u, hc);
    float sig_hat = 0.f;
    uint32_t idx1 = 0u;
    if ((unsigned)lane < take) {
        const HardRec &h = A.hard[(size_t)gw * HARD_CAP + (hc - 1u - lane)];
        load_rec(p, h.r);
        sig_hat = h.sig_hat;
        idx1 = h.idx;
    }
    __syncwarp();
    if (lane == 0) {
        S.ws[w].stk[1] = base + __popc(actm);
        S.ws[w].hc = hc - take;
        atomicAdd(&S.cnt[CNT_HARD_PASSES], 1ull);
    }
    __syncwarp();
    // headroom for the events' secondaries (at most one per lane per type)
    if (S.ws[w].stk[0] + 64u > A.stack_cap) spill_to_queue(A, S, gw, w, 0, 64u);
    if (S.ws[w].stk[1] + 64u > A.stack_cap) spill_to_queue(A, S, gw, w, 1, 64u);
    if (p.act) hard_event(A, S, p, sig_hat, idx1, gw, w);
    __syncwarp();
}

// Woodcock flights a photon takes in one pass while its events are fictitious.
constexpr int PH_FLIGHTS = 3;

// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// PROF compiles in the per-type cycle profile (GPUMCD_LAUNCH_PROFILE), AGG
// the warp-aggregated deposit (GPUMCD_LAUNCH_WARP_AGGREGATE), SCHED the
// refill policies of the divergence-reduction ablation (refill_period != 1),
// KERMA the photon-only mode (GPUMCD_LAUNCH_KERMA) and PHSP phase-space
// sources; the production instantiations carry none of them.
template <int MAXT, int MINB, bool PROF, bool AGG, bool SCHED, bool KERMA, bool PHSP>
__global__ void __launch_bounds__(MAXT, MINB) k_transport(const __grid_constant__ TransportArgs A) {
    // the fixed-size parts first, at offsets known at compile time; the tables
    // of the loaded materials after them
    extern __shared__ __align__(128) unsigned char smem_raw[];
    PlanDev *plans = (PlanDev *)smem_raw;
    WarpState *ws = (WarpState *)(plans + GPUMCD_MAX_PLANS_PER_RUN);
    unsigned long long *cnt = (unsigned long long *)(ws + MAX_WARPS);
    unsigned long long *ledger = cnt + CNT_N;
    unsigned long long *mbar = ledger + 3 * GPUMCD_MAX_PLANS_PER_RUN;
    CtaFlags *flags = (CtaFlags *)(mbar + 1);
    float *tab = (float *)(smem_raw + SMEM_FIXED);

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int gw = blockIdx.x * (blockDim.x >> 5) + w;

    // Stage the material tables into shared memory with one bulk (TMA) copy
    // completed on an mbarrier; the other threads set up the rest meanwhile.
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)),
                     "r"(A.tab_bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_addr(tab)),
            "l"(A.tables), "r"(A.tab_bytes), "r"(smem_addr(mbar))
            : "memory");
    }
    // every entry is set (unused ones copy plan 0), so any masked plan index
    // a record carries reaches valid pointers
    for (int i = tid; i < GPUMCD_MAX_PLANS_PER_RUN; i += blockDim.x) plans[i] = A.plans[i < A.n_plans ? i : 0];
    for (int i = tid; i < MAX_WARPS; i += blockDim.x) {
        ws[i].stk[0] = ws[i].stk[1] = 0;
        ws[i].hc = 0;
        ws[i].p_lo[0] = ws[i].p_hi[0] = ws[i].p_lo[1] = ws[i].p_hi[1] = 0;
        ws[i].q_lo[0] = ws[i].q_hi[0] = ws[i].q_lo[1] = ws[i].q_hi[1] = 0;
    }
    for (int i = tid; i < CNT_N + 3 * GPUMCD_MAX_PLANS_PER_RUN; i += blockDim.x) cnt[i] = 0;
    if (tid < 2) {
        flags->in_done[tid] = A.in_count[tid] == 0;
        flags->prim_done[tid] = A.prim_off[tid][A.n_prim_plans[tid]] == 0;
    }
    __syncthreads();  // also orders the mbarrier init before the waits below
    uint32_t done = 0;
    for (uint32_t it = 0; it < (1u << 26) && !done; ++it) {
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(smem_addr(mbar))
            : "memory");
    }
    if (__syncthreads_or(!done)) {
        // The table copy did not complete within the bound: report it and
        // leave without touching the tables.
        if (tid == 0) atomicExch(A.error, GPUMCD_ERR_TIMEOUT);
        return;
    }
    const Smem S{tab, plans, ws, cnt, ledger};
    CtaFlags &F = *flags;

    Lane p;
    p.act = false;
    p.x = p.y = p.z = p.ux = p.uy = p.uz = 0.f;
    p.E = p.hist = p.lin_lo = p.lin_hi = p.draw = p.plan = 0;
    constexpr bool agg = AGG;
    constexpr bool prof = PROF;
    // start on the type that has work (electron-beam launches start on electrons)
    int t = available(A, S, F, w, 1) > available(A, S, F, w, 0) ? 1 : 0;
    unsigned iter = 0;
    for (;;) {
        __syncwarp();
        if ((++iter & 255u) == 0u) {
            int err = 0;
            if (lane == 0) err = *(volatile int *)A.error;
            if (__shfl_sync(FULL, err, 0) != 0) break;
            if (iter >= (1u << 24)) {
                if (lane == 0) atomicExch(A.error, GPUMCD_ERR_TIMEOUT);
                break;
            }
        }
        long long c0 = prof ? clock64() : 0;
        int n_act;
        bool fresh = true;  // this pass refilled the lanes
        if (SCHED && A.refill_period != 1u) {
            // the ablation's refill policies (GPUMCD §II.C.3): empty lanes wait
            // for every N-th pass, or for the whole warp to empty
            const unsigned actm = __ballot_sync(FULL, p.act);
            if (actm != 0u && (A.refill_period == 0xFFFFFFFFu || iter % A.refill_period != 0u)) {
                n_act = __popc(actm);
                fresh = false;
            } else {
                n_act = refill<KERMA, PHSP>(A, S, F, p, gw, w, t);
            }
        } else {
            n_act = refill<KERMA, PHSP>(A, S, F, p, gw, w, t);
        }
        if (prof && lane == 0) atomicAdd(&S.cnt[CNT_PROF_REFILL_CYC], (unsigned long long)(clock64() - c0));
        const int o = 1 - t;
        // electrons: a converged hard pass once 32 candidates are parked (a
        // step parks at most 32 more, within HARD_CAP), or sooner when the
        // warp has few electrons left to step
        if (t == 1) {
            const unsigned hc = S.ws[w].hc;
            // With few electrons left (the drain), a pass runs once the parked
            // candidates outnumber the stepping electrons, not at every
            // iteration; n_act == 0 keeps parked candidates from being left
            // behind (also when refill_low is 0).
            if (hc >= 32u || (hc > 0u && (n_act == 0 || (n_act < (int)A.refill_low && hc >= (unsigned)n_act)))) {
                hard_pass(A, S, p, gw, w);
                continue;
            }
        }
        if (n_act == 0) {
            if (available(A, S, F, w, o) > 0u) {
                t = o;
                continue;
            }
            break;  // nothing left of either type for this warp
        }
        const unsigned so = S.ws[w].stk[o], st = S.ws[w].stk[t];
        if ((so >= A.switch_high && so > st + 32u) ||
            (n_act < (int)A.refill_low && fresh && available(A, S, F, w, o) >= 32u)) {
            if (prof && lane == 0) atomicAdd(&S.cnt[CNT_PROF_SWITCHES], 1ull);
            // switch type: park the current particles on their stack
            if (S.ws[w].stk[t] + 32u > A.stack_cap) spill_to_queue(A, S, gw, w, t, 64u);
            const unsigned actm = __ballot_sync(FULL, p.act);
            const unsigned base = S.ws[w].stk[t];
            if (p.act) {
                const unsigned rank = __popc(actm & lanemask_lt());
                A.stacks[((size_t)gw * 2 + t) * A.stack_cap + base + rank] = make_rec(p);
                p.act = false;
            }
            __syncwarp();
            if (lane == 0) S.ws[w].stk[t] = base + __popc(actm);
            __syncwarp();
            t = o;
            continue;
        }
        if (prof) c0 = clock64();
        // headroom for this step's secondaries (at most two per lane)
        if (S.ws[w].stk[0] + 64u > A.stack_cap) spill_to_queue(A, S, gw, w, 0, 64u);
        if (S.ws[w].stk[1] + 64u > A.stack_cap) spill_to_queue(A, S, gw, w, 1, 64u);
        if (t == 0) {
            // Up to PH_FLIGHTS Woodcock flights per lane until its event is
            // real, then the real events' interactions together: with many
            // fictitious events (low densities under a high majorant) more
            // lanes reach an interaction per pass; in a homogeneous medium
            // every first flight is real and the loop ends at once.  The
            // energy, so its grid coordinate and majorant, stays the same
            // over the flights of a pass.
            uint32_t pidx = 0u, prz = 0u;
            bool real = false;
            const float xp = fmaf(__log2f((float)p.E), A.phys.grid.ph_a, A.phys.grid.ph_bq);
            const float mu_hat = p.act ? interp_ldg(S.plans[p.plan].maj, xp) : 1.0f;
            int rm = 0;
            float rrho = 0.f, rmu = 0.f;
            for (int k = 0; k < PH_FLIGHTS; ++k) {
                const bool fly = p.act && !real;
                const unsigned flym = __ballot_sync(FULL, fly);
                if (flym == 0u) break;
                if (lane == 0) atomicAdd(&S.cnt[CNT_PH_EVENTS], (unsigned long long)__popc(flym));
                if (fly) real = photon_flight(A, S, p, xp, mu_hat, pidx, prz, rm, rrho, rmu);
            }
            if (real) photon_interact<KERMA>(A, S, p, pidx, prz, xp, rm, rrho, rmu, gw, w);
        } else {
            uint32_t dep_idx = 0, dep_e = 0;
            bool stepped = false;
            if (p.act) stepped = electron_step(A, S, p, gw, w, dep_idx, dep_e);
            const unsigned sm = __ballot_sync(FULL, stepped);
            if (lane == 0) atomicAdd(&S.cnt[CNT_E_STEPS], (unsigned long long)__popc(sm));
            const PlanDev &P = S.plans[p.plan];
            if (agg)
                deposit_aggregated(P, p.hist, dep_idx, dep_e);
            else
                deposit(P, p.hist, dep_idx, dep_e);
        }
        if (prof) {
            __syncwarp();
            if (lane == 0) {
                atomicAdd(&S.cnt[CNT_PROF_CYC + t], (unsigned long long)(clock64() - c0));
                atomicAdd(&S.cnt[CNT_PROF_ITER + t], 1ull);
                atomicAdd(&S.cnt[CNT_PROF_LANES + t], (unsigned long long)n_act);
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < CNT_N; i += blockDim.x)
        if (cnt[i]) atomicAdd(&A.counters[i], cnt[i]);
    for (int i = tid; i < 3 * A.n_plans; i += blockDim.x)
        if (ledger[i]) atomicAdd(&plans[i / 3].ledger[i % 3], ledger[i]);
}

size_t transport_smem_bytes(uint32_t tab_bytes) { return (size_t)SMEM_FIXED + tab_bytes; }

// Instantiations by register budget.  A launch bound (threads, CTAs) caps the
// registers at 65536 / (threads x CTAs), and a kernel built for a budget runs
// any launch with no more threads per CTA and no more threads per SM than its
// bound: 128 registers up to 512 threads per SM, 80 up to 768, 64 up to 1024.
// The 64-register kernel is the production one at its default shape, 1024
// threads x 1 CTA per SM: the same 32 warps per SM as 512 x 2 but one copy of
// the tables in shared memory, which leaves the larger L1 carve-out to the
// voxel words, majorants and stack records (5-6% faster on the batched
// workload than 512 x 2 in a same-box A/B).  The profile, aggregation,
// refill-policy, photon-only and phase-space kernels are built for it too.
typedef void (*TransportKernel)(const TransportArgs);
struct Variant {
    int max_threads, min_blocks;
    bool prof, agg, sched, kerma, phsp;
    TransportKernel fn;
};
static const Variant kVariants[] = {
    {512, 1, false, false, false, false, false, k_transport<512, 1, false, false, false, false, false>},
    {384, 2, false, false, false, false, false, k_transport<384, 2, false, false, false, false, false>},
    {1024, 1, false, false, false, false, false, k_transport<1024, 1, false, false, false, false, false>},
    {1024, 1, true, false, false, false, false, k_transport<1024, 1, true, false, false, false, false>},
    {1024, 1, false, true, false, false, false, k_transport<1024, 1, false, true, false, false, false>},
    {1024, 1, false, false, true, false, false, k_transport<1024, 1, false, false, true, false, false>},
    {1024, 1, false, false, false, true, false, k_transport<1024, 1, false, false, false, true, false>},
    {1024, 1, false, false, false, false, true, k_transport<1024, 1, false, false, false, false, true>},
};

// The first variant (most registers first) whose bound covers the launch.
static TransportKernel pick_variant(int block, int blocks_per_sm, bool prof, bool agg, bool sched, bool kerma,
                                    bool phsp) {
    for (const Variant &v : kVariants)
        if (v.prof == prof && v.agg == agg && v.sched == sched && v.kerma == kerma && v.phsp == phsp &&
            block <= v.max_threads && block * blocks_per_sm <= v.max_threads * v.min_blocks)
            return v.fn;
    return nullptr;
}

cudaError_t transport_configure() {
    for (const Variant &v : kVariants) {
        cudaError_t e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)transport_smem_bytes(TAB_BYTES));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

const void *transport_kernel(const TransportArgs &a, int block, int blocks_per_sm) {
    return (const void *)pick_variant(block, blocks_per_sm, (a.flags & GPUMCD_LAUNCH_PROFILE) != 0u,
                                      (a.flags & GPUMCD_LAUNCH_WARP_AGGREGATE) != 0u, a.refill_period != 1u,
                                      (a.flags & GPUMCD_LAUNCH_KERMA) != 0u, a.phsp != 0u);
}

cudaError_t launch_transport(const TransportArgs &a, int grid, int block, int blocks_per_sm, cudaStream_t s) {
    TransportKernel fn = (TransportKernel)transport_kernel(a, block, blocks_per_sm);
    if (!fn) return cudaErrorInvalidConfiguration;
    if (a.tab_bytes < tab_bytes(1) || a.tab_bytes > (uint32_t)TAB_BYTES) return cudaErrorInvalidValue;
    fn<<<grid, block, transport_smem_bytes(a.tab_bytes), s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Energy grouping of a spectrum or a phase space (GPUMCD §IV): before a
// launch, a counting sort puts the plan's histories in decreasing order of
// their primary's energy bin, and the launch claims them in that order.  Each
// history starts as an ungrouped one does (the same draw, or the same record,
// in make_primary), so the tally does not change; warps, and the whole grid at
// any moment, start histories of similar energy, the longest first.
// ---------------------------------------------------------------------------
constexpr int GROUP_THREADS = 256;
constexpr uint32_t GROUP_PER_BLOCK = 16 * GROUP_THREADS;

// Energy bins of a grouped phase space: 64 to an octave over [2^-10, 2^6) MeV,
// from the float's exponent and top six mantissa bits (exact and monotone for
// E > 0; energies outside the range share the end bins).
constexpr int PHSP_GROUP_BINS = GPUMCD_MAX_SPECTRUM_BINS;
static_assert(PHSP_GROUP_BINS == 1024, "16 octaves x 64 bins");

__device__ __forceinline__ int group_bins(const PlanDev &P) {
    return P.beam == GPUMCD_BEAM_PHASE_SPACE ? PHSP_GROUP_BINS : P.n_spec;
}

// The energy bin of history h's primary, counted from the top: a phase
// space's record h mod n, or the spectrum bin the history's own draw picks.
__device__ __forceinline__ int group_key(const PlanDev &P, unsigned long long h) {
    if (P.beam == GPUMCD_BEAM_PHASE_SPACE) {
        const float4 *ps = reinterpret_cast<const float4 *>(P.spec);
        const float E = __ldg(ps + 2 * (size_t)(h % (unsigned long long)P.n_phsp)).w;
        const int b = (int)(__float_as_uint(E) >> 17) - ((127 - 10) << 6);
        return PHSP_GROUP_BINS - 1 - min(max(b, 0), PHSP_GROUP_BINS - 1);
    }
    Lane p;
    p.hist = (uint32_t)h;
    p.lin_lo = 1u;
    p.lin_hi = 0u;
    p.draw = 0u;
    p.plan = 0u;
    const uint4 r = draw4(p, P);
    const float z = u01(r.z);
    const float *cdf = P.spec;
    int lo = 0, hi = P.n_spec - 1;  // first bin with cdf[i+1] >= z, as sample_spectrum finds it
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(cdf + mid + 1) >= z) hi = mid; else lo = mid + 1;
    }
    return P.n_spec - 1 - lo;
}

// Count: each history's key, once, into keys[j]; the block's bin counts into
// count.  Lanes of a warp with the same key add once (one shared atomic per
// distinct key in the warp).
__global__ void __launch_bounds__(GROUP_THREADS) k_group_count(const __grid_constant__ PlanDev P, uint32_t n,
                                                               unsigned *count, uint16_t *keys) {
    __shared__ unsigned local[GPUMCD_MAX_SPECTRUM_BINS];
    const int nb = group_bins(P);
    const unsigned lt = lanemask_lt();
    // the block's histories in rounds of one per thread: the same trip count
    // for every thread, so whole warps take part in each match
    const uint32_t j0 = blockIdx.x * GROUP_PER_BLOCK, jend = min(n, j0 + GROUP_PER_BLOCK);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) local[i] = 0u;
    __syncthreads();
    for (uint32_t jb = j0; jb < jend; jb += blockDim.x) {
        const uint32_t j = jb + threadIdx.x;
        const int k = j < jend ? group_key(P, P.hist_base + j) : -1;
        const unsigned same = __match_any_sync(FULL, k);
        if (k >= 0) {
            keys[j] = (uint16_t)k;
            if ((same & lt) == 0u) atomicAdd(&local[k], (unsigned)__popc(same));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (local[i]) atomicAdd(&count[i], local[i]);
}

// Exclusive prefix sum of the bin counts, in place: one block of
// GPUMCD_MAX_SPECTRUM_BINS threads, a bin each (scans within the warps, then
// over the warps' totals).
constexpr int GROUP_SCAN_THREADS = GPUMCD_MAX_SPECTRUM_BINS;
__global__ void __launch_bounds__(GROUP_SCAN_THREADS) k_group_scan(unsigned *count, int n_bins) {
    __shared__ unsigned warp_sum[GROUP_SCAN_THREADS / 32];
    const int i = threadIdx.x, lane = i & 31, wid = i >> 5;
    const unsigned c = i < n_bins ? count[i] : 0u;
    unsigned v = c;  // inclusive scan within the warp
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned u = __shfl_up_sync(FULL, v, d);
        if (lane >= d) v += u;
    }
    if (lane == 31) warp_sum[wid] = v;
    __syncthreads();
    if (wid == 0) {
        unsigned t = lane < GROUP_SCAN_THREADS / 32 ? warp_sum[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned u = __shfl_up_sync(FULL, t, d);
            if (lane >= d) t += u;
        }
        if (lane < GROUP_SCAN_THREADS / 32) warp_sum[lane] = t;  // inclusive over the warps
    }
    __syncthreads();
    if (i < n_bins) count[i] = v - c + (wid > 0 ? warp_sum[wid - 1] : 0u);
}

// Each block reserves, per bin, room for its histories of that bin, then
// writes their offsets there (the order within a bin is not fixed: claims in
// any order give the same tally).  The keys come from k_group_count.
__global__ void __launch_bounds__(GROUP_THREADS) k_group_scatter(const __grid_constant__ PlanDev P, uint32_t n,
                                                                 unsigned *cursor, const uint16_t *keys,
                                                                 uint32_t *order) {
    __shared__ unsigned local[GPUMCD_MAX_SPECTRUM_BINS];
    __shared__ unsigned base[GPUMCD_MAX_SPECTRUM_BINS];
    const int nb = group_bins(P);
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const uint32_t j0 = blockIdx.x * GROUP_PER_BLOCK, jend = min(n, j0 + GROUP_PER_BLOCK);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) local[i] = 0u;
    __syncthreads();
    for (uint32_t jb = j0; jb < jend; jb += blockDim.x) {
        const uint32_t j = jb + threadIdx.x;
        const int k = j < jend ? (int)keys[j] : -1;
        const unsigned same = __match_any_sync(FULL, k);
        if (k >= 0 && (same & lt) == 0u) atomicAdd(&local[k], (unsigned)__popc(same));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        base[i] = local[i] ? atomicAdd(&cursor[i], local[i]) : 0u;
        local[i] = 0u;
    }
    __syncthreads();
    for (uint32_t jb = j0; jb < jend; jb += blockDim.x) {
        const uint32_t j = jb + threadIdx.x;
        const int k = j < jend ? (int)keys[j] : -1;
        const unsigned same = __match_any_sync(FULL, k);
        const int leader = __ffs(same) - 1;
        unsigned slot = 0u;
        if (k >= 0 && lane == leader) slot = atomicAdd(&local[k], (unsigned)__popc(same));
        slot = __shfl_sync(FULL, slot, leader);
        if (k >= 0) order[base[k] + slot + (unsigned)__popc(same & lt)] = j;
    }
}

cudaError_t launch_group_order(const PlanDev &P, uint32_t n, unsigned *count, uint16_t *keys, uint32_t *order,
                               cudaStream_t s) {
    const int nb = P.beam == GPUMCD_BEAM_PHASE_SPACE ? (P.n_phsp > 0 ? PHSP_GROUP_BINS : 0) : P.n_spec;
    if (nb < 1 || nb > GPUMCD_MAX_SPECTRUM_BINS || n == 0 || !P.spec) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(count, 0, (size_t)nb * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (n + GROUP_PER_BLOCK - 1) / GROUP_PER_BLOCK;
    k_group_count<<<blocks, GROUP_THREADS, 0, s>>>(P, n, count, keys);
    k_group_scan<<<1, GROUP_SCAN_THREADS, 0, s>>>(count, nb);
    k_group_scatter<<<blocks, GROUP_THREADS, 0, s>>>(P, n, count, keys, order);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Sampler diagnostics: the same device samplers, one draw per thread.
// ---------------------------------------------------------------------------
__global__ void k_debug_sample(const float *tabg, Phys ph, int kind, float p0, int material,
                               const float *spec, int n_spec, uint64_t n, uint64_t seed, float *out) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    PlanDev P{};
    P.key_lo = (uint32_t)seed;
    P.key_hi = (uint32_t)(seed >> 32);
    P.spec = spec;
    P.n_spec = n_spec;
    Lane p;
    p.hist = (uint32_t)i;
    p.lin_lo = (uint32_t)(i >> 32);
    p.lin_hi = 0x5EEDu;
    p.draw = 0;
    p.plan = 0;
    float v = 0.f;
    uint32_t wd;
    unsigned capped = 0;
    if (kind == 0 || kind == 6) {
        float c;
        const float eps = sample_kn(p, P, p0 / kMC2f, &c, &wd, &capped);
        v = kind == 0 ? c : eps;
    } else if (kind == 1) {
        v = sample_sauter(p, P, p0, &wd, &capped);
    } else if (kind == 2) {
        v = sample_moller(p, P, p0, ph.t_c, &wd, &capped);
    } else if (kind == 3) {
        v = sample_brem(p, P, p0, ph.k_c, __ldg(tabg + TAB_BREM + 2 * material),
                        __ldg(tabg + TAB_BREM + 2 * material + 1), &wd, &capped);
    } else if (kind == 4) {
        // the transport's own ms_mu, given the tables in global memory instead
        // of their shared-memory copy (the same word of the draw as a step uses)
        const uint4 r = draw4(p, P);
        v = ms_mu(tabg, ph.grid, p0, u01(r.z));
    } else if (kind == 5) {
        const uint4 r = draw4(p, P);
        v = sample_spectrum(P, u01(r.z));
    }
    out[i] = capped ? __int_as_float(0x7fc00000) : v;  // a capped draw shows up as NaN
}

cudaError_t launch_debug_sample(const float *tab, const Phys &phys, int kind, float p0, int material,
                                const float *spec, int n_spec, uint64_t n, uint64_t seed, float *out,
                                cudaStream_t s) {
    const int grid = (int)((n + 255) / 256);
    k_debug_sample<<<grid ? grid : 1, 256, 0, s>>>(tab, phys, kind, p0, material, spec, n_spec, n, seed, out);
    return cudaGetLastError();
}

}  // namespace gm
