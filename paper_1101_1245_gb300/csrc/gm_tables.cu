// FP64 device kernels of the gpumcd library: material tables, phantom
// packing, majorants, spectrum CDF, the dose/uncertainty fold and reductions.
#include <curand_kernel.h>

#include <mutex>

#include "gm_common.cuh"
#include "gm_host.h"

namespace gm {

// ---------------------------------------------------------------------------
// Closed-form physics in FP64 (tables are built from these on the device).
// ---------------------------------------------------------------------------
struct MatDev {
    int n;
    int Z[GPUMCD_MAX_ELEMENTS];
    double N[GPUMCD_MAX_ELEMENTS];  // atoms per gram
    double I_mc2;                    // mean excitation energy / mc^2
};

__device__ double electrons_per_gram(const MatDev &m) {
    double s = 0.0;
    for (int j = 0; j < m.n; ++j) s += m.N[j] * m.Z[j];
    return s;
}

// Klein-Nishina total per electron (GPUMCD §II.A, Compton scattering).
__device__ double kn_total(double k) {
    const double r2 = kRE * kRE;
    const double b = 1.0 + 2.0 * k;
    const double lb = log1p(2.0 * k);
    const double inv_k = 1.0 / k;
    const double part1 = (1.0 + k) * inv_k * inv_k * (2.0 * (1.0 + k) / b - lb * inv_k);
    const double part2 = 0.5 * lb * inv_k;
    const double part3 = (1.0 + 3.0 * k) / (b * b);
    return 2.0 * kPI * r2 * (part1 + part2 - part3);
}

// Photon mass attenuation components at E (cm^2/g): Compton, K-shell Born
// photoelectric, complete-screening pair with the (1 - 2mc^2/E)^3 threshold factor.
__device__ void photon_mu(const MatDev &m, double E, double *muC, double *mupe, double *mupp) {
    const double k = E / kMC2;
    *muC = electrons_per_gram(m) * kn_total(k);
    const double sT = 8.0 * kPI / 3.0 * kRE * kRE;
    const double a2 = kALPHA * kALPHA;
    const double kpow = 1.0 / (k * k * k * sqrt(k));
    double pe = 0.0, pp = 0.0;
    for (int j = 0; j < m.n; ++j) {
        const double z = m.Z[j];
        const double z2 = z * z;
        pe += m.N[j] * 4.0 * sqrt(2.0) * a2 * a2 * z2 * z2 * z * sT * kpow;
        const double lscr = log(183.0) - log(z) / 3.0;
        pp += m.N[j] * 4.0 * kALPHA * kRE * kRE * z * (z + 1.0) * ((7.0 / 9.0) * lscr - 1.0 / 54.0);
    }
    *mupe = pe;
    if (E > 2.0 * kMC2) {
        const double t = 1.0 - 2.0 * kMC2 / E;
        *mupp = pp * t * t * t;
    } else {
        *mupp = 0.0;
    }
}

// Restricted collision stopping power (GPUMCD §II.B.3, L(E, K_cut)), Bethe
// with Moller close collisions, no density effect; energy transfers above
// t_c excluded (Delta = min(t_c, T/2)).
__device__ double collision_loss(const MatDev &m, double T, double t_c) {
    const double tau = T / kMC2, g = tau + 1.0, b2 = 1.0 - 1.0 / (g * g);
    const double D = fmin(t_c, 0.5 * T) / kMC2;
    const double F = -1.0 - b2 + log((tau - D) * D) + tau / (tau - D) +
                     (0.5 * D * D + (2.0 * tau + 1.0) * log1p(-D / tau)) / (g * g);
    const double lead = log(2.0 * (tau + 2.0)) - 2.0 * log(m.I_mc2);
    return 2.0 * kPI * kRE * kRE * kMC2 * electrons_per_gram(m) / b2 * (lead + F);
}

// Complete-screening bremsstrahlung: per-material sums S_A = sum N Z(Z+1)
// ln(183 Z^-1/3) and S_1 = sum N Z(Z+1).
__device__ void brem_sums(const MatDev &m, double *SA, double *S1) {
    double a = 0.0, b = 0.0;
    for (int j = 0; j < m.n; ++j) {
        const double z = m.Z[j];
        const double w = m.N[j] * z * (z + 1.0);
        a += w * (log(183.0) - log(z) / 3.0);
        b += w;
    }
    *SA = a;
    *S1 = b;
}

// Soft radiative loss (photons below k_c) and hard bremsstrahlung
// cross-section (photons in [k_c, T]), GPUMCD §II.B.1 and §II.B.3.
__device__ void brem_parts(const MatDev &m, double T, double k_c, double *soft, double *hard) {
    double SA, S1;
    brem_sums(m, &SA, &S1);
    const double c = 4.0 * kALPHA * kRE * kRE;
    const double E = T + kMC2;
    const double K = fmin(k_c, T);
    const double ia = K * (4.0 / 3.0 - K * (2.0 / 3.0) / E + K * K / (3.0 * E * E));
    const double ib = K * (1.0 - 0.5 * K / E);
    *soft = c * (SA * ia + S1 * ib / 9.0);
    if (T > k_c) {
        const double L = log(T / k_c);
        const double ha = (4.0 / 3.0) * (L - (T - k_c) / E) + 0.5 * (T - k_c) * (T + k_c) / (E * E);
        const double hb = L - (T - k_c) / E;
        *hard = c * (SA * ha + S1 * hb / 9.0);
    } else {
        *hard = 0.0;
    }
}

// Hard Moller cross-section per gram, knock-on fraction in [t_c/T, 1/2].
__device__ double moller_hard(const MatDev &m, double T, double t_c) {
    if (T <= 2.0 * t_c) return 0.0;
    const double g = T / kMC2 + 1.0, b2 = 1.0 - 1.0 / (g * g);
    const double e = t_c / T;
    const double cA = (g - 1.0) * (g - 1.0) / (g * g);
    const double cB = (2.0 * g - 1.0) / (g * g);
    const double br = 1.0 / e - 1.0 / (1.0 - e) + cA * (0.5 - e) - cB * log((1.0 - e) / e);
    return electrons_per_gram(m) * 2.0 * kPI * kRE * kRE * kMC2 / (b2 * T) * br;
}

// First transport cross-section per gram of the screened Rutherford
// cross-section with Moliere screening (stands in for §II.B.2's q_SR data).
__device__ double ms_l1inv(const MatDev &m, double T) {
    const double pc2 = T * (T + 2.0 * kMC2);
    const double g = T / kMC2 + 1.0, b2 = 1.0 - 1.0 / (g * g);
    double s = 0.0;
    for (int j = 0; j < m.n; ++j) {
        const double z = m.Z[j];
        const double az = kALPHA * z;
        const double eta = kALPHA * kALPHA * cbrt(z * z) / (4.0 * 0.885 * 0.885) * (kMC2 * kMC2 / pc2) *
                           (1.13 + 3.76 * az * az / b2);
        const double K = z * (z + 1.0) * kRE * kRE * kMC2 * kMC2 / (b2 * pc2);
        s += m.N[j] * 2.0 * kPI * K * (log1p(1.0 / eta) - 1.0 / (1.0 + eta));
    }
    return s;
}

// <mu> for f(mu) ~ (mu + a)^-2 on [0, 1], and its derivative in ln a.
__device__ void ms_mean(double a, double *h, double *dh_dlna) {
    if (a < 2.0e3) {
        const double L = log1p(1.0 / a);
        *h = a * (1.0 + a) * L - a;
        *dh_dlna = a * ((1.0 + 2.0 * a) * L - 2.0);
    } else {
        const double x = 1.0 / a;  // h = 1/2 - x/6 + x^2/12 - x^3/20 + x^4/30 - x^5/42
        *h = 0.5 - x * (1.0 / 6.0 - x * (1.0 / 12.0 - x * (1.0 / 20.0 - x * (1.0 / 30.0 - x / 42.0))));
        *dh_dlna = x * (1.0 / 6.0 - x * (2.0 / 12.0 - x * (3.0 / 20.0 - x * (4.0 / 30.0 - 5.0 * x / 42.0))));
    }
}

// ln a such that <mu> = (1 - exp(-G1))/2: safeguarded Newton in ln a.
__device__ double ms_solve_ln_a(double g1) {
    const double target = -0.5 * expm1(-g1);
    double lo = -90.0, hi = 40.0, x = log(fmax(g1, 1e-30));
    for (int it = 0; it < 200; ++it) {
        if (!(x > lo && x < hi)) x = 0.5 * (lo + hi);
        double h, dh;
        ms_mean(exp(x), &h, &dh);
        const double f = h - target;
        if (f < 0.0) lo = x; else hi = x;
        const double nx = x - f / dh;
        if (fabs(nx - x) < 1e-14 * fmax(1.0, fabs(x)) || hi - lo < 1e-14) { x = nx; break; }
        x = nx;
    }
    return x;
}

__global__ void k_build_tables(const MatDev *mats, int n_mat, double p0, double p1, double e0,
                               double e1, double t_c, double k_c, float *tab) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_ph = NMAT * G, n_el = NMAT * G;
    if (tid < n_ph) {
        const int m = tid / G, i = tid % G;
        float mt = 0.f, mc = 0.f, mp = 0.f;
        if (m < n_mat) {
            const double E = exp(log(p0) + (log(p1) - log(p0)) * i / (G - 1));
            double c, pe, pp;
            photon_mu(mats[m], E, &c, &pe, &pp);
            mt = (float)(c + pe + pp);
            mc = (float)c;
            mp = (float)pe;
        }
        tab[tab_ph(m) + 0 * G + i] = mt;
        tab[tab_ph(m) + 1 * G + i] = mc;
        tab[tab_ph(m) + 2 * G + i] = mp;
    } else if (tid < n_ph + n_el) {
        const int t = tid - n_ph;
        const int m = t / G, i = t % G;
        float L = 0.f, H = 0.f, B = 0.f, M = 0.f;
        if (m < n_mat) {
            const double T = exp(log(e0) + (log(e1) - log(e0)) * i / (G - 1));
            double soft, hard;
            brem_parts(mats[m], T, k_c, &soft, &hard);
            L = (float)(collision_loss(mats[m], T, t_c) + soft);
            B = (float)hard;
            H = (float)(hard + moller_hard(mats[m], T, t_c));
            M = (float)ms_l1inv(mats[m], T);
        }
        tab[tab_el(m) + 0 * G + i] = L;
        tab[tab_el(m) + 1 * G + i] = H;
        tab[tab_el(m) + 2 * G + i] = B;
        tab[tab_el(m) + 3 * G + i] = M;
    } else if (tid < n_ph + n_el + G_MS) {
        const int i = tid - n_ph - n_el;
        const double lg = log(MS_G_MIN) + (log(MS_G_MAX) - log(MS_G_MIN)) * i / (G_MS - 1);
        tab[TAB_MS + i] = (float)ms_solve_ln_a(exp(lg));
    } else if (tid < n_ph + n_el + G_MS + NMAT) {
        const int m = tid - n_ph - n_el - G_MS;
        float ca = 0.f, c1 = 0.f;
        if (m < n_mat) {
            double SA, S1;
            brem_sums(mats[m], &SA, &S1);
            const double g0 = (4.0 / 3.0) * SA + S1 / 9.0;  // shape at y = 0, its maximum
            ca = (float)(SA / g0);
            c1 = (float)(S1 / (9.0 * g0));
        }
        tab[TAB_BREM + 2 * m] = ca;
        tab[TAB_BREM + 2 * m + 1] = c1;
    }
}

// Grid energies, for the diagnostics.
__global__ void k_grid_energies(double p0, double p1, double e0, double e1, float *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < G) out[i] = (float)exp(log(p0) + (log(p1) - log(p0)) * i / (G - 1));
    else if (i < 2 * G) out[i] = (float)exp(log(e0) + (log(e1) - log(e0)) * (i - G) / (G - 1));
}

// Voxel words: material id in bits 0-3, density in units of 2^-24 g/cm^3 in
// bits 4-31.  rho_max per material via integer max of positive float bits:
// reduced in the warp, then in the CTA's shared memory, then one global
// atomic per material and CTA.
__global__ void k_pack_phantom(const uint8_t *mat, const float *rho, uint64_t nvox, int n_mat,
                               uint32_t *vox, unsigned int *rho_max_bits, int *bad) {
    __shared__ unsigned int smax[NMAT];
    __shared__ int sbad;
    for (int i = threadIdx.x; i < NMAT; i += blockDim.x) smax[i] = 0u;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < nvox;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const int m = mat[v];
        const float r = rho[v];
        if (m >= n_mat || !(r > 0.f) || !(r < 16.f)) {
            sbad = 1;
            vox[v] = 0;
            continue;
        }
        uint32_t rq = __float2uint_rn(r * 16777216.0f);
        if (rq == 0) rq = 1;
        if (rq >= (1u << 28)) rq = (1u << 28) - 1;
        vox[v] = (rq << 4) | (uint32_t)m;
        // one shared-memory atomic per distinct material in the warp
        const unsigned bits = __float_as_uint(__uint2float_rn(rq) * kRhoQ);
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, m);
        const unsigned mx = __reduce_max_sync(peers, bits);
        if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicMax(&smax[m], mx);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_mat && i < NMAT; i += blockDim.x)
        if (smax[i]) atomicMax(&rho_max_bits[i], smax[i]);
    if (threadIdx.x == 0 && sbad) atomicExch(bad, 1);
}

// Majorants of one phantom (GPUMCD §II.A mu_max; §II.B.3 electron Woodcock):
// photon: max_m rho_max,m mu_m(E) per grid point; electron: running maximum
// over the grid of max_m rho_max,m Sigma_hard,m(T), so that the value at T
// bounds the hard cross-section at every energy an electron passes below T.
// One thread per grid point (a block of G threads); the running maximum is an
// inclusive prefix maximum, in the warp by shuffles and then across warps.
__global__ void k_majorants(const float *tab, const unsigned int *rho_max_bits, int n_mat, float *maj) {
    __shared__ float wmax[G / 32];
    const int i = threadIdx.x;
    if (i >= G) return;
    float mp = 0.f, me = 0.f;
    for (int m = 0; m < n_mat; ++m) {
        const float r = __uint_as_float(rho_max_bits[m]);
        if (r <= 0.f) continue;
        mp = fmaxf(mp, r * tab[tab_ph(m) + i]);
        me = fmaxf(me, r * tab[tab_el(m) + 1 * G + i]);
    }
    maj[i] = mp;
    const int lane = i & 31, w = i >> 5;
    float run = me;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const float o = __shfl_up_sync(0xffffffffu, run, d);
        if (lane >= d) run = fmaxf(run, o);
    }
    if (lane == 31) wmax[w] = run;
    __syncthreads();
    float base = 0.f;
    for (int k = 0; k < w; ++k) base = fmaxf(base, wmax[k]);
    maj[G + i] = fmaxf(base, run);
}

// Spectrum: FP64 prefix sum of the weights into a normalised CDF (the
// inverse-CDF table), stored with the bin edges as floats.
__global__ void k_spectrum(const double *edges, const double *w, int n, float *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double tot = 0.0;
    for (int i = 0; i < n; ++i) tot += w[i];
    double acc = 0.0;
    out[0] = 0.f;
    for (int i = 0; i < n; ++i) {
        acc += w[i];
        out[i + 1] = (float)(acc / tot);
    }
    out[n] = 1.f;
    for (int i = 0; i <= n; ++i) out[n + 1 + i] = (float)edges[i];
}

// Fold of a plan's batch tallies (GPUMCD §II.D): mean dose per history and
// the standard error of the mean from the W batch sums S_b (n_b histories
// each), in FP64:
//   D = sum_b S_b / N,   var(D) = W / ((W - 1) N^2) sum_b (S_b - n_b D)^2
// (the batch-mean estimator; it reduces to sum (d_b - D)^2 / (W (W - 1)) for
// equal batches).  The sum over batches is an exact integer; the per-voxel
// integer sums are also added into the plan's deposited-energy ledger.
struct FoldArgs {
    double n_b[64];
};

// Per-voxel arithmetic of the fold with per-batch history counts n_b: the
// mean energy per history and the batch-mean variance, scaled to Gy.
template <int W>
__device__ __forceinline__ void fold_voxel(const unsigned long long *tally, const uint32_t *vox, uint64_t nvox,
                                           uint64_t v, const FoldArgs &fa, double n_tot, double inv_vol,
                                           double &dv, double &sv, unsigned long long &tot_out) {
    unsigned long long s[W];
    unsigned long long tot = 0;
#pragma unroll
    for (int b = 0; b < W; ++b) {
        s[b] = __ldcs(tally + (uint64_t)b * nvox + v);
        tot += s[b];
    }
    const double mean = (double)tot / n_tot;
    double acc = 0.0;
#pragma unroll
    for (int b = 0; b < W; ++b) {
        const double t = fma(-fa.n_b[b], mean, (double)s[b]);
        acc = fma(t, t, acc);
    }
    const double var = acc * ((double)W / ((double)(W - 1) * n_tot * n_tot));
    const double rho = (double)(vox[v] >> 4) * (double)kRhoQ;
    const double scale = kQ * kMeVPerGramToGy * inv_vol / rho;
    dv = mean * scale;
    sv = sqrt(var) * scale;
    tot_out = tot;
}

template <int W>
__global__ void k_fold(const unsigned long long *tally, const uint32_t *vox, uint64_t nvox,
                       const __grid_constant__ FoldArgs fa, double n_tot, double inv_vol, double *dose,
                       double *sigma, unsigned long long *dmax_bits, unsigned long long *dep_sum) {
    double local_max = 0.0;
    unsigned long long local_sum = 0;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < nvox;
         v += (uint64_t)gridDim.x * blockDim.x) {
        double dv, sv;
        unsigned long long tot;
        fold_voxel<W>(tally, vox, nvox, v, fa, n_tot, inv_vol, dv, sv, tot);
        if (dose) dose[v] = dv;
        if (sigma) sigma[v] = sv;
        local_max = fmax(local_max, dv);
        local_sum += tot;
    }
    for (int o = 16; o > 0; o >>= 1) {
        local_max = fmax(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
        local_sum += __shfl_xor_sync(0xffffffffu, local_sum, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(dmax_bits, (unsigned long long)__double_as_longlong(local_max));
        if (local_sum) atomicAdd(dep_sum, local_sum);
    }
}

// The same fold for equal batches (n_b = N / W for every b): the variance
// numerator is formed exactly in 128-bit integers,
//   sum_b (S_b - S/W)^2 = (W sum_b S_b^2 - S^2) / W,
// so only one conversion to FP64 per voxel remains (FP64 is scarce on GB300
// and the per-batch FP64 work of k_fold bounds it).  A voxel whose sums would
// not fit 128 bits (sum S_b^2 >= 2^121, far beyond realistic tallies) takes
// the FP64 two-pass form instead.
struct U128 {
    unsigned long long lo, hi;
};

__device__ __forceinline__ void add_sq(U128 &acc, unsigned long long x) {
    const unsigned long long lo = x * x, hi = __umul64hi(x, x);
    const unsigned long long nl = acc.lo + lo;
    acc.hi += hi + (nl < lo ? 1ull : 0ull);
    acc.lo = nl;
}

__device__ __forceinline__ double u128_to_double(U128 v) {
    return (double)v.hi * 18446744073709551616.0 + (double)v.lo;
}

// FP64 is scarce on GB300, so the per-voxel FP64 work is one division (by
// the voxel's density code, shared by dose and sigma) and one square root;
// the other divisors are loop constants whose reciprocals come from the host.
struct FoldConst {
    double inv_n;   // 1 / N
    double c_var;   // 1 / (W^2 (W - 1) n^2), n = N / W
    double k_dose;  // q * (MeV/g -> Gy) / (voxel volume * density quantum)
};

// Per-voxel arithmetic of the equal-batch fold.
template <int W>
__device__ __forceinline__ void fold_voxel_equal(const unsigned long long *tally, const uint32_t *vox,
                                                 uint64_t nvox, uint64_t v, const FoldConst &fc, double &dv,
                                                 double &sv, unsigned long long &tot_out) {
    unsigned long long s[W];
    unsigned long long tot = 0;
    U128 sq{0ull, 0ull};
#pragma unroll
    for (int b = 0; b < W; ++b) {
        s[b] = __ldcs(tally + (uint64_t)b * nvox + v);
        tot += s[b];
        add_sq(sq, s[b]);
    }
    double var_sum;  // sum_b (S_b - S/W)^2, in quanta^2
    if (sq.hi < (1ull << 57)) {
        // W sum S_b^2 - S^2, exact and non-negative (Cauchy-Schwarz), = W var_sum
        const U128 ws{sq.lo * (unsigned long long)W, sq.hi * (unsigned long long)W + __umul64hi(sq.lo, (unsigned long long)W)};
        const U128 t2{tot * tot, __umul64hi(tot, tot)};
        const U128 num{ws.lo - t2.lo, ws.hi - t2.hi - (ws.lo < t2.lo ? 1ull : 0ull)};
        var_sum = u128_to_double(num) * (1.0 / (double)W);
    } else {
        const double m = (double)tot * (1.0 / (double)W);
        double acc = 0.0;
        for (int b = 0; b < W; ++b) {
            const double t = (double)s[b] - m;
            acc = fma(t, t, acc);
        }
        var_sum = acc;
    }
    // var(D) = var_sum / (W (W - 1) n^2) in quanta^2 per history^2
    const double r = fc.k_dose / (double)(vox[v] >> 4);
    dv = (double)tot * fc.inv_n * r;
    sv = sqrt(var_sum * ((double)W * fc.c_var)) * r;
    tot_out = tot;
}

template <int W>
__global__ void k_fold_equal(const unsigned long long *tally, const uint32_t *vox, uint64_t nvox, FoldConst fc,
                             double *dose, double *sigma, unsigned long long *dmax_bits,
                             unsigned long long *dep_sum) {
    double local_max = 0.0;
    unsigned long long local_sum = 0;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < nvox;
         v += (uint64_t)gridDim.x * blockDim.x) {
        double dv, sv;
        unsigned long long tot;
        fold_voxel_equal<W>(tally, vox, nvox, v, fc, dv, sv, tot);
        if (dose) dose[v] = dv;
        if (sigma) sigma[v] = sv;
        local_max = fmax(local_max, dv);
        local_sum += tot;
    }
    for (int o = 16; o > 0; o >>= 1) {
        local_max = fmax(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
        local_sum += __shfl_xor_sync(0xffffffffu, local_sum, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(dmax_bits, (unsigned long long)__double_as_longlong(local_max));
        if (local_sum) atomicAdd(dep_sum, local_sum);
    }
}

// s_thr = mean of sigma/D over voxels with D > thr * D_max (GPUMCD §II.D, s).
// Each block writes its partial sum and count to its own slot; one block then
// adds the slots in a fixed order, so s_thr is the same bit for bit for the
// same tally (the run-to-uncertainty schedule depends on it).
constexpr int kSthrThreads = 256;

__global__ void __launch_bounds__(kSthrThreads) k_sthr(const double *dose, const double *sigma, uint64_t nvox,
                                                       const unsigned long long *dmax_bits, double thr,
                                                       double2 *part) {
    __shared__ double ss[kSthrThreads / 32];
    __shared__ double sc[kSthrThreads / 32];
    const double cut = thr * __longlong_as_double((long long)*dmax_bits);
    double s = 0.0;
    unsigned long long c = 0;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < nvox;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const double d = dose[v];
        if (d > cut && d > 0.0) {
            s += sigma[v] / d;
            ++c;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        sc[threadIdx.x >> 5] = (double)c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < kSthrThreads / 32; ++i) {
            a += ss[i];
            b += sc[i];
        }
        part[blockIdx.x] = make_double2(a, b);
    }
}

__global__ void __launch_bounds__(kSthrThreads) k_sthr_combine(const double2 *part, int n, double *sum,
                                                               unsigned long long *count) {
    __shared__ double ss[kSthrThreads];
    __shared__ double sc[kSthrThreads];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += kSthrThreads) {
        a += part[i].x;
        b += part[i].y;
    }
    ss[threadIdx.x] = a;
    sc[threadIdx.x] = b;
    __syncthreads();
    for (int w = kSthrThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            ss[threadIdx.x] += ss[threadIdx.x + w];
            sc[threadIdx.x] += sc[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *sum = ss[0];
        *count = (unsigned long long)sc[0];
    }
}

// Exact integer sum of a tally (for the energy ledger).
__global__ void k_sum_u64(const unsigned long long *a, uint64_t n, unsigned long long *out) {
    unsigned long long s = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        s += a[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

__global__ void k_philox(const uint4 *ctr, uint2 key, uint64_t n, uint4 *out) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], key);
}

// cuRAND's Philox4_32_10 started at counter c: the generator's counter is
// (offset/4 low, offset/4 high, subsequence low, subsequence high), so
// c = (x, y, z, w) is reached with subsequence = w:z and offset = 4 (y:x).
__global__ void k_curand_philox(const uint4 *ctr, uint2 key, uint64_t n, uint4 *out) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = ctr[i];
    curandStatePhilox4_32_10_t st;
    const unsigned long long seed = ((unsigned long long)key.y << 32) | key.x;
    const unsigned long long sub = ((unsigned long long)c.w << 32) | c.z;
    const unsigned long long off = (((unsigned long long)c.y << 32) | c.x) * 4ull;
    curand_init(seed, sub, off, &st);
    out[i] = curand4(&st);
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
cudaError_t launch_build_tables(const gpumcd_material *mats, int n_mat, const TableGeom &g,
                                double t_c, double k_c, float *d_tab, cudaStream_t s) {
    MatDev h[NMAT];
    for (int m = 0; m < n_mat; ++m) {
        double wsum = 0.0;
        for (int j = 0; j < mats[m].n_elements; ++j) wsum += mats[m].w[j];
        h[m].n = mats[m].n_elements;
        for (int j = 0; j < h[m].n; ++j) {
            h[m].Z[j] = mats[m].Z[j];
            h[m].N[j] = kNA * (mats[m].w[j] / wsum) / mats[m].A[j];
        }
        h[m].I_mc2 = mats[m].I_eV * 1e-6 / kMC2;
    }
    MatDev *d = nullptr;
    cudaError_t e = cudaMallocAsync(&d, sizeof(MatDev) * NMAT, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(d, h, sizeof(MatDev) * n_mat, cudaMemcpyHostToDevice, s);
    const int total = NMAT * G * 2 + G_MS + NMAT;
    if (e == cudaSuccess) {
        k_build_tables<<<(total + 127) / 128, 128, 0, s>>>(d, n_mat, g.p0, g.p1, g.e0, g.e1, t_c, k_c, d_tab);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaFreeAsync(d, s);
    return e != cudaSuccess ? e : e2;
}

cudaError_t launch_grid_energies(const TableGeom &g, float *out, cudaStream_t s) {
    k_grid_energies<<<(2 * G + 127) / 128, 128, 0, s>>>(g.p0, g.p1, g.e0, g.e1, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_phantom(const uint8_t *mat, const float *rho, uint64_t nvox, int n_mat,
                                uint32_t *vox, unsigned int *rho_max_bits, int *bad, cudaStream_t s) {
    const int grid = (int)((nvox + 255) / 256 < 1024 ? (nvox + 255) / 256 : 1024);
    k_pack_phantom<<<grid > 0 ? grid : 1, 256, 0, s>>>(mat, rho, nvox, n_mat, vox, rho_max_bits, bad);
    return cudaGetLastError();
}

cudaError_t launch_majorants(const float *tab, const unsigned int *rho_max_bits, int n_mat, float *maj,
                             cudaStream_t s) {
    static_assert(G % 32 == 0 && G <= 1024, "one thread per grid point in one block");
    k_majorants<<<1, G, 0, s>>>(tab, rho_max_bits, n_mat, maj);
    return cudaGetLastError();
}

cudaError_t launch_spectrum(const double *edges, const double *w, int n, float *out, cudaStream_t s) {
    k_spectrum<<<1, 32, 0, s>>>(edges, w, n, out);
    return cudaGetLastError();
}

// Host side of both folds: the per-batch history counts and whether they are
// all equal (the integer-variance form), and the constants of that form.
static bool fold_args(int W, const double *n_b, FoldArgs &fa) {
    bool equal = true;
    for (int b = 0; b < 64; ++b) {
        fa.n_b[b] = b < W ? n_b[b] : 0.0;
        if (b < W && n_b[b] != n_b[0]) equal = false;
    }
    return equal;
}

static FoldConst fold_const(int W, double n_tot, double inv_vol) {
    FoldConst fc;
    const double n = n_tot / (double)W;
    fc.inv_n = 1.0 / n_tot;
    fc.c_var = 1.0 / ((double)W * (double)W * (double)(W - 1) * n * n);
    fc.k_dose = kQ * kMeVPerGramToGy * inv_vol / kRhoQ;
    return fc;
}

cudaError_t launch_fold(const unsigned long long *tally, const uint32_t *vox, uint64_t nvox, int W,
                        const double *n_b, double n_tot, double inv_vol, double *dose, double *sigma,
                        unsigned long long *dmax_bits, unsigned long long *dep_sum, int n_sm, cudaStream_t s) {
    FoldArgs fa;
    const bool equal = fold_args(W, n_b, fa);
    uint64_t blocks = (nvox + 255) / 256;
    const uint64_t cap = (uint64_t)n_sm * 8;
    const int grid = (int)(blocks < cap ? (blocks ? blocks : 1) : cap);
    if (equal) {
        const FoldConst fc = fold_const(W, n_tot, inv_vol);
        switch (W) {
            case 8: k_fold_equal<8><<<grid, 256, 0, s>>>(tally, vox, nvox, fc, dose, sigma, dmax_bits, dep_sum); break;
            case 16: k_fold_equal<16><<<grid, 256, 0, s>>>(tally, vox, nvox, fc, dose, sigma, dmax_bits, dep_sum); break;
            case 32: k_fold_equal<32><<<grid, 256, 0, s>>>(tally, vox, nvox, fc, dose, sigma, dmax_bits, dep_sum); break;
            case 64: k_fold_equal<64><<<grid, 256, 0, s>>>(tally, vox, nvox, fc, dose, sigma, dmax_bits, dep_sum); break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (W) {
        case 8: k_fold<8><<<grid, 256, 0, s>>>(tally, vox, nvox, fa, n_tot, inv_vol, dose, sigma, dmax_bits, dep_sum); break;
        case 16: k_fold<16><<<grid, 256, 0, s>>>(tally, vox, nvox, fa, n_tot, inv_vol, dose, sigma, dmax_bits, dep_sum); break;
        case 32: k_fold<32><<<grid, 256, 0, s>>>(tally, vox, nvox, fa, n_tot, inv_vol, dose, sigma, dmax_bits, dep_sum); break;
        case 64: k_fold<64><<<grid, 128, 0, s>>>(tally, vox, nvox, fa, n_tot, inv_vol, dose, sigma, dmax_bits, dep_sum); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int sthr_blocks(uint64_t nvox, int n_sm) {
    const uint64_t blocks = (nvox + kSthrThreads - 1) / kSthrThreads;
    const uint64_t cap = (uint64_t)n_sm * 8;
    return (int)(blocks < cap ? (blocks ? blocks : 1) : cap);
}

cudaError_t launch_sthr(const double *dose, const double *sigma, uint64_t nvox,
                        const unsigned long long *dmax_bits, double thr, double *sum,
                        unsigned long long *count, void *part, int n_sm, cudaStream_t s) {
    const int grid = sthr_blocks(nvox, n_sm);
    k_sthr<<<grid, kSthrThreads, 0, s>>>(dose, sigma, nvox, dmax_bits, thr, (double2 *)part);
    k_sthr_combine<<<1, kSthrThreads, 0, s>>>((const double2 *)part, grid, sum, count);
    return cudaGetLastError();
}

cudaError_t launch_sum_u64(const unsigned long long *a, uint64_t n, unsigned long long *out, int n_sm,
                           cudaStream_t s) {
    uint64_t blocks = (n + 255) / 256;
    const uint64_t cap = (uint64_t)n_sm * 8;
    k_sum_u64<<<(int)(blocks < cap ? (blocks ? blocks : 1) : cap), 256, 0, s>>>(a, n, out);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t *ctr, uint2 key, uint64_t n, int curand, uint32_t *out,
                          cudaStream_t s) {
    const int grid = (int)((n + 127) / 128);
    if (curand)
        k_curand_philox<<<grid ? grid : 1, 128, 0, s>>>((const uint4 *)ctr, key, n, (uint4 *)out);
    else
        k_philox<<<grid ? grid : 1, 128, 0, s>>>((const uint4 *)ctr, key, n, (uint4 *)out);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Allocation-free fold (gpumcd_plan_result_noalloc).
//
// The same dose / uncertainty fold as k_fold and k_fold_equal (the same
// per-voxel functions), with its reduction scratch in a
// file-scope device array instead of device memory allocated at run time.
// Each block folds one fixed range of voxels and writes its partial results
// to its own slots of the array; single-block kernels then combine the
// partials in a fixed order.  Every call rewrites the slots it reads, so
// nothing needs clearing; calls that overlap on the GPU share the array and
// race.
// ---------------------------------------------------------------------------
namespace noalloc {

constexpr int kThreads = 256;
constexpr int kVoxPerThread = 64;
constexpr uint64_t kVoxPerBlock = (uint64_t)kThreads * kVoxPerThread;
constexpr int kMaxBlocks = GPUMCD_NOALLOC_MAX_VOXELS / (kThreads * kVoxPerThread);
static_assert((uint64_t)kMaxBlocks * kVoxPerBlock == GPUMCD_NOALLOC_MAX_VOXELS, "exact block count");

// [kMaxBlocks][4] partials (max dose bits, deposited energy, sum sigma/D,
// count) followed by 4 result words (D_max bits, deposited, s_thr bits, count).
static __device__ __align__(256) unsigned long long scratch[kMaxBlocks * 4 + 4];

// EQUAL selects the integer-variance form of k_fold_equal, else the form of
// k_fold: the per-voxel arithmetic is the same function as the regular
// fold's, so dose and sigma match gpumcd_plan_result's bit for bit.
template <int W, bool EQUAL>
__global__ void __launch_bounds__(kThreads) k_fold_blocks(const unsigned long long *tally, const uint32_t *vox,
                                                          uint64_t nvox, const __grid_constant__ FoldArgs fa,
                                                          FoldConst fc, double n_tot, double inv_vol, double *dose,
                                                          double *sigma, unsigned long long *part) {
    __shared__ double smax[kThreads / 32];
    __shared__ unsigned long long ssum[kThreads / 32];
    const uint64_t v0 = blockIdx.x * kVoxPerBlock;
    double local_max = 0.0;
    unsigned long long local_sum = 0;
    for (int k = 0; k < kVoxPerThread; ++k) {
        const uint64_t v = v0 + (uint64_t)k * kThreads + threadIdx.x;
        if (v >= nvox) break;
        double dv, sv;
        unsigned long long tot;
        if (EQUAL)
            fold_voxel_equal<W>(tally, vox, nvox, v, fc, dv, sv, tot);
        else
            fold_voxel<W>(tally, vox, nvox, v, fa, n_tot, inv_vol, dv, sv, tot);
        dose[v] = dv;
        sigma[v] = sv;
        local_max = fmax(local_max, dv);
        local_sum += tot;
    }
    for (int o = 16; o > 0; o >>= 1) {
        local_max = fmax(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
        local_sum += __shfl_xor_sync(0xffffffffu, local_sum, o);
    }
    if ((threadIdx.x & 31) == 0) {
        smax[threadIdx.x >> 5] = local_max;
        ssum[threadIdx.x >> 5] = local_sum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        unsigned long long t = 0;
        for (int i = 0; i < kThreads / 32; ++i) {
            m = fmax(m, smax[i]);
            t += ssum[i];
        }
        part[4 * blockIdx.x + 0] = (unsigned long long)__double_as_longlong(m);
        part[4 * blockIdx.x + 1] = t;
    }
}

// Combine the per-block maxima and deposits (one block, fixed order).
__global__ void k_combine_max(unsigned long long *part, int n_blocks) {
    __shared__ double smax[kThreads];
    __shared__ unsigned long long ssum[kThreads];
    double m = 0.0;
    unsigned long long t = 0;
    for (int b = threadIdx.x; b < n_blocks; b += kThreads) {
        m = fmax(m, __longlong_as_double((long long)part[4 * b + 0]));
        t += part[4 * b + 1];
    }
    smax[threadIdx.x] = m;
    ssum[threadIdx.x] = t;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + w]);
            ssum[threadIdx.x] += ssum[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[4 * kMaxBlocks + 0] = (unsigned long long)__double_as_longlong(smax[0]);
        part[4 * kMaxBlocks + 1] = ssum[0];
    }
}

// Per-block sums of sigma/D over voxels above thr * D_max.
__global__ void k_sthr_blocks(const double *dose, const double *sigma, uint64_t nvox, double thr,
                              unsigned long long *part) {
    __shared__ double ss[kThreads / 32];
    __shared__ unsigned long long sc[kThreads / 32];
    const double cut = thr * __longlong_as_double((long long)part[4 * kMaxBlocks + 0]);
    const uint64_t v0 = blockIdx.x * kVoxPerBlock;
    double s = 0.0;
    unsigned long long c = 0;
    for (int k = 0; k < kVoxPerThread; ++k) {
        const uint64_t v = v0 + (uint64_t)k * kThreads + threadIdx.x;
        if (v >= nvox) break;
        const double d = dose[v];
        if (d > cut && d > 0.0) {
            s += sigma[v] / d;
            ++c;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        sc[threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        unsigned long long b = 0;
        for (int i = 0; i < kThreads / 32; ++i) {
            a += ss[i];
            b += sc[i];
        }
        part[4 * blockIdx.x + 2] = (unsigned long long)__double_as_longlong(a);
        part[4 * blockIdx.x + 3] = b;
    }
}

__global__ void k_combine_sthr(unsigned long long *part, int n_blocks) {
    __shared__ double ss[kThreads];
    __shared__ unsigned long long sc[kThreads];
    double s = 0.0;
    unsigned long long c = 0;
    for (int b = threadIdx.x; b < n_blocks; b += kThreads) {
        s += __longlong_as_double((long long)part[4 * b + 2]);
        c += part[4 * b + 3];
    }
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            ss[threadIdx.x] += ss[threadIdx.x + w];
            sc[threadIdx.x] += sc[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sthr = sc[0] ? ss[0] / (double)sc[0] : 0.0;
        part[4 * kMaxBlocks + 2] = (unsigned long long)__double_as_longlong(sthr);
        part[4 * kMaxBlocks + 3] = sc[0];
    }
}

}  // namespace noalloc

// The address of the scratch array on `device`, looked up once per device
// with that device current.  In host code the array's name is only a host-side
// stand-in, so kernels must be given this address instead.  Host threads may
// make their first calls at the same time, so the lookup is done under a lock.
static unsigned long long *noalloc_scratch(int device, cudaError_t *err) {
    static std::mutex mu;
    static unsigned long long *addr[64] = {nullptr};
    if (device < 0 || device >= 64) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, noalloc::scratch);
        if (e != cudaSuccess) {
            *err = e;
            return nullptr;
        }
        if (!p) {
            *err = cudaErrorInvalidDevicePointer;
            return nullptr;
        }
        addr[device] = (unsigned long long *)p;
    }
    *err = cudaSuccess;
    return addr[device];
}

template <int W>
static void launch_fold_blocks(bool equal, int nb, cudaStream_t s, const unsigned long long *tally,
                               const uint32_t *vox, uint64_t nvox, const FoldArgs &fa, const FoldConst &fc,
                               double n_tot, double inv_vol, double *dose, double *sigma, unsigned long long *part) {
    using namespace noalloc;
    if (equal)
        k_fold_blocks<W, true><<<nb, kThreads, 0, s>>>(tally, vox, nvox, fa, fc, n_tot, inv_vol, dose, sigma, part);
    else
        k_fold_blocks<W, false><<<nb, kThreads, 0, s>>>(tally, vox, nvox, fa, fc, n_tot, inv_vol, dose, sigma, part);
}

cudaError_t launch_fold_noalloc(int device, const unsigned long long *tally, const uint32_t *vox, uint64_t nvox,
                                int W, const double *n_b, double n_tot, double inv_vol, double thr, double *dose,
                                double *sigma, cudaStream_t s, unsigned long long result[4]) {
    cudaError_t e = cudaSuccess;
    unsigned long long *part = noalloc_scratch(device, &e);
    if (!part) return e != cudaSuccess ? e : cudaErrorInvalidDevicePointer;
    FoldArgs fa;
    const bool equal = fold_args(W, n_b, fa);
    const FoldConst fc = fold_const(W, n_tot, inv_vol);
    const int nb = (int)((nvox + noalloc::kVoxPerBlock - 1) / noalloc::kVoxPerBlock);
    using namespace noalloc;
    switch (W) {
        case 8: launch_fold_blocks<8>(equal, nb, s, tally, vox, nvox, fa, fc, n_tot, inv_vol, dose, sigma, part); break;
        case 16: launch_fold_blocks<16>(equal, nb, s, tally, vox, nvox, fa, fc, n_tot, inv_vol, dose, sigma, part); break;
        case 32: launch_fold_blocks<32>(equal, nb, s, tally, vox, nvox, fa, fc, n_tot, inv_vol, dose, sigma, part); break;
        case 64: launch_fold_blocks<64>(equal, nb, s, tally, vox, nvox, fa, fc, n_tot, inv_vol, dose, sigma, part); break;
        default: return cudaErrorInvalidValue;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_combine_max<<<1, kThreads, 0, s>>>(part, nb);
    k_sthr_blocks<<<nb, kThreads, 0, s>>>(dose, sigma, nvox, thr, part);
    k_combine_sthr<<<1, kThreads, 0, s>>>(part, nb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = cudaMemcpyAsync(result, part + 4 * kMaxBlocks, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

}  // namespace gm
