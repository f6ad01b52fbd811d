/*
 * Oracle for the coupled photon-electron transport of GPUMCD (Hissoiny et al.).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded FP64 CPU
 * transport written to check the CUDA path.  Only the tests, the smoke check
 * and the CPU-baseline leg of bench.py may load it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Model (the same on both sides):
 *  - photons: analogue transport with Woodcock tracking (GPUMCD §II.A);
 *    Compton (Klein-Nishina, free electron), K-shell photoelectric with a
 *    Sauter photo-electron, pair production with no positrons and a uniform
 *    kinetic-energy split (§II.A).
 *  - electrons: Class II condensed history (§II.B): restricted CSDA loss,
 *    random-hinge multiple scattering, hard Moller and bremsstrahlung events
 *    found with electron Woodcock tracking against an energy-envelope majorant.
 *  - cross-sections are closed forms evaluated exactly at each energy; the
 *    oracle uses no tables.
 *
 * Parity status: every function below is pinned by a -m "not gpu" test against
 * mathematics or published values other than its own formula.  The identity of
 * the Philox generator with the published Philox4x32-10 is pinned on the GPU,
 * against cuRAND's generator.
 */
#ifndef GPUMCD_ORACLE_H
#define GPUMCD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OM_MAX_ELEMENTS 16
#define OM_MAX_MATERIALS 16

/* Physical constants (CODATA 2018). */
#define OM_MC2 0.51099895000          /* electron rest energy, MeV */
#define OM_RE 2.8179403262e-13        /* classical electron radius, cm */
#define OM_ALPHA (1.0 / 137.035999084)
#define OM_NA 6.02214076e23
#define OM_PI 3.14159265358979323846

typedef struct {
    int32_t n_el;
    int32_t Z[OM_MAX_ELEMENTS];
    double A[OM_MAX_ELEMENTS]; /* g/mol */
    double w[OM_MAX_ELEMENTS]; /* mass fractions, sum 1 */
    double I_eV;               /* mean excitation energy */
} om_material;

typedef struct {
    double p_cut, e_abs, t_c, k_c, estepe, e_max, nudge_cm;
} om_physics;

typedef struct {
    int32_t nx, ny, nz;
    double dx, dy, dz;
    const uint8_t *mat; /* nx*ny*nz, x fastest */
    const float *rho;   /* g/cm^3 */
} om_phantom;

typedef struct {
    int32_t particle; /* 0 photon, 1 electron */
    int32_t beam;     /* 0 pencil, 1 square field, 2 phase space */
    double energy;    /* MeV (mono) */
    int32_t n_spec;   /* >0: histogram spectrum with n_spec bins */
    const double *spec_edges;
    const double *spec_weights;
    double cx, cy, field;
    int32_t n_phsp;      /* beam 2: records */
    const double *phsp;  /* beam 2: [n_phsp][7] x, y, z (cm), ux, uy, uz, E (MeV) */
    /* Energy grouping (§IV) changes no sample here: a grouped spectrum or
     * phase space starts every history as an ungrouped one does (the GPU
     * orders the claims of its histories by energy, which leaves each
     * history's primary and draws unchanged), so the source has no flag. */
} om_source;

typedef struct {
    double e_incident, e_deposited, e_escaped, e_rest;
    double e_cut_photon, e_cut_electron; /* deposits made by the cut-offs (part of e_deposited) */
    double track_length_cm;              /* total electron path length */
    uint64_t n_histories;
    uint64_t n_photon_real, n_photon_fict;
    uint64_t n_compton, n_photo, n_pair;
    uint64_t n_e_steps, n_hard_real, n_hard_fict, n_moller, n_brem;
    uint64_t n_electrons, n_photons; /* particles transported (primaries + secondaries) */
} om_stats;

/* Flags for om_simulate (test modes). */
#define OM_FLAG_KERMA 1u           /* electrons deposit their energy where they are created */
#define OM_FLAG_FIRST_COLLISION 2u /* a photon's first real interaction ends it: the photon leaving it is escaped */
#define OM_FLAG_NO_MS 4u           /* electrons are not deflected */
/* The electron Woodcock majorant of a step is its own voxel's hard
 * cross-section at the start energy, rho0 Sigma_m0(T0) (Sigma_m rises with T,
 * and a step stays in its voxel), and the candidate is tested in that voxel;
 * without the flag, §II.B.3's majorant over the whole phantom, tested at the
 * end point.  Both are exact Woodcock schemes; they differ in how often a
 * fictitious candidate splits a step. */
#define OM_FLAG_VOXEL_EMAJOR 8u

/* ---- cross-sections and stopping powers (all mass quantities, cm^2/g or MeV cm^2/g) ---- */
double om_sigma_kn(double k);                              /* per electron, cm^2; k = E/mc^2 */
double om_kn_dsigma_domega(double k, double cos_t);        /* per electron, cm^2/sr */
double om_electron_density(const om_material *m);          /* electrons per gram */
double om_mu_compton(const om_material *m, double E);
double om_mu_photo(const om_material *m, double E);
double om_mu_pair(const om_material *m, double E);
double om_mu_total(const om_material *m, double E);
double om_l_col(const om_material *m, double T, double t_c);   /* restricted collision stopping power */
double om_s_col(const om_material *m, double T);               /* unrestricted */
double om_l_rad(const om_material *m, double T, double k_c);   /* soft radiative loss, photons below k_c */
double om_s_rad(const om_material *m, double T);               /* total radiative stopping power */
double om_sigma_moller(const om_material *m, double T, double t_c);
double om_moller_dsigma_deps(double T, double eps);            /* per electron, cm^2 per unit eps */
double om_sigma_brem(const om_material *m, double T, double k_c);
double om_brem_dsigma_dk(const om_material *m, double T, double k); /* cm^2/g per MeV */
double om_ms_lambda1_inv(const om_material *m, double T);      /* first transport cross-section, cm^2/g */
double om_ms_screening(int Z, double T);                       /* Moliere screening parameter eta */
double om_ms_mean_mu(double a);
double om_ms_solve_a(double g1);

/* ---- samplers (exact), for the distribution pins; n draws into out ---- */
void om_sample_kn(double k, int64_t n, uint64_t seed, double *cos_out, double *eps_out);
void om_sample_sauter(double T, int64_t n, uint64_t seed, double *cos_out);
void om_sample_moller(double T, double t_c, int64_t n, uint64_t seed, double *eps_out);
void om_sample_brem(const om_material *m, double T, double k_c, int64_t n, uint64_t seed, double *k_out);
void om_sample_ms(double g1, int64_t n, uint64_t seed, double *mu_out);
void om_sample_spectrum(int32_t n_bins, const double *edges, const double *weights, int64_t n,
                        uint64_t seed, double *e_out);
/* Primary energies of histories [hist_begin, hist_end) of a pencil or square
 * source, as the transport draws them (e_out[h - hist_begin]); -1 on invalid
 * input. */
int32_t om_primary_energies(const om_source *src, uint64_t hist_begin, uint64_t hist_end,
                            uint64_t seed, double *e_out);

/* ---- kinematics the transport uses, for the pins ---- */
/* out = u rotated by polar angle acos(c) and azimuth phi (a unit vector). */
void om_rotate(const double u[3], double c, double phi, double out[3]);
/* Compton scattering of a photon of energy E along u at (cos_t, phi) with
 * k'/k = eps: u1_out the photon's new direction, ue_out the recoil electron's,
 * out = {E', T}. */
void om_compton_kinematics(double E, const double u[3], double cos_t, double eps, double phi,
                           double u1_out[3], double ue_out[3], double out[2]);
/* Moller event of an electron of kinetic energy T with knock-on fraction eps:
 * out = {T_knock-on, T_scattered, cos_knock-on, cos_scattered}. */
void om_moller_kinematics(double T, double eps, double out[4]);

/* ---- RNG: Philox4x32-10 (Salmon et al., SC'11) ---- */
void om_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- transport ---- */
/* Simulates histories [hist_begin, hist_end).  sum_e / sum_e2 (nvox each,
 * accumulated into, MeV) receive the history-by-history first and second
 * moments of the energy deposited per voxel.  Returns 0, or a negative code
 * on invalid input (-1) or a violated majorant (-2). */
int32_t om_simulate(const om_material *mats, int32_t n_mat, const om_physics *phys,
                    const om_phantom *ph, const om_source *src, uint64_t hist_begin,
                    uint64_t hist_end, uint64_t seed, uint32_t flags, double *sum_e,
                    double *sum_e2, om_stats *stats);

/* Runs the Woodcock photon loop of om_simulate for n primaries of the source
 * and stores the z of each primary's first real interaction (or +inf when it
 * leaves the phantom first). */
int32_t om_first_interaction_z(const om_material *mats, int32_t n_mat, const om_physics *phys,
                               const om_phantom *ph, const om_source *src, int64_t n,
                               uint64_t seed, double *z_out, uint64_t *n_fict_out);

#ifdef __cplusplus
}
#endif
#endif
