/*
 * Oracle physics: closed-form cross-sections and stopping powers in FP64.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper takes its data from PEGS4/EGSnrc (GPUMCD §II.A-B), which is not
 * available here; every quantity below is a textbook closed form, evaluated at
 * the exact energy on every call.
 */
#include <math.h>

#include "oracle.h"

static double atoms_per_gram(const om_material *m, int j) { return OM_NA * m->w[j] / m->A[j]; }

double om_electron_density(const om_material *m) {
    double s = 0.0;
    for (int j = 0; j < m->n_el; ++j) s += atoms_per_gram(m, j) * m->Z[j];
    return s;
}

/* ------------------------------------------------------------------------
 * Photons (GPUMCD §II.A: mu = N_A/A rho (sigma_compton + sigma_photo + sigma_pair))
 * ------------------------------------------------------------------------ */

/* Klein-Nishina total cross-section per free electron (§II.A, Compton). */
double om_sigma_kn(double k) {
    double a = 1.0 + 2.0 * k;
    double l = log1p(2.0 * k); /* keeps the small-k cancellation accurate */
    double t1 = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - l / k);
    double t2 = l / (2.0 * k);
    double t3 = (1.0 + 3.0 * k) / (a * a);
    return 2.0 * OM_PI * OM_RE * OM_RE * (t1 + t2 - t3);
}

/* Klein-Nishina differential cross-section per electron per steradian. */
double om_kn_dsigma_domega(double k, double c) {
    double r = 1.0 / (1.0 + k * (1.0 - c)); /* k'/k */
    return 0.5 * OM_RE * OM_RE * r * r * (r + 1.0 / r - (1.0 - c * c));
}

double om_mu_compton(const om_material *m, double E) {
    return om_electron_density(m) * om_sigma_kn(E / OM_MC2);
}

/* K-shell photoelectric cross-section, Born (Heitler) form per atom:
 * 4 sqrt(2) alpha^4 Z^5 sigma_Thomson k^(-7/2) (§II.A, photoelectric effect;
 * the paper gives no cross-section form). */
double om_mu_photo(const om_material *m, double E) {
    double k = E / OM_MC2;
    double sigma_t = 8.0 * OM_PI / 3.0 * OM_RE * OM_RE;
    double a4 = OM_ALPHA * OM_ALPHA * OM_ALPHA * OM_ALPHA;
    double kfac = pow(k, -3.5);
    double s = 0.0;
    for (int j = 0; j < m->n_el; ++j) {
        double z = (double)m->Z[j];
        s += atoms_per_gram(m, j) * 4.0 * sqrt(2.0) * a4 * z * z * z * z * z * sigma_t * kfac;
    }
    return s;
}

/* Bethe-Heitler pair production with complete screening, times the threshold
 * factor (1 - 2mc^2/E)^3 (§II.A, pair production). */
double om_mu_pair(const om_material *m, double E) {
    if (E <= 2.0 * OM_MC2) return 0.0;
    double f = 1.0 - 2.0 * OM_MC2 / E;
    f = f * f * f;
    double s = 0.0;
    for (int j = 0; j < m->n_el; ++j) {
        double z = (double)m->Z[j];
        double bracket = (7.0 / 9.0) * log(183.0 * pow(z, -1.0 / 3.0)) - 1.0 / 54.0;
        s += atoms_per_gram(m, j) * 4.0 * OM_ALPHA * OM_RE * OM_RE * z * (z + 1.0) * bracket;
    }
    return s * f;
}

double om_mu_total(const om_material *m, double E) {
    return om_mu_compton(m, E) + om_mu_photo(m, E) + om_mu_pair(m, E);
}

/* ------------------------------------------------------------------------
 * Electrons (GPUMCD §II.B)
 * ------------------------------------------------------------------------ */

/* Restricted collision stopping power L(E, K_cut) of §II.B.3, in the
 * Bethe form with Moller close collisions (delta = 0):
 *   L/rho = 2 pi re^2 mc^2 (n_e/rho)/beta^2 [ln(2(tau+2)/(I/mc^2)^2) + F-(tau,Delta)]
 *   F- = -1 - beta^2 + ln((tau-Delta)Delta) + tau/(tau-Delta)
 *        + [Delta^2/2 + (2tau+1) ln(1 - Delta/tau)]/(tau+1)^2
 * with Delta = min(t_c, T/2)/mc^2; Delta = tau/2 gives the unrestricted value. */
double om_l_col(const om_material *m, double T, double t_c) {
    double tau = T / OM_MC2;
    double gam = tau + 1.0;
    double beta2 = 1.0 - 1.0 / (gam * gam);
    double cut = t_c < 0.5 * T ? t_c : 0.5 * T;
    double D = cut / OM_MC2;
    double iom = m->I_eV * 1e-6 / OM_MC2;
    double Fm = -1.0 - beta2 + log((tau - D) * D) + tau / (tau - D) +
                (0.5 * D * D + (2.0 * tau + 1.0) * log(1.0 - D / tau)) / (gam * gam);
    double br = log(2.0 * (tau + 2.0) / (iom * iom)) + Fm;
    return 2.0 * OM_PI * OM_RE * OM_RE * OM_MC2 * om_electron_density(m) / beta2 * br;
}

double om_s_col(const om_material *m, double T) { return om_l_col(m, T, T); }

/* Bethe-Heitler complete-screening bremsstrahlung, per atom:
 *   dsigma/dk = (4 alpha re^2 / k) Z(Z+1) {(4/3 - 4y/3 + y^2) ln(183 Z^-1/3) + (1-y)/9}
 * with y = k/E and E the electron's total energy.  Per material the two
 * element sums S_A = sum N_j Z(Z+1) ln(183 Z^-1/3) and S_1 = sum N_j Z(Z+1)
 * carry the composition. */
static void brem_sums(const om_material *m, double *SA, double *S1) {
    double a = 0.0, b = 0.0;
    for (int j = 0; j < m->n_el; ++j) {
        double z = (double)m->Z[j];
        double n = atoms_per_gram(m, j);
        a += n * z * (z + 1.0) * log(183.0 * pow(z, -1.0 / 3.0));
        b += n * z * (z + 1.0);
    }
    *SA = a;
    *S1 = b;
}

double om_brem_dsigma_dk(const om_material *m, double T, double k) {
    if (k <= 0.0 || k > T) return 0.0;
    double SA, S1;
    brem_sums(m, &SA, &S1);
    double E = T + OM_MC2;
    double y = k / E;
    return 4.0 * OM_ALPHA * OM_RE * OM_RE / k *
           ((4.0 / 3.0 - 4.0 * y / 3.0 + y * y) * SA + (1.0 - y) * S1 / 9.0);
}

/* Energy radiated per unit path by photons of energy below K:
 * integral_0^min(K,T) k dsigma/dk dk. */
static double rad_loss_below(const om_material *m, double T, double K) {
    if (K > T) K = T;
    if (K <= 0.0) return 0.0;
    double SA, S1;
    brem_sums(m, &SA, &S1);
    double E = T + OM_MC2;
    double ia = 4.0 * K / 3.0 - 2.0 * K * K / (3.0 * E) + K * K * K / (3.0 * E * E);
    double ib = K - K * K / (2.0 * E);
    return 4.0 * OM_ALPHA * OM_RE * OM_RE * (SA * ia + S1 * ib / 9.0);
}

double om_l_rad(const om_material *m, double T, double k_c) { return rad_loss_below(m, T, k_c); }
double om_s_rad(const om_material *m, double T) { return rad_loss_below(m, T, T); }

/* Hard bremsstrahlung cross-section, photons in [k_c, T] (§II.B.1). */
double om_sigma_brem(const om_material *m, double T, double k_c) {
    if (T <= k_c) return 0.0;
    double SA, S1;
    brem_sums(m, &SA, &S1);
    double E = T + OM_MC2;
    double L = log(T / k_c);
    double ia = (4.0 / 3.0) * L - (4.0 / 3.0) * (T - k_c) / E + (T * T - k_c * k_c) / (2.0 * E * E);
    double ib = L - (T - k_c) / E;
    return 4.0 * OM_ALPHA * OM_RE * OM_RE * (SA * ia + S1 * ib / 9.0);
}

/* Moller cross-section per electron, eps = T'/T (§II.B.1, inelastic collisions):
 *   dsigma/deps = (2 pi re^2 mc^2/(beta^2 T)) [1/eps^2 + 1/(1-eps)^2 + ((g-1)/g)^2
 *                 - ((2g-1)/g^2)/(eps(1-eps))]. */
double om_moller_dsigma_deps(double T, double eps) {
    double gam = T / OM_MC2 + 1.0;
    double beta2 = 1.0 - 1.0 / (gam * gam);
    double c1 = (gam - 1.0) / gam;
    c1 *= c1;
    double c2 = (2.0 * gam - 1.0) / (gam * gam);
    double pre = 2.0 * OM_PI * OM_RE * OM_RE * OM_MC2 / (beta2 * T);
    return pre * (1.0 / (eps * eps) + 1.0 / ((1.0 - eps) * (1.0 - eps)) + c1 -
                  c2 / (eps * (1.0 - eps)));
}

/* Hard Moller cross-section (knock-on above t_c), cm^2/g; zero for T <= 2 t_c. */
double om_sigma_moller(const om_material *m, double T, double t_c) {
    if (T <= 2.0 * t_c) return 0.0;
    double gam = T / OM_MC2 + 1.0;
    double beta2 = 1.0 - 1.0 / (gam * gam);
    double ec = t_c / T;
    double c1 = (gam - 1.0) / gam;
    c1 *= c1;
    double c2 = (2.0 * gam - 1.0) / (gam * gam);
    double pre = 2.0 * OM_PI * OM_RE * OM_RE * OM_MC2 / (beta2 * T);
    double s = 1.0 / ec - 1.0 / (1.0 - ec) + c1 * (0.5 - ec) - c2 * log((1.0 - ec) / ec);
    return om_electron_density(m) * pre * s;
}

/* Moliere screening parameter for a screened Rutherford cross-section. */
double om_ms_screening(int Z, double T) {
    double z = (double)Z;
    double pc2 = T * (T + 2.0 * OM_MC2);
    double gam = T / OM_MC2 + 1.0;
    double beta2 = 1.0 - 1.0 / (gam * gam);
    double az = OM_ALPHA * z;
    return OM_ALPHA * OM_ALPHA * pow(z, 2.0 / 3.0) / (4.0 * 0.885 * 0.885) * (OM_MC2 * OM_MC2 / pc2) *
           (1.13 + 3.76 * az * az / beta2);
}

/* First transport cross-section of the screened Rutherford (Wentzel)
 * cross-section, summed over elements:
 *   (1/lambda_1)/rho = sum_j N_j 2 pi Z(Z+1) re^2 (mc^2)^2/(beta^2 (pc)^2)
 *                      [ln(1 + 1/eta) - 1/(1 + eta)]
 * (stands in for the q_SR^{2+} data of §II.B.2, which are not available). */
double om_ms_lambda1_inv(const om_material *m, double T) {
    double pc2 = T * (T + 2.0 * OM_MC2);
    double gam = T / OM_MC2 + 1.0;
    double beta2 = 1.0 - 1.0 / (gam * gam);
    double s = 0.0;
    for (int j = 0; j < m->n_el; ++j) {
        double z = (double)m->Z[j];
        double eta = om_ms_screening(m->Z[j], T);
        double K = z * (z + 1.0) * OM_RE * OM_RE * OM_MC2 * OM_MC2 / (beta2 * pc2);
        s += atoms_per_gram(m, j) * 2.0 * OM_PI * K * (log1p(1.0 / eta) - 1.0 / (1.0 + eta));
    }
    return s;
}

/* Mean of mu = (1 - cos)/2 under f(mu) ~ (mu + a)^-2 on [0, 1]:
 *   <mu> = a [(1 + a) ln(1 + 1/a) - 1]. */
double om_ms_mean_mu(double a) {
    if (a > 1e3) {
        double x = 1.0 / a;
        return 0.5 - x / 6.0 + x * x / 12.0 - x * x * x / 20.0 + x * x * x * x / 30.0;
    }
    return a * ((1.0 + a) * log1p(1.0 / a) - 1.0);
}

/* Screening parameter a with <mu> = (1 - exp(-G1))/2, the Goudsmit-Saunderson
 * mean of (1 - cos theta)/2 after a path of G1 transport mean free paths.
 * Bisection on ln a (<mu> is increasing in a). */
double om_ms_solve_a(double g1) {
    double target = -0.5 * expm1(-g1);
    double lo = -80.0, hi = 40.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (om_ms_mean_mu(exp(mid)) < target)
            lo = mid;
        else
            hi = mid;
        if (hi - lo < 1e-13) break;
    }
    return exp(0.5 * (lo + hi));
}
