/*
 * Oracle transport: one history at a time, a LIFO particle stack, FP64.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Follows GPUMCD §II.A (photons: Woodcock tracking, Compton, photoelectric,
 * pair) and §II.B (electrons: Class II condensed history, step length
 * e_s = min{d_vox, e_s-max, e_hard}, CSDA loss, random hinge, hard Moller and
 * bremsstrahlung events).  Every cross-section is evaluated exactly at the
 * current energy (physics.c).  Dose moments are kept history by history
 * (§II.D, the Delta D^2 estimator).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* ------------------------------------------------------------------------
 * Random streams: a particle draws from Philox with key = seed and counter =
 * (draw index, lineage low, lineage high, history).  Two 32-bit words make one
 * 53-bit uniform in (0, 1].
 * ------------------------------------------------------------------------ */
typedef struct {
    uint32_t key[2];
    uint32_t hist;
    uint64_t lin;
    uint32_t draw;
    uint32_t buf[4];
    int used; /* words of buf consumed; 4 = empty */
} stream_t;

static void stream_init(stream_t *s, uint64_t seed, uint64_t hist, uint64_t lin, uint32_t draw) {
    s->key[0] = (uint32_t)seed;
    s->key[1] = (uint32_t)(seed >> 32);
    s->hist = (uint32_t)hist;
    s->lin = lin;
    s->draw = draw;
    s->used = 4;
}

static uint32_t next_word(stream_t *s) {
    if (s->used == 4) {
        uint32_t ctr[4] = {s->draw, (uint32_t)s->lin, (uint32_t)(s->lin >> 32), s->hist};
        om_philox4x32_10(ctr, s->key, s->buf);
        s->draw++;
        s->used = 0;
    }
    return s->buf[s->used++];
}

static double uniform(stream_t *s) {
    uint32_t a = next_word(s) >> 5, b = next_word(s) >> 6;
    return ((double)a * 67108864.0 + (double)b + 1.0) / 9007199254740992.0;
}

/* Lineage of the j-th particle created at draw index `draw` of parent `lin`:
 * a 64-bit mix, so that a particle's stream never depends on scheduling. */
static uint64_t child_lineage(uint64_t lin, uint32_t draw, uint32_t j) {
    uint64_t z = lin * 0x9E3779B97F4A7C15ull + (((uint64_t)draw << 8) | (j + 1));
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z | 2ull; /* never the primary's lineage (1) */
}

/* ------------------------------------------------------------------------
 * Direction change: rotate unit vector u by polar angle (cos c) and azimuth phi.
 * ------------------------------------------------------------------------ */
static void rotate(double u[3], double c, double phi) {
    double s = sqrt(fmax(0.0, 1.0 - c * c));
    double cp = cos(phi), sp = sin(phi);
    double a = u[0], b = u[1], w = u[2];
    double r2 = a * a + b * b;
    if (r2 > 1e-20) {
        double r = sqrt(r2);
        u[0] = a * c + s * (a * w * cp - b * sp) / r;
        u[1] = b * c + s * (b * w * cp + a * sp) / r;
        u[2] = w * c - s * cp * r;
    } else {
        double sg = w >= 0.0 ? 1.0 : -1.0;
        u[0] = s * cp;
        u[1] = s * sp;
        u[2] = sg * c;
    }
    double n = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    u[0] /= n;
    u[1] /= n;
    u[2] /= n;
}

void om_rotate(const double u[3], double c, double phi, double out[3]) {
    out[0] = u[0];
    out[1] = u[1];
    out[2] = u[2];
    rotate(out, c, phi);
}

/* Compton kinematics (§II.A): the photon leaves along u rotated by (cos_t, phi)
 * with energy eps E; the recoil electron takes T = E - eps E along the momentum
 * balance E u - E' u'. */
static void compton_kinematics(double E, const double u[3], double cos_t, double eps, double phi,
                               double u1[3], double ue[3], double *E1, double *T) {
    *E1 = eps * E;
    *T = E - *E1;
    u1[0] = u[0];
    u1[1] = u[1];
    u1[2] = u[2];
    rotate(u1, cos_t, phi);
    for (int a = 0; a < 3; ++a) ue[a] = E * u[a] - *E1 * u1[a];
    double n = sqrt(ue[0] * ue[0] + ue[1] * ue[1] + ue[2] * ue[2]);
    if (n > 0.0)
        for (int a = 0; a < 3; ++a) ue[a] /= n;
}

void om_compton_kinematics(double E, const double u[3], double cos_t, double eps, double phi,
                           double u1_out[3], double ue_out[3], double out[2]) {
    compton_kinematics(E, u, cos_t, eps, phi, u1_out, ue_out, &out[0], &out[1]);
}

/* Moller kinematics (§II.B.1): a knock-on of kinetic energy eps T and the
 * scattered electron with the rest, at the polar angles of a free two-body
 * collision, cos = sqrt(T'(T + 2mc^2)/(T (T' + 2mc^2))) for each. */
static void moller_kinematics(double T, double eps, double *Tk, double *Tp, double *ck, double *cp) {
    *Tk = eps * T;
    *Tp = T - *Tk;
    *ck = sqrt(*Tk * (T + 2.0 * OM_MC2) / (T * (*Tk + 2.0 * OM_MC2)));
    *cp = sqrt(*Tp * (T + 2.0 * OM_MC2) / (T * (*Tp + 2.0 * OM_MC2)));
}

void om_moller_kinematics(double T, double eps, double out[4]) {
    moller_kinematics(T, eps, &out[0], &out[1], &out[2], &out[3]);
}

/* ------------------------------------------------------------------------
 * Samplers (exact).
 * ------------------------------------------------------------------------ */

/* Klein-Nishina (§II.A, Compton): plain rejection on cos(theta) uniform in
 * [-1, 1] against (k'/k)^2 (k'/k + k/k' - sin^2) <= 2.  Returns cos and k'/k. */
static void sample_kn(stream_t *s, double k, double *cos_out, double *eps_out) {
    for (;;) {
        double c = 2.0 * uniform(s) - 1.0;
        double r = 1.0 / (1.0 + k * (1.0 - c));
        double f = r * r * (r + 1.0 / r - (1.0 - c * c));
        if (2.0 * uniform(s) <= f) {
            *cos_out = c;
            *eps_out = r;
            return;
        }
    }
}

/* Sauter K-shell photo-electron direction (§II.A, photoelectric effect).
 * With nu = 1 - cos, A = 1/beta - 1 and B = beta g (g-1)(g-2)/2 the density is
 * p(nu) ~ (2 - nu) [1/(A + nu) + B] nu/(A + nu)^3 on [0, 2].  nu is drawn from
 * nu/(A+nu)^3 (CDF [nu (A+2)/(2(A+nu))]^2) and accepted with
 * (2 - nu)[1/(A+nu) + B] / (2 [1/A + B]). */
static double sample_sauter(stream_t *s, double T) {
    double g = T / OM_MC2 + 1.0;
    double beta = sqrt(1.0 - 1.0 / (g * g));
    double A = 1.0 / beta - 1.0;
    double B = 0.5 * beta * g * (g - 1.0) * (g - 2.0);
    double gmax = 2.0 * (1.0 / A + B);
    for (;;) {
        double sq = sqrt(uniform(s));
        double nu = 2.0 * A * sq / (A + 2.0 - 2.0 * sq);
        double g2 = (2.0 - nu) * (1.0 / (A + nu) + B);
        if (uniform(s) * gmax <= g2) return 1.0 - nu;
    }
}

/* Moller knock-on fraction eps in [t_c/T, 1/2] (§II.B.1): proposal from
 * 1/eps^2, rejection with eps^2 dsigma/deps <= 2 + ((g-1)/g)^2/4. */
static double sample_moller(stream_t *s, double T, double t_c) {
    double g = T / OM_MC2 + 1.0;
    double c1 = (g - 1.0) / g;
    c1 *= c1;
    double c2 = (2.0 * g - 1.0) / (g * g);
    double ec = t_c / T;
    double bound = 2.0 + 0.25 * c1;
    for (;;) {
        double eps = ec / (1.0 - uniform(s) * (1.0 - 2.0 * ec));
        double r = eps / (1.0 - eps);
        double f = 1.0 + r * r + c1 * eps * eps - c2 * r;
        if (uniform(s) * bound <= f) return eps;
    }
}

/* Bremsstrahlung photon energy in [k_c, T] (§II.B.1): proposal from 1/k,
 * rejection with the bracket of dsigma/dk, which is largest at y = 0. */
typedef struct {
    double SA, S1;
} brem_sums_t;

static brem_sums_t brem_sums_of(const om_material *m) {
    brem_sums_t b = {0.0, 0.0};
    for (int j = 0; j < m->n_el; ++j) {
        double z = (double)m->Z[j];
        double n = OM_NA * m->w[j] / m->A[j];
        b.SA += n * z * (z + 1.0) * log(183.0 * pow(z, -1.0 / 3.0));
        b.S1 += n * z * (z + 1.0);
    }
    return b;
}

static double sample_brem(stream_t *s, const brem_sums_t *b, double T, double k_c) {
    double E = T + OM_MC2;
    double g0 = (4.0 / 3.0) * b->SA + b->S1 / 9.0;
    for (;;) {
        double k = k_c * pow(T / k_c, uniform(s));
        double y = k / E;
        double g = (4.0 / 3.0 - 4.0 * y / 3.0 + y * y) * b->SA + (1.0 - y) * b->S1 / 9.0;
        if (uniform(s) * g0 <= g) return k;
    }
}

/* Multiple-scattering deflection (§II.B.2 substitute): mu = (1 - cos)/2 from
 * f(mu) ~ (mu + a)^-2 on [0, 1], a fixed by <mu> = (1 - exp(-G1))/2; the
 * inverse CDF is mu = a z / (1 + a - z).  Paths under G1 = 1e-8 are not
 * deflected, paths over G1 = 20 come out isotropic. */
#define MS_G_MIN 1e-8
#define MS_G_MAX 20.0
static double sample_ms_mu(stream_t *s, double g1) {
    if (g1 < MS_G_MIN) return 0.0;
    double z = uniform(s);
    if (g1 > MS_G_MAX) return z;
    double a = om_ms_solve_a(g1);
    return a * z / (1.0 + a - z);
}

static int spectrum_bin(int32_t n, const double *cdf, double z) {
    int lo = 0, hi = n - 1; /* first bin with cdf[i+1] >= z */
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (cdf[mid + 1] >= z)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

/* Inverse CDF of a histogram spectrum at quantile z: the bin by the
 * cumulative weights, then linear inside it (a uniform z gives a uniform energy
 * within the bin). */
static double spectrum_at(int32_t n, const double *edges, const double *cdf, double z) {
    int i = spectrum_bin(n, cdf, z);
    double w = cdf[i + 1] - cdf[i];
    double f = w > 0.0 ? (z - cdf[i]) / w : 0.5;
    if (f < 0.0) f = 0.0;
    if (f > 1.0) f = 1.0;
    return edges[i] + f * (edges[i + 1] - edges[i]);
}

/* Inverse-CDF draw from a histogram spectrum. */
static double sample_spectrum(stream_t *s, int32_t n, const double *edges, const double *cdf) {
    return spectrum_at(n, edges, cdf, uniform(s));
}

static double *spectrum_cdf(int32_t n, const double *w) {
    double *cdf = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double tot = 0.0;
    for (int i = 0; i < n; ++i) tot += w[i];
    cdf[0] = 0.0;
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
        acc += w[i];
        cdf[i + 1] = acc / tot;
    }
    cdf[n] = 1.0;
    return cdf;
}

/* ------------------------------------------------------------------------
 * Transport context.
 * ------------------------------------------------------------------------ */
typedef struct {
    double x[3], u[3];
    double E; /* photon energy or electron kinetic energy, MeV */
    int type; /* 0 photon, 1 electron */
    uint64_t lin;
    uint32_t draw;
} part_t;

#define E_GRID 4096

typedef struct {
    const om_material *mats;
    int n_mat;
    om_physics ph;
    const om_phantom *geo;
    uint32_t flags;
    uint64_t seed;
    uint64_t hist;
    double rho_max[OM_MAX_MATERIALS];
    int present[OM_MAX_MATERIALS];
    brem_sums_t brem[OM_MAX_MATERIALS];
    double sig_hat[E_GRID]; /* electron hard-event majorant, running max */
    double lnT0, dlnT;
    /* per-history tally */
    double *hist_e;
    int64_t *touched;
    int64_t n_touched;
    /* particle stack */
    part_t *stack;
    int64_t n_stack, cap_stack;
    om_stats *st;
    int err;
} ctx_t;

static int64_t voxel_of(const ctx_t *c, const double x[3]) {
    const om_phantom *g = c->geo;
    if (!(x[0] >= 0.0 && x[1] >= 0.0 && x[2] >= 0.0)) return -1;
    if (!(x[0] < g->nx * g->dx && x[1] < g->ny * g->dy && x[2] < g->nz * g->dz)) return -1;
    int64_t ix = (int64_t)floor(x[0] / g->dx), iy = (int64_t)floor(x[1] / g->dy),
            iz = (int64_t)floor(x[2] / g->dz);
    if (ix > g->nx - 1) ix = g->nx - 1;
    if (iy > g->ny - 1) iy = g->ny - 1;
    if (iz > g->nz - 1) iz = g->nz - 1;
    return ix + (int64_t)g->nx * (iy + (int64_t)g->ny * iz);
}

static void deposit(ctx_t *c, int64_t v, double e) {
    if (e <= 0.0) return;
    if (c->hist_e[v] == 0.0) c->touched[c->n_touched++] = v;
    c->hist_e[v] += e;
    c->st->e_deposited += e;
}

static void push(ctx_t *c, const part_t *p) {
    if (c->n_stack == c->cap_stack) {
        c->cap_stack = c->cap_stack ? 2 * c->cap_stack : 256;
        c->stack = (part_t *)realloc(c->stack, sizeof(part_t) * (size_t)c->cap_stack);
    }
    c->stack[c->n_stack++] = *p;
}

/* Photon majorant mu_hat(E) = max over materials present of rho_max,m (mu/rho)_m(E)
 * (§II.A, Woodcock tracking: mu_max of the most attenuating voxel). */
static double photon_majorant(const ctx_t *c, double E) {
    double best = 0.0;
    for (int m = 0; m < c->n_mat; ++m)
        if (c->present[m]) {
            double v = c->rho_max[m] * om_mu_total(&c->mats[m], E);
            if (v > best) best = v;
        }
    return best;
}

static double hard_sigma(const ctx_t *c, int m, double T) {
    return om_sigma_moller(&c->mats[m], T, c->ph.t_c) + om_sigma_brem(&c->mats[m], T, c->ph.k_c);
}

/* Electron hard-event majorant (§II.B.3, electron Woodcock): the largest
 * rho_max,m Sigma_m(T') over T' in [e_abs, T], so that it bounds the cross-
 * section anywhere along a step that starts at T.  Kept as a running max on a
 * fine log grid, read at the grid point at or above T, with a 0.2% margin. */
static void build_electron_majorant(ctx_t *c) {
    double t0 = c->ph.e_abs, t1 = c->ph.e_max;
    c->lnT0 = log(t0);
    c->dlnT = (log(t1) - c->lnT0) / (E_GRID - 1);
    double run = 0.0;
    for (int i = 0; i < E_GRID; ++i) {
        double T = exp(c->lnT0 + i * c->dlnT);
        for (int m = 0; m < c->n_mat; ++m)
            if (c->present[m]) {
                double v = c->rho_max[m] * hard_sigma(c, m, T);
                if (v > run) run = v;
            }
        c->sig_hat[i] = run;
    }
}

static double electron_majorant(const ctx_t *c, double T) {
    double f = (log(T) - c->lnT0) / c->dlnT;
    int64_t i = (int64_t)ceil(f);
    if (i < 0) i = 0;
    if (i > E_GRID - 1) i = E_GRID - 1;
    return c->sig_hat[i] * 1.002;
}

/* Distance along u to the faces of the voxel holding x, plus the nudge. */
static double distance_to_voxel_exit(const ctx_t *c, const double x[3], const double u[3]) {
    const om_phantom *g = c->geo;
    double d[3] = {g->dx, g->dy, g->dz};
    double best = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (u[a] == 0.0) continue;
        double i = floor(x[a] / d[a]);
        double face = u[a] > 0.0 ? (i + 1.0) * d[a] : i * d[a];
        double t = (face - x[a]) / u[a];
        if (t < 0.0) t = 0.0;
        if (t < best) best = t;
    }
    return best + c->ph.nudge_cm;
}

/* A new electron of kinetic energy T at x: transported later, or deposited on
 * the spot below the cut-off (and always in the KERMA test mode). */
static void emit_electron(ctx_t *c, const double x[3], const double u[3], double T,
                          const part_t *parent, uint32_t j) {
    if (T <= 0.0) return;
    if ((c->flags & OM_FLAG_KERMA) || T < c->ph.e_abs) {
        int64_t v = voxel_of(c, x);
        if (v >= 0) {
            deposit(c, v, T);
            c->st->e_cut_electron += T;
        } else {
            c->st->e_escaped += T;
        }
        return;
    }
    part_t p;
    memcpy(p.x, x, sizeof p.x);
    memcpy(p.u, u, sizeof p.u);
    p.E = T;
    p.type = 1;
    p.lin = child_lineage(parent->lin, parent->draw, j);
    p.draw = 0;
    push(c, &p);
}

static void emit_photon(ctx_t *c, const double x[3], const double u[3], double k,
                        const part_t *parent, uint32_t j) {
    if (k <= 0.0) return;
    if (k < c->ph.p_cut) {
        int64_t v = voxel_of(c, x);
        if (v >= 0) {
            deposit(c, v, k);
            c->st->e_cut_photon += k;
        } else {
            c->st->e_escaped += k;
        }
        return;
    }
    part_t p;
    memcpy(p.x, x, sizeof p.x);
    memcpy(p.u, u, sizeof p.u);
    p.E = k;
    p.type = 0;
    p.lin = child_lineage(parent->lin, parent->draw, j);
    p.draw = 0;
    push(c, &p);
}

/* Woodcock flight (§II.A): fly with mu_hat until a real interaction (returns 1,
 * with the voxel in *v_out) or until the photon leaves the phantom (returns 0).
 * Distances follow s = -ln(z)/mu_hat, z in (0, 1]. */
static int woodcock_flight(ctx_t *c, part_t *p, stream_t *s, int64_t *v_out) {
    for (;;) {
        double mu_hat = photon_majorant(c, p->E);
        double d = -log(uniform(s)) / mu_hat;
        for (int a = 0; a < 3; ++a) p->x[a] += d * p->u[a];
        int64_t v = voxel_of(c, p->x);
        if (v < 0) return 0;
        int m = c->geo->mat[v];
        double mu = c->geo->rho[v] * om_mu_total(&c->mats[m], p->E);
        if (mu > mu_hat * (1.0 + 1e-12)) {
            c->err = -2;
            return 0;
        }
        if (uniform(s) * mu_hat <= mu) {
            c->st->n_photon_real++;
            *v_out = v;
            return 1;
        }
        c->st->n_photon_fict++;
    }
}

static void transport_photon(ctx_t *c, part_t *p) {
    stream_t s;
    stream_init(&s, c->seed, c->hist, p->lin, p->draw);
    c->st->n_photons++;
    for (;;) {
        if (p->E < c->ph.p_cut) {
            int64_t v = voxel_of(c, p->x);
            if (v >= 0) {
                deposit(c, v, p->E);
                c->st->e_cut_photon += p->E;
            } else {
                c->st->e_escaped += p->E;
            }
            return;
        }
        int64_t v;
        if (!woodcock_flight(c, p, &s, &v)) {
            c->st->e_escaped += p->E;
            return;
        }
        if (c->err) return;
        const om_material *m = &c->mats[c->geo->mat[v]];
        double rho = c->geo->rho[v];
        double mc = rho * om_mu_compton(m, p->E), mpe = rho * om_mu_photo(m, p->E);
        double mpp = rho * om_mu_pair(m, p->E);
        double r = uniform(&s) * (mc + mpe + mpp);
        p->draw = s.draw; /* secondaries take their lineage from this point */
        if (r < mc) {
            /* Compton: scattered photon and recoil electron (momentum balance). */
            c->st->n_compton++;
            double cs, eps;
            sample_kn(&s, p->E / OM_MC2, &cs, &eps);
            double phi = 2.0 * OM_PI * uniform(&s);
            double E1, T, u1[3], pe[3];
            compton_kinematics(p->E, p->u, cs, eps, phi, u1, pe, &E1, &T);
            emit_electron(c, p->x, pe, T, p, 0);
            p->E = E1;
            memcpy(p->u, u1, sizeof u1);
            if (c->flags & OM_FLAG_FIRST_COLLISION) {
                c->st->e_escaped += p->E;
                return;
            }
        } else if (r < mc + mpe) {
            /* Photoelectric: one electron with kinetic energy E (binding ignored). */
            c->st->n_photo++;
            double cs = sample_sauter(&s, p->E);
            double phi = 2.0 * OM_PI * uniform(&s);
            double ue[3] = {p->u[0], p->u[1], p->u[2]};
            rotate(ue, cs, phi);
            emit_electron(c, p->x, ue, p->E, p, 0);
            return;
        } else {
            /* Pair: no positron; two electrons share E - 2mc^2 uniformly, the
             * rest energy 2mc^2 is booked apart; polar angles mc^2/E_total. */
            c->st->n_pair++;
            double Tt = p->E - 2.0 * OM_MC2;
            c->st->e_rest += 2.0 * OM_MC2;
            double T1 = uniform(&s) * Tt;
            double T2 = Tt - T1;
            double phi = 2.0 * OM_PI * uniform(&s);
            double u1[3] = {p->u[0], p->u[1], p->u[2]};
            double u2[3] = {p->u[0], p->u[1], p->u[2]};
            rotate(u1, cos(OM_MC2 / (T1 + OM_MC2)), phi);
            rotate(u2, cos(OM_MC2 / (T2 + OM_MC2)), phi + OM_PI);
            emit_electron(c, p->x, u1, T1, p, 0);
            emit_electron(c, p->x, u2, T2, p, 1);
            return;
        }
        p->draw = s.draw;
    }
}

static void transport_electron(ctx_t *c, part_t *p) {
    stream_t s;
    stream_init(&s, c->seed, c->hist, p->lin, p->draw);
    c->st->n_electrons++;
    const om_physics *P = &c->ph;
    for (;;) {
        int64_t v0 = voxel_of(c, p->x);
        if (v0 < 0) {
            c->st->e_escaped += p->E;
            return;
        }
        if (p->E < P->e_abs) {
            deposit(c, v0, p->E);
            c->st->e_cut_electron += p->E;
            return;
        }
        int m0 = c->geo->mat[v0];
        const om_material *mat0 = &c->mats[m0];
        double rho0 = c->geo->rho[v0];
        double T = p->E;
        /* restricted loss: collision below t_c plus radiative below k_c (§II.B.3) */
        double L0 = rho0 * (om_l_col(mat0, T, P->t_c) + om_l_rad(mat0, T, P->k_c));
        double smax = P->estepe * T / L0;
        double dvox = distance_to_voxel_exit(c, p->x, p->u);
        double sig_hat = (c->flags & OM_FLAG_VOXEL_EMAJOR) ? rho0 * hard_sigma(c, m0, T) * 1.002
                                                           : electron_majorant(c, T);
        double ehard = sig_hat > 0.0 ? -log(uniform(&s)) / sig_hat : INFINITY;
        /* e_s = min{d_vox, e_s-max, e_hard} */
        double es = dvox < smax ? dvox : smax;
        int hard = 0;
        if (ehard < es) {
            es = ehard;
            hard = 1;
        }
        /* Delta E = e_s L(E0 - L(E0) e_s / 2) (EGSnrc Eq. 4.11.3; the s factor is
         * implied by the integral of L over the step) */
        double Tm = T - 0.5 * L0 * es;
        double dE = es * rho0 * (om_l_col(mat0, Tm, P->t_c) + om_l_rad(mat0, Tm, P->k_c));
        if (dE > T) dE = T;
        double T1 = T - dE;
        /* random hinge (§II.B.3): move z e_s, deflect, deposit, move (1 - z) e_s;
         * the deflection uses the energy before or after the loss at random */
        double zh = uniform(&s);
        double xh[3];
        for (int a = 0; a < 3; ++a) xh[a] = p->x[a] + zh * es * p->u[a];
        if (!(c->flags & OM_FLAG_NO_MS)) {
            double Tms = uniform(&s) < 0.5 ? T : T1;
            double g1 = Tms > 0.0 ? es * rho0 * om_ms_lambda1_inv(mat0, Tms) : INFINITY;
            double mu = sample_ms_mu(&s, g1);
            if (mu > 0.0) {
                double phi = 2.0 * OM_PI * uniform(&s);
                rotate(p->u, 1.0 - 2.0 * mu, phi);
            }
        }
        deposit(c, v0, dE); /* the hinge lies in the step-start voxel */
        for (int a = 0; a < 3; ++a) p->x[a] = xh[a] + (1.0 - zh) * es * p->u[a];
        c->st->track_length_cm += es;
        c->st->n_e_steps++;
        p->E = T1;
        int64_t v1 = voxel_of(c, p->x);
        if (v1 < 0) {
            c->st->e_escaped += T1;
            return;
        }
        if (T1 < P->e_abs) {
            deposit(c, v1, T1);
            c->st->e_cut_electron += T1;
            return;
        }
        if (!hard) continue;
        /* Woodcock acceptance at the end point with the end energy (in the
         * step's voxel with the per-voxel majorant) */
        int m1 = (c->flags & OM_FLAG_VOXEL_EMAJOR) ? m0 : c->geo->mat[v1];
        double rho1 = (c->flags & OM_FLAG_VOXEL_EMAJOR) ? rho0 : c->geo->rho[v1];
        double sm = rho1 * om_sigma_moller(&c->mats[m1], T1, P->t_c);
        double sb = rho1 * om_sigma_brem(&c->mats[m1], T1, P->k_c);
        if (sm + sb > sig_hat) {
            c->err = -2;
            return;
        }
        if (uniform(&s) * sig_hat >= sm + sb) {
            c->st->n_hard_fict++;
            continue;
        }
        c->st->n_hard_real++;
        int moller = uniform(&s) * (sm + sb) < sm;
        p->draw = s.draw;
        if (moller) {
            c->st->n_moller++;
            double eps = sample_moller(&s, T1, P->t_c);
            double Tk, Tp, ck, cp;
            moller_kinematics(T1, eps, &Tk, &Tp, &ck, &cp);
            double phi = 2.0 * OM_PI * uniform(&s);
            double uk[3] = {p->u[0], p->u[1], p->u[2]};
            rotate(uk, ck, phi);
            rotate(p->u, cp, phi + OM_PI);
            emit_electron(c, p->x, uk, Tk, p, 0);
            p->E = Tp;
        } else {
            c->st->n_brem++;
            double k = sample_brem(&s, &c->brem[m1], T1, P->k_c);
            double th = OM_MC2 / (T1 + OM_MC2);
            double phi = 2.0 * OM_PI * uniform(&s);
            double ug[3] = {p->u[0], p->u[1], p->u[2]};
            rotate(ug, cos(th), phi);
            emit_photon(c, p->x, ug, k, p, 0);
            p->E = T1 - k;
        }
        p->draw = s.draw;
    }
}

static int validate(const om_material *mats, int32_t n_mat, const om_physics *phys,
                    const om_phantom *ph, const om_source *src) {
    if (!mats || n_mat < 1 || n_mat > OM_MAX_MATERIALS || !phys || !ph || !src) return -1;
    if (ph->nx < 1 || ph->ny < 1 || ph->nz < 1 || !(ph->dx > 0 && ph->dy > 0 && ph->dz > 0)) return -1;
    if (src->beam == 2) {
        if (src->n_phsp < 1 || !src->phsp) return -1;
        for (int32_t i = 0; i < src->n_phsp; ++i) {
            const double *r = src->phsp + 7 * (size_t)i;
            for (int a = 0; a < 7; ++a)
                if (!isfinite(r[a])) return -1;
            if (!(r[6] > 0.0 && r[6] <= phys->e_max)) return -1;
            if (!(r[3] * r[3] + r[4] * r[4] + r[5] * r[5] > 0.0)) return -1;
        }
        return 0;
    }
    if (src->n_spec < 0) return -1;
    if (src->n_spec == 0 && !(src->energy > 0.0 && src->energy <= phys->e_max)) return -1;
    if (src->n_spec > 0 && !(src->spec_edges[src->n_spec] <= phys->e_max)) return -1;
    return 0;
}

static int ctx_setup(ctx_t *c, const om_material *mats, int32_t n_mat, const om_physics *phys,
                     const om_phantom *ph, uint64_t seed, uint32_t flags, om_stats *st) {
    memset(c, 0, sizeof *c);
    c->mats = mats;
    c->n_mat = n_mat;
    c->ph = *phys;
    c->geo = ph;
    c->seed = seed;
    c->flags = flags;
    c->st = st;
    int64_t nvox = (int64_t)ph->nx * ph->ny * ph->nz;
    for (int64_t v = 0; v < nvox; ++v) {
        int m = ph->mat[v];
        if (m >= n_mat) return -1;
        c->present[m] = 1;
        if (ph->rho[v] > c->rho_max[m]) c->rho_max[m] = ph->rho[v];
    }
    for (int m = 0; m < n_mat; ++m) c->brem[m] = brem_sums_of(&mats[m]);
    build_electron_majorant(c);
    c->hist_e = (double *)calloc((size_t)nvox, sizeof(double));
    c->touched = (int64_t *)malloc(sizeof(int64_t) * (size_t)nvox);
    return 0;
}

static void ctx_free(ctx_t *c) {
    free(c->hist_e);
    free(c->touched);
    free(c->stack);
}

/* Primary particle of history h (§II.C.2, initParticle): a pencil or square
 * parallel beam entering through z = 0 along +z, mono energy or a spectrum;
 * or, for a phase-space source, record h mod n as given (direction
 * normalised). */
static void make_primary(ctx_t *c, const om_source *src, const double *cdf, uint64_t h,
                         part_t *p, stream_t *s) {
    stream_init(s, c->seed, h, 1ull, 0);
    if (src->beam == 2) {
        const double *r = src->phsp + 7 * (h % (uint64_t)src->n_phsp);
        const double nu = sqrt(r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
        for (int a = 0; a < 3; ++a) {
            p->x[a] = r[a];
            p->u[a] = r[3 + a] / nu;
        }
        p->E = r[6];
        p->type = src->particle;
        p->lin = 1ull;
        p->draw = s->draw;
        return;
    }
    p->x[0] = src->cx;
    p->x[1] = src->cy;
    p->x[2] = 0.0;
    if (src->beam == 1) {
        p->x[0] = src->cx + (uniform(s) - 0.5) * src->field;
        p->x[1] = src->cy + (uniform(s) - 0.5) * src->field;
    }
    p->u[0] = 0.0;
    p->u[1] = 0.0;
    p->u[2] = 1.0;
    p->E = src->n_spec > 0 ? sample_spectrum(s, src->n_spec, src->spec_edges, cdf) : src->energy;
    p->type = src->particle;
    p->lin = 1ull;
    p->draw = s->draw;
}

int32_t om_simulate(const om_material *mats, int32_t n_mat, const om_physics *phys,
                    const om_phantom *ph, const om_source *src, uint64_t hist_begin,
                    uint64_t hist_end, uint64_t seed, uint32_t flags, double *sum_e,
                    double *sum_e2, om_stats *stats) {
    if (validate(mats, n_mat, phys, ph, src) != 0 || !sum_e || !sum_e2 || !stats) return -1;
    ctx_t c;
    if (ctx_setup(&c, mats, n_mat, phys, ph, seed, flags, stats) != 0) {
        ctx_free(&c);
        return -1;
    }
    double *cdf = src->n_spec > 0 ? spectrum_cdf(src->n_spec, src->spec_weights) : NULL;
    for (uint64_t h = hist_begin; h < hist_end && !c.err; ++h) {
        c.hist = h;
        part_t p;
        stream_t s;
        make_primary(&c, src, cdf, h, &p, &s);
        stats->e_incident += p.E;
        stats->n_histories++;
        c.n_stack = 0;
        push(&c, &p);
        while (c.n_stack > 0 && !c.err) {
            part_t q = c.stack[--c.n_stack];
            if (q.type == 0)
                transport_photon(&c, &q);
            else if (c.flags & OM_FLAG_KERMA) {
                int64_t v = voxel_of(&c, q.x);
                if (v >= 0)
                    deposit(&c, v, q.E);
                else
                    stats->e_escaped += q.E;
            } else
                transport_electron(&c, &q);
        }
        /* history-by-history moments (§II.D) */
        for (int64_t i = 0; i < c.n_touched; ++i) {
            int64_t v = c.touched[i];
            double e = c.hist_e[v];
            sum_e[v] += e;
            sum_e2[v] += e * e;
            c.hist_e[v] = 0.0;
        }
        c.n_touched = 0;
    }
    int err = c.err;
    free(cdf);
    ctx_free(&c);
    return err;
}

int32_t om_first_interaction_z(const om_material *mats, int32_t n_mat, const om_physics *phys,
                               const om_phantom *ph, const om_source *src, int64_t n,
                               uint64_t seed, double *z_out, uint64_t *n_fict_out) {
    if (validate(mats, n_mat, phys, ph, src) != 0 || src->particle != 0) return -1;
    om_stats st;
    memset(&st, 0, sizeof st);
    ctx_t c;
    if (ctx_setup(&c, mats, n_mat, phys, ph, seed, 0, &st) != 0) {
        ctx_free(&c);
        return -1;
    }
    double *cdf = src->n_spec > 0 ? spectrum_cdf(src->n_spec, src->spec_weights) : NULL;
    for (int64_t h = 0; h < n && !c.err; ++h) {
        c.hist = (uint64_t)h;
        part_t p;
        stream_t s;
        make_primary(&c, src, cdf, (uint64_t)h, &p, &s);
        int64_t v;
        z_out[h] = woodcock_flight(&c, &p, &s, &v) ? p.x[2] : INFINITY;
    }
    if (n_fict_out) *n_fict_out = st.n_photon_fict;
    int err = c.err;
    free(cdf);
    ctx_free(&c);
    return err;
}

/* ------------------------------------------------------------------------
 * Sampler entry points for the distribution pins.
 * ------------------------------------------------------------------------ */
void om_sample_kn(double k, int64_t n, uint64_t seed, double *cos_out, double *eps_out) {
    stream_t s;
    stream_init(&s, seed, 0, 7, 0);
    for (int64_t i = 0; i < n; ++i) sample_kn(&s, k, &cos_out[i], &eps_out[i]);
}

void om_sample_sauter(double T, int64_t n, uint64_t seed, double *cos_out) {
    stream_t s;
    stream_init(&s, seed, 0, 7, 0);
    for (int64_t i = 0; i < n; ++i) cos_out[i] = sample_sauter(&s, T);
}

void om_sample_moller(double T, double t_c, int64_t n, uint64_t seed, double *eps_out) {
    stream_t s;
    stream_init(&s, seed, 0, 7, 0);
    for (int64_t i = 0; i < n; ++i) eps_out[i] = sample_moller(&s, T, t_c);
}

void om_sample_brem(const om_material *m, double T, double k_c, int64_t n, uint64_t seed,
                    double *k_out) {
    stream_t s;
    stream_init(&s, seed, 0, 7, 0);
    brem_sums_t b = brem_sums_of(m);
    for (int64_t i = 0; i < n; ++i) k_out[i] = sample_brem(&s, &b, T, k_c);
}

void om_sample_ms(double g1, int64_t n, uint64_t seed, double *mu_out) {
    stream_t s;
    stream_init(&s, seed, 0, 7, 0);
    for (int64_t i = 0; i < n; ++i) mu_out[i] = sample_ms_mu(&s, g1);
}

int32_t om_primary_energies(const om_source *src, uint64_t hist_begin, uint64_t hist_end,
                            uint64_t seed, double *e_out) {
    if (!src || !e_out || src->beam == 2 || src->n_spec < 0 || hist_end < hist_begin) return -1;
    ctx_t c;
    memset(&c, 0, sizeof c);
    c.seed = seed;
    double *cdf = src->n_spec > 0 ? spectrum_cdf(src->n_spec, src->spec_weights) : NULL;
    for (uint64_t h = hist_begin; h < hist_end; ++h) {
        part_t p;
        stream_t s;
        make_primary(&c, src, cdf, h, &p, &s);
        e_out[h - hist_begin] = p.E;
    }
    free(cdf);
    return 0;
}

void om_sample_spectrum(int32_t n_bins, const double *edges, const double *weights, int64_t n,
                        uint64_t seed, double *e_out) {
    stream_t s;
    stream_init(&s, seed, 0, 7, 0);
    double *cdf = spectrum_cdf(n_bins, weights);
    for (int64_t i = 0; i < n; ++i) e_out[i] = sample_spectrum(&s, n_bins, edges, cdf);
    free(cdf);
}
