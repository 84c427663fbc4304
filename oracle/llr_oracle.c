/*
 * llr_oracle.c -- plain FP64 reference implementation ("oracle") of the
 * window-restricted Monte Carlo of the LLR density-of-states method for
 * compact U(1) lattice gauge theory.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline timing of the benchmark may load this library.  The product
 * (the CUDA library under paper_1509_08391_gb300/) shares no code with it.
 *
 * Paper: K. Langfeld, B. Lucini, R. Pellegrini, A. Rago, "An efficient
 * algorithm for numerical computations of continuous densities of states"
 * (arXiv:1509.08391).  Equations are cited by their printed numbers, e.g.
 * eq. (2.30) is the under-relaxed Robbins-Monro update of Sec. 2.2.
 *
 * What is computed (and where it is defined):
 *   - Sec. 3.1: link angles theta_mu(x) in [-pi,pi), plaquette angle
 *     theta_munu(x) = theta_mu(x) + theta_nu(x+mu) - theta_mu(x+nu) - theta_nu(x),
 *     energy E = sum_{x, mu<nu} cos theta_munu(x) (beta factored out), Haar
 *     measure prod dtheta/2pi.
 *   - Sec. 2.2, eqs. (2.13)-(2.16): expectation values restricted to the closed
 *     window E_k <= E <= E_k + dE, reweighted by exp(-a E).
 *   - Sec. 2.4, Algorithm 1: N_TH + N_SW importance-sampling sweeps per
 *     Robbins-Monro iteration, measuring E after N_TH, then the update of a.
 *   - Sec. 2.2, eq. (2.30): a <- a + 12 <<dE>> / (dE^2 (n+1)) (sign of eq. (2.30);
 *     Algorithm 1 prints the opposite sign, see the readings below).
 *
 * Readings where the paper is silent:
 *   R1 update scheme: the paper names only "an importance sampling
 *      algorithm for one sweep" (Algorithm 1) and mentions heat-bath and
 *      Metropolis.  A composite sweep here is one heat-bath pass followed by
 *      n_or overrelaxation passes.  A heat-bath pass visits the 2*d
 *      checkerboard classes (direction mu, site parity p) in the order
 *      mu = 0..d-1, p = 0,1, each over the whole lattice; an overrelaxation
 *      pass walks the slabs of the last coordinate and, within a slab, the
 *      classes in the same order.  Links of one class share no plaquette, so
 *      each group (a class, or a class within a slab) is one set of
 *      independent proposals.
 *   R2 window restriction (Sec. 2.4 allows imposing it after the proposal):
 *      within a class every link draws an independent proposal from its
 *      unrestricted conditional distribution (heat-bath at weight exp(-aE),
 *      or the overrelaxation reflection); the proposals are then accepted
 *      or rejected in ascending site order, in blocks of B consecutive
 *      links starting at the group's first link, by the Metropolis rule for
 *      the restricted measure: a heat-bath block is
 *      accepted iff dist(E + dE_block) <= dist(E), where dist is the distance
 *      of E from the window (0 inside).  Inside the window this is exactly
 *      the indicator of eq. (2.13); outside it only lets E move towards the
 *      window (used while approaching the window from a hot start).
 *  R19 overrelaxation blocks: the reflection keeps E in exact arithmetic, so
 *      the running energy is not moved by overrelaxation moves (their dE is
 *      rounding, ~1e-15 in FP64) and a block is accepted iff E + dE_block lies
 *      in the window, or E does not (outside the window reflections are
 *      always taken), E being the running energy before the pass.  A
 *      reflection whose |dE| exceeds 2^-14 is refused (a guard for float32
 *      arithmetic; FP64 never reaches it).  The fresh energy at the end of the
 *      composite sweep takes up the moves' rounding.
 *   R3 heat-bath proposal: von Mises variate by Best & Fisher (1979).
 *   R4 random numbers: Philox4x32-10 (Salmon et al., SC'11), keyed by
 *      (seed, interval, replica), counter (link, sweep, tag, attempt / 2):
 *      one call serves two sampler attempts (words 0-1 and 2-3; the sign of
 *      X is the lowest bit of the attempt's first word).
 *   R5 approach phase: from a hot start, heat-bath at a = -beta_up (E below
 *      the window) or a = -beta_dn (E above) with the dist rule, until the
 *      energy lies in the window at the end of a composite sweep.
 *   R6 the tracked energy is re-synchronised with a fresh plaquette sum at
 *      the end of every composite sweep; the measurement uses that value.
 *   R7 replica exchange (Sec. 2.5): the caller names the pairs of overlapping
 *      intervals tried in one exchange round and a round number; the draw
 *      deciding a pair comes from Philox keyed by the pair's first lattice,
 *      counter (0, round, swap tag, 0), as a 53-bit uniform in [0, 1).
 *   R8 multicanonical run (Sec. 2.6, eq. (2.50)): weight W(E) = 1/rho~(E), with
 *      ln rho~ the piecewise-linear function of eq. (2.10) built from the
 *      slopes of n contiguous intervals and continued linearly with the end
 *      slopes outside them (the micro-canonical beta_1, beta_2 tails).  A
 *      heat-bath pass proposes every link of a class from its conditional
 *      at a fixed slope a0 (the same proposals as the restricted heat-bath)
 *      and accepts them in link order by Metropolis-Hastings for W:
 *      u < exp(a0 dE - (ln rho~(E + dE) - ln rho~(E))), u from Philox
 *      counter (link, sweep, 12, 0) word 0.  Overrelaxation passes keep E
 *      and are always taken.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): 10 rounds of a multiply-xor bijection on a
 * 128-bit counter, with a Weyl-sequence key schedule.
 * ---------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A 32-bit word to a uniform in the open interval (0,1): the top 23 bits
 * k give (2k+1) * 2^-24, exact in both float and double. */
double orc_uniform(uint32_t w)
{
    return (double)((w >> 9) * 2u + 1u) * (1.0 / 16777216.0);
}

/* Wrap an angle to [-pi, pi). */
static double wrap_angle(double t)
{
    return t - 2.0 * M_PI * floor((t + M_PI) / (2.0 * M_PI));
}

/* ------------------------------------------------------------------------
 * Geometry: a d-dimensional hypercubic lattice (d <= 4), periodic or open.
 * Sites are numbered lexicographically with x_0 fastest.  Link slot
 * l = mu * nsite + site (a slot exists only if the link does, which always
 * holds with periodic boundaries).  Plaquettes are listed explicitly from
 * the definition of Sec. 3.1, and every link gets the list of plaquettes it
 * belongs to, with the sign it carries there.
 * ---------------------------------------------------------------------- */
typedef struct {
    int d, periodic, dims[4], nsite, nslot;
    int *exists;             /* [nslot] */
    int nplaq;
    int *plaq_link;          /* [nplaq][4] */
    int *plaq_sign;          /* [nplaq][4] */
    int *lp_start;           /* [nslot+1] into lp_plaq/lp_pos */
    int *lp_plaq, *lp_pos;   /* plaquette index and position of the link in it */
    int *class_start;        /* [2d+1] */
    int *class_links;        /* links of class (mu,p) in ascending site order */
} orc_geom;

static void site_coords(const orc_geom *g, int s, int x[4])
{
    for (int i = 0; i < 4; ++i) x[i] = 0;
    for (int i = 0; i < g->d; ++i) { x[i] = s % g->dims[i]; s /= g->dims[i]; }
}

static int coords_site(const orc_geom *g, const int x[4])
{
    int s = 0;
    for (int i = g->d - 1; i >= 0; --i) s = s * g->dims[i] + x[i];
    return s;
}

/* neighbour of s one step in direction mu (dir = +1 or -1); -1 if it
 * leaves an open lattice */
static int neighbour(const orc_geom *g, int s, int mu, int dir)
{
    int x[4];
    site_coords(g, s, x);
    x[mu] += dir;
    if (x[mu] < 0 || x[mu] >= g->dims[mu]) {
        if (!g->periodic) return -1;
        x[mu] = (x[mu] + g->dims[mu]) % g->dims[mu];
    }
    return coords_site(g, x);
}

orc_geom *orc_geom_new(int d, const int *dims, int periodic)
{
    if (d < 1 || d > 4) return NULL;
    orc_geom *g = (orc_geom *)calloc(1, sizeof(orc_geom));
    g->d = d; g->periodic = periodic; g->nsite = 1;
    for (int i = 0; i < d; ++i) { g->dims[i] = dims[i]; g->nsite *= dims[i]; }
    g->nslot = d * g->nsite;
    g->exists = (int *)calloc((size_t)g->nslot, sizeof(int));
    for (int mu = 0; mu < d; ++mu)
        for (int s = 0; s < g->nsite; ++s)
            g->exists[mu * g->nsite + s] = neighbour(g, s, mu, +1) >= 0;

    /* plaquettes (x, mu<nu): theta_mu(x) + theta_nu(x+mu) - theta_mu(x+nu) - theta_nu(x) */
    int maxp = g->nsite * d * (d - 1) / 2;
    g->plaq_link = (int *)malloc(sizeof(int) * 4 * (size_t)(maxp > 0 ? maxp : 1));
    g->plaq_sign = (int *)malloc(sizeof(int) * 4 * (size_t)(maxp > 0 ? maxp : 1));
    g->nplaq = 0;
    for (int s = 0; s < g->nsite; ++s)
        for (int mu = 0; mu < d; ++mu)
            for (int nu = mu + 1; nu < d; ++nu) {
                int xm = neighbour(g, s, mu, +1), xn = neighbour(g, s, nu, +1);
                if (xm < 0 || xn < 0) continue;
                int p = g->nplaq++;
                g->plaq_link[4 * p + 0] = mu * g->nsite + s;  g->plaq_sign[4 * p + 0] = +1;
                g->plaq_link[4 * p + 1] = nu * g->nsite + xm; g->plaq_sign[4 * p + 1] = +1;
                g->plaq_link[4 * p + 2] = mu * g->nsite + xn; g->plaq_sign[4 * p + 2] = -1;
                g->plaq_link[4 * p + 3] = nu * g->nsite + s;  g->plaq_sign[4 * p + 3] = -1;
            }

    /* link -> plaquettes */
    g->lp_start = (int *)calloc((size_t)g->nslot + 1, sizeof(int));
    for (int p = 0; p < g->nplaq; ++p)
        for (int j = 0; j < 4; ++j) g->lp_start[g->plaq_link[4 * p + j] + 1]++;
    for (int l = 0; l < g->nslot; ++l) g->lp_start[l + 1] += g->lp_start[l];
    int tot = g->lp_start[g->nslot];
    g->lp_plaq = (int *)malloc(sizeof(int) * (size_t)(tot > 0 ? tot : 1));
    g->lp_pos = (int *)malloc(sizeof(int) * (size_t)(tot > 0 ? tot : 1));
    int *fill = (int *)calloc((size_t)g->nslot, sizeof(int));
    for (int p = 0; p < g->nplaq; ++p)
        for (int j = 0; j < 4; ++j) {
            int l = g->plaq_link[4 * p + j];
            int k = g->lp_start[l] + fill[l]++;
            g->lp_plaq[k] = p; g->lp_pos[k] = j;
        }
    free(fill);

    /* checkerboard classes (mu, parity) in ascending site order */
    g->class_start = (int *)calloc(2 * (size_t)d + 1, sizeof(int));
    g->class_links = (int *)malloc(sizeof(int) * (size_t)g->nslot);
    int n = 0;
    for (int mu = 0; mu < d; ++mu)
        for (int par = 0; par < 2; ++par) {
            g->class_start[2 * mu + par] = n;
            for (int s = 0; s < g->nsite; ++s) {
                int x[4]; site_coords(g, s, x);
                int ps = 0;
                for (int i = 0; i < d; ++i) ps += x[i];
                if ((ps & 1) == par && g->exists[mu * g->nsite + s])
                    g->class_links[n++] = mu * g->nsite + s;
            }
        }
    g->class_start[2 * d] = n;
    return g;
}

void orc_geom_free(orc_geom *g)
{
    if (!g) return;
    free(g->exists); free(g->plaq_link); free(g->plaq_sign); free(g->lp_start);
    free(g->lp_plaq); free(g->lp_pos); free(g->class_start); free(g->class_links);
    free(g);
}

int orc_geom_nslot(const orc_geom *g) { return g->nslot; }
int orc_geom_nplaq(const orc_geom *g) { return g->nplaq; }
int orc_geom_nsite(const orc_geom *g) { return g->nsite; }
int orc_geom_link_exists(const orc_geom *g, int l) { return g->exists[l]; }

/* ------------------------------------------------------------------------
 * Lattice state
 * ---------------------------------------------------------------------- */
typedef struct {
    const orc_geom *g;
    double *theta;           /* [nslot] */
    double E;                /* tracked energy */
    double E_lo, dE;         /* window [E_lo, E_lo + dE] */
    uint32_t key[2];
    uint32_t sweep;          /* composite sweeps done (Philox counter word 1) */
    int n_or, block;
    double beta_up, beta_dn;
    /* statistics */
    double hb_acc, hb_tot, or_acc, or_tot, caps;
    double max_drift;        /* max |tracked - fresh| seen at a resync */
    /* scratch */
    double *prop, *dEl;
} orc_lat;

#define TAG_HB 0u
#define TAG_MUCA 12u
#define TAG_SWAP 13u
#define TAG_APPROACH 14u
#define TAG_INIT 15u
#define SAMPLER_MAX_ATTEMPTS 64
#define KAPPA_MIN 1e-6

orc_lat *orc_lat_new(const orc_geom *g, uint64_t seed, int interval_id, int replica_id,
                     double E_lo, double dE, int n_or, int block,
                     double beta_up, double beta_dn)
{
    orc_lat *t = (orc_lat *)calloc(1, sizeof(orc_lat));
    t->g = g;
    t->theta = (double *)calloc((size_t)g->nslot, sizeof(double));
    t->prop = (double *)calloc((size_t)g->nslot, sizeof(double));
    t->dEl = (double *)calloc((size_t)g->nslot, sizeof(double));
    t->E_lo = E_lo; t->dE = dE;
    t->key[0] = (uint32_t)seed ^ (uint32_t)interval_id;
    t->key[1] = (uint32_t)(seed >> 32) ^ (uint32_t)replica_id;
    t->n_or = n_or; t->block = block > 0 ? block : 1;
    t->beta_up = beta_up; t->beta_dn = beta_dn;
    return t;
}

void orc_lat_free(orc_lat *t)
{
    if (!t) return;
    free(t->theta); free(t->prop); free(t->dEl); free(t);
}

/* Fresh energy: sum over plaquettes of cos(theta_P) (Sec. 3.1). */
double orc_energy(const orc_lat *t)
{
    const orc_geom *g = t->g;
    double E = 0.0;
    for (int p = 0; p < g->nplaq; ++p) {
        double a = 0.0;
        for (int j = 0; j < 4; ++j) a += g->plaq_sign[4 * p + j] * t->theta[g->plaq_link[4 * p + j]];
        E += cos(a);
    }
    return E;
}

/* Staple angles of link l: cos(theta_P) = cos(theta_l + phi_P) for every
 * plaquette P that contains l.  Returns their number. */
static int staples(const orc_lat *t, int l, double *phi)
{
    const orc_geom *g = t->g;
    int n = 0;
    for (int k = g->lp_start[l]; k < g->lp_start[l + 1]; ++k) {
        int p = g->lp_plaq[k], pos = g->lp_pos[k];
        double rest = 0.0;
        for (int j = 0; j < 4; ++j)
            if (j != pos) rest += g->plaq_sign[4 * p + j] * t->theta[g->plaq_link[4 * p + j]];
        phi[n++] = g->plaq_sign[4 * p + pos] * rest;
    }
    return n;
}

/* local energy of link l at angle th: sum_P cos(th + phi_P) */
static double local_energy(int n, const double *phi, double th)
{
    double e = 0.0;
    for (int j = 0; j < n; ++j) e += cos(th + phi[j]);
    return e;
}

void orc_lat_set_links(orc_lat *t, const double *th)
{
    memcpy(t->theta, th, sizeof(double) * (size_t)t->g->nslot);
    t->E = orc_energy(t);
}
void orc_lat_get_links(const orc_lat *t, double *th)
{
    memcpy(th, t->theta, sizeof(double) * (size_t)t->g->nslot);
}
double orc_lat_get_E(const orc_lat *t) { return t->E; }
void orc_lat_set_E(orc_lat *t, double E) { t->E = E; }
uint32_t orc_lat_get_sweep(const orc_lat *t) { return t->sweep; }
void orc_lat_set_sweep(orc_lat *t, uint32_t s) { t->sweep = s; }
void orc_lat_set_window(orc_lat *t, double E_lo, double dE) { t->E_lo = E_lo; t->dE = dE; }
void orc_lat_stats(const orc_lat *t, double out[6])
{
    out[0] = t->hb_acc; out[1] = t->hb_tot; out[2] = t->or_acc; out[3] = t->or_tot;
    out[4] = t->caps; out[5] = t->max_drift;
}

/* Hot start: theta = -pi + 2 pi u, Haar measure (Sec. 3.1). */
void orc_lat_hot_start(orc_lat *t)
{
    const orc_geom *g = t->g;
    for (int l = 0; l < g->nslot; ++l) {
        t->theta[l] = 0.0;
        if (!g->exists[l]) continue;
        uint32_t ctr[4] = {(uint32_t)l, 0u, TAG_INIT, 0u}, w[4];
        orc_philox4x32_10(ctr, t->key, w);
        t->theta[l] = -M_PI + 2.0 * M_PI * orc_uniform(w[0]);
    }
    t->E = orc_energy(t);
}

/* Best & Fisher (1979) von Mises sampler for density ~ exp(kappa cos X).
 * Attempt t uses Philox call t/2 (counter word 3): words 0, 1 for even t and
 * words 2, 3 for odd t give u1 and u2, and the lowest bit of the attempt's
 * first word (not used by its uniform) gives the sign of X.
 * Returns the number of attempts used, or -1 if the attempt cap was hit. */
int orc_vonmises(double kappa, const uint32_t key[2], uint32_t c0, uint32_t c1, uint32_t c2,
                 double *X)
{
    if (fabs(kappa) < KAPPA_MIN) {
        uint32_t ctr[4] = {c0, c1, c2, 0u}, w[4];
        orc_philox4x32_10(ctr, key, w);
        *X = M_PI * (2.0 * orc_uniform(w[0]) - 1.0);
        return 1;
    }
    double k = fabs(kappa);
    double tau = 1.0 + sqrt(1.0 + 4.0 * k * k);
    double rho = (tau - sqrt(2.0 * tau)) / (2.0 * k);
    double r = (1.0 + rho * rho) / (2.0 * rho);
    uint32_t w[4];
    for (uint32_t att = 0; att < SAMPLER_MAX_ATTEMPTS; ++att) {
        if ((att & 1u) == 0u) {
            uint32_t ctr[4] = {c0, c1, c2, att >> 1};
            orc_philox4x32_10(ctr, key, w);
        }
        uint32_t wa = w[2 * (att & 1u)], wb = w[2 * (att & 1u) + 1];
        double u1 = orc_uniform(wa), u2 = orc_uniform(wb);
        double z = cos(M_PI * u1);
        double f = (1.0 + r * z) / (r + z);
        double c = k * (r - f);
        if (c * (2.0 - c) - u2 > 0.0 || log(c / u2) + 1.0 - c >= 0.0) {
            double x = (wa & 1u ? 1.0 : -1.0) * acos(f);
            if (kappa < 0.0) x = wrap_angle(x + M_PI);
            *X = x;
            return (int)att + 1;
        }
    }
    return -1;
}

/* Every attempt of the sampler above, accepted or not (test diagnostics):
 * for attempts 0 .. n_max-1, the variate X the attempt gives if it is taken,
 * and the two margins of its accept test, m1 = c (2 - c) - u2 and
 * m2 = ln(c / u2) + 1 - c (taken iff m1 > 0 or m2 >= 0).  A float32 sampler
 * can take a different attempt than this FP64 one only where a margin is
 * within its rounding of zero.  Returns the number of attempts written (0
 * for the uniform proposal at |kappa| < 1e-6). */
int orc_vonmises_attempts(double kappa, const uint32_t key[2], uint32_t c0, uint32_t c1,
                          uint32_t c2, int n_max, double *X, double *m1, double *m2)
{
    if (fabs(kappa) < KAPPA_MIN) return 0;
    double k = fabs(kappa);
    double tau = 1.0 + sqrt(1.0 + 4.0 * k * k);
    double rho = (tau - sqrt(2.0 * tau)) / (2.0 * k);
    double r = (1.0 + rho * rho) / (2.0 * rho);
    uint32_t w[4];
    int n = n_max < SAMPLER_MAX_ATTEMPTS ? n_max : SAMPLER_MAX_ATTEMPTS;
    for (int att = 0; att < n; ++att) {
        if ((att & 1) == 0) {
            uint32_t ctr[4] = {c0, c1, c2, (uint32_t)att >> 1};
            orc_philox4x32_10(ctr, key, w);
        }
        uint32_t wa = w[2 * (att & 1)], wb = w[2 * (att & 1) + 1];
        double u1 = orc_uniform(wa), u2 = orc_uniform(wb);
        double z = cos(M_PI * u1);
        double f = (1.0 + r * z) / (r + z);
        double c = k * (r - f);
        double x = (wa & 1u ? 1.0 : -1.0) * acos(f);
        if (kappa < 0.0) x = wrap_angle(x + M_PI);
        X[att] = x;
        m1[att] = c * (2.0 - c) - u2;
        m2[att] = log(c / u2) + 1.0 - c;
    }
    return n;
}

static double dist_to_window(double E, double lo, double hi)
{
    if (E < lo) return lo - E;
    if (E > hi) return E - hi;
    return 0.0;
}

/* The window decision of one block of a group (R2, R19).  Heat-bath (mode
 * 0): taken iff dist(E + d) <= dist(E), E the running energy.  Overrelaxation
 * (mode 1): the reflection keeps E in exact arithmetic, so outside the window
 * it is always taken and inside it is taken iff E + d stays inside, E being
 * the energy before the pass (overrelaxation does not move the running
 * energy).  Inside the window both are the indicator of eq. (2.13). */
static int block_taken(int mode, double E, double d, double lo, double hi)
{
    if (mode == 1) return dist_to_window(E, lo, hi) > 0.0 || dist_to_window(E + d, lo, hi) == 0.0;
    return dist_to_window(E + d, lo, hi) <= dist_to_window(E, lo, hi);
}

/* Largest |dE| an overrelaxation move may carry (R19): 2^-14.  A reflection
 * changes E only by rounding; a move beyond the bound is refused (a guard for
 * float32 arithmetic that FP64 never reaches). */
#define OR_DELTA_MAX 6.103515625e-05

/* Index range of class cls's links (in update order) that lie in slab sl,
 * the sites whose last coordinate x_{d-1} equals sl.  The class lists are in
 * ascending site order, which is slab-major. */
static void slab_range(const orc_geom *g, int cls, int sl, int *b, int *e)
{
    int c0 = g->class_start[cls], c1 = g->class_start[cls + 1];
    int per_slab = g->nsite / g->dims[g->d - 1];
    int i = c0;
    while (i < c1 && (g->class_links[i] % g->nsite) / per_slab < sl) ++i;
    *b = i;
    while (i < c1 && (g->class_links[i] % g->nsite) / per_slab == sl) ++i;
    *e = i;
}

/* Update the links class_links[c0 .. c1) of one class.  mode 0: heat-bath at
 * parameter a with Philox tag `tag`; mode 1: overrelaxation.  Window-accept
 * blocks of B links start at c0. */
static void group_update(orc_lat *t, int c0, int c1, int mode, double a, uint32_t tag)
{
    const orc_geom *g = t->g;
    double phi[8];
    double lo = t->E_lo, hi = t->E_lo + t->dE;
    /* proposals: independent for all links of the group */
    for (int i = c0; i < c1; ++i) {
        int l = g->class_links[i];
        int n = staples(t, l, phi);
        double Sr = 0.0, Si = 0.0;
        for (int j = 0; j < n; ++j) { Sr += cos(phi[j]); Si += sin(phi[j]); }
        double alpha = atan2(Si, Sr), Sabs = sqrt(Sr * Sr + Si * Si);
        double th = t->theta[l], thn;
        if (mode == 0) {
            double X;
            int att = orc_vonmises(-a * Sabs, t->key, (uint32_t)l, t->sweep, tag, &X);
            if (att < 0) { thn = th; t->caps += 1.0; }
            else thn = wrap_angle(X - alpha);
        } else {
            thn = wrap_angle(-th - 2.0 * alpha);
        }
        t->prop[l] = thn;
        t->dEl[l] = local_energy(n, phi, thn) - local_energy(n, phi, th);
        if (mode == 1 && fabs(t->dEl[l]) > OR_DELTA_MAX) { t->prop[l] = th; t->dEl[l] = 0.0; }
    }
    /* sequential Metropolis accept in blocks of B links, update order */
    for (int b0 = c0; b0 < c1; b0 += t->block) {
        int b1 = b0 + t->block < c1 ? b0 + t->block : c1;
        double d = 0.0;
        for (int i = b0; i < b1; ++i) d += t->dEl[g->class_links[i]];
        int acc = block_taken(mode, t->E, d, lo, hi);
        if (acc) {
            for (int i = b0; i < b1; ++i) t->theta[g->class_links[i]] = t->prop[g->class_links[i]];
            if (mode == 0) t->E += d;   /* R19: overrelaxation leaves the running energy */
        }
        if (mode == 0) { t->hb_tot += b1 - b0; if (acc) t->hb_acc += b1 - b0; }
        else           { t->or_tot += b1 - b0; if (acc) t->or_acc += b1 - b0; }
    }
}

/* The groups of one class in update order: a heat-bath pass takes the whole
 * class as one group, an overrelaxation pass one group per slab. */
static int class_groups(const orc_geom *g, int cls, int mode, int *b, int *e)
{
    if (mode == 0) {
        b[0] = g->class_start[cls];
        e[0] = g->class_start[cls + 1];
        return 1;
    }
    int ns = g->dims[g->d - 1];
    for (int sl = 0; sl < ns; ++sl) slab_range(g, cls, sl, &b[sl], &e[sl]);
    return ns;
}

static void class_pass(orc_lat *t, int cls, int mode, double a, uint32_t tag)
{
    int b[64], e[64];
    int n = class_groups(t->g, cls, mode, b, e);
    for (int k = 0; k < n; ++k) group_update(t, b[k], e[k], mode, a, tag);
}

/* The same class update as class_pass, recording for every link of the
 * class (in update order) its old angle, its proposal, the energy before its
 * block, the block's dE and whether the block was accepted (test
 * diagnostics: how close a window decision was to a tie). */
int orc_lat_class_trace(orc_lat *t, int cls, int mode, double a, double *th_old, double *th_prop,
                        double *E_before, double *dE_block, int *accepted)
{
    const orc_geom *g = t->g;
    if (cls < 0 || cls >= 2 * g->d) return 0;
    int c0 = g->class_start[cls], c1 = g->class_start[cls + 1];
    for (int i = c0; i < c1; ++i) th_old[i - c0] = t->theta[g->class_links[i]];
    double lo = t->E_lo, hi = t->E_lo + t->dE;
    /* replay the decisions of class_pass on a copy of the energy */
    double E = t->E;
    class_pass(t, cls, mode, a, TAG_HB);
    int gb[64], ge[64];
    int ng = class_groups(g, cls, mode, gb, ge);
    for (int k = 0; k < ng; ++k) {
        int g0 = gb[k], g1 = ge[k];
        for (int b0 = g0; b0 < g1; b0 += t->block) {
            int b1 = b0 + t->block < g1 ? b0 + t->block : g1;
            double d = 0.0;
            for (int i = b0; i < b1; ++i) d += t->dEl[g->class_links[i]];
            int acc = block_taken(mode, E, d, lo, hi);
            for (int i = b0; i < b1; ++i) {
                th_prop[i - c0] = t->prop[g->class_links[i]];
                E_before[i - c0] = E;
                dE_block[i - c0] = d;
                accepted[i - c0] = acc;
            }
            if (acc && mode == 0) E += d;
        }
    }
    return c1 - c0;
}

/* One pass.  Heat-bath: the classes in the order mu = 0..d-1, parity 0,1,
 * each over the whole lattice.  Overrelaxation: slab by slab (last
 * coordinate), and within a slab the classes in the same order. */
static void pass(orc_lat *t, int mode, double a, uint32_t tag)
{
    const orc_geom *g = t->g;
    if (mode == 0) {
        for (int cls = 0; cls < 2 * g->d; ++cls) class_pass(t, cls, mode, a, tag);
        return;
    }
    for (int sl = 0; sl < g->dims[g->d - 1]; ++sl)
        for (int cls = 0; cls < 2 * g->d; ++cls) {
            int b, e;
            slab_range(g, cls, sl, &b, &e);
            group_update(t, b, e, mode, a, tag);
        }
}

/* One composite sweep: heat-bath pass + n_or overrelaxation passes, then
 * re-synchronise the tracked energy with the fresh plaquette sum. */
static void composite_sweep(orc_lat *t, double a, uint32_t tag)
{
    pass(t, 0, a, tag);
    for (int k = 0; k < t->n_or; ++k) pass(t, 1, a, tag);
    double fresh = orc_energy(t);
    double drift = fabs(fresh - t->E);
    if (drift > t->max_drift) t->max_drift = drift;
    t->E = fresh;
    t->sweep += 1u;
}

void orc_lat_sweep(orc_lat *t, double a, int n_sweeps)
{
    for (int s = 0; s < n_sweeps; ++s) composite_sweep(t, a, TAG_HB);
}

/* only the heat-bath pass or only an overrelaxation pass (no resync) */
void orc_lat_pass(orc_lat *t, int mode, double a)
{
    pass(t, mode, a, TAG_HB);
}

/* a single class (cls = 2 mu + parity), no resync */
void orc_lat_class_pass(orc_lat *t, int cls, int mode, double a)
{
    if (cls >= 0 && cls < 2 * t->g->d) class_pass(t, cls, mode, a, TAG_HB);
}

/* Approach the window from the current state (reading R5).  Returns the
 * number of composite sweeps used, or -1 if the window was not reached. */
int orc_lat_approach(orc_lat *t, int max_sweeps)
{
    double lo = t->E_lo, hi = t->E_lo + t->dE;
    int s = 0;
    while (dist_to_window(t->E, lo, hi) > 0.0) {
        if (s >= max_sweeps) return -1;
        double a = t->E < lo ? -t->beta_up : -t->beta_dn;
        composite_sweep(t, a, TAG_APPROACH);
        ++s;
    }
    return s;
}

/* One Robbins-Monro iteration (Algorithm 1 inner loop, eq. (2.30)):
 * n_therm + n_meas composite sweeps at weight exp(-a E); the mean of
 * E - E_lo - dE/2 over the last n_meas sweeps gives <<dE>>; then
 * a <- a + 12 <<dE>> / (dE^2 (rm_index + 1)).  Returns the new a. */
double orc_lat_rm_step(orc_lat *t, double a, int n_therm, int n_meas, int rm_index,
                       double *mean_out)
{
    double sum = 0.0;
    for (int j = 0; j < n_therm + n_meas; ++j) {
        composite_sweep(t, a, TAG_HB);
        if (j >= n_therm) sum += t->E - t->E_lo - 0.5 * t->dE;
    }
    double mean = n_meas > 0 ? sum / n_meas : 0.0;
    if (mean_out) *mean_out = mean;
    return a + 12.0 * mean / (t->dE * t->dE * (double)(rm_index + 1));
}

/* Replica exchange between overlapping intervals (Sec. 2.5).  For each pair
 * (I1, I2) = (pairs[2k], pairs[2k+1]), in order: when the current energies
 * E1, E2 of both configurations lie in the common part of the two closed
 * windows, the configurations are exchanged with probability
 * min(1, exp((a_I1 - a_I2)(E1 - E2))), the Metropolis probability of the
 * swap under the product of the two restricted weights exp(-a E).  An
 * exchange moves the link angles and the tracked energy; the window, the
 * slope, the Philox key and the sweep counter stay with the interval.
 * a: slopes a^(n) indexed like lats.  accepted (nullable): 1 per exchanged
 * pair.  Returns the number of exchanges. */
int orc_replica_exchange(orc_lat **lats, int n_pairs, const int *pairs, const double *a,
                         uint32_t round, int *accepted)
{
    int n_acc = 0;
    for (int k = 0; k < n_pairs; ++k) {
        int i1 = pairs[2 * k], i2 = pairs[2 * k + 1];
        orc_lat *t1 = lats[i1], *t2 = lats[i2];
        double lo = fmax(t1->E_lo, t2->E_lo);
        double hi = fmin(t1->E_lo + t1->dE, t2->E_lo + t2->dE);
        int acc = 0;
        if (t1->E >= lo && t1->E <= hi && t2->E >= lo && t2->E <= hi) {
            double x = (a[i1] - a[i2]) * (t1->E - t2->E);
            uint32_t ctr[4] = {0u, round, TAG_SWAP, 0u}, w[4];
            orc_philox4x32_10(ctr, t1->key, w);
            double u = ((double)(w[0] >> 11) * 4294967296.0 + (double)w[1]) *
                       (1.0 / 9007199254740992.0);
            acc = x >= 0.0 || u < exp(x);
        }
        if (acc) {
            double *th = t1->theta; t1->theta = t2->theta; t2->theta = th;
            double E = t1->E; t1->E = t2->E; t2->E = E;
        }
        if (accepted) accepted[k] = acc;
        n_acc += acc;
    }
    return n_acc;
}

/* ------------------------------------------------------------------------
 * Multicanonical update (Sec. 2.6, eq. (2.50)).  ln rho~ at the edges of n
 * contiguous intervals of width de from e0: lnr[0] = 0,
 * lnr[k+1] = lnr[k] + a_k de (eq. (2.10)), linear with slope a_k inside
 * interval k and with the first / last slope beyond the ends.
 * ---------------------------------------------------------------------- */
typedef struct {
    int n;
    double e0, de;
    double *lnr, *a;
} orc_muca;

orc_muca *orc_muca_new(int n, double e0, double de, const double *a)
{
    if (n < 1 || !(de > 0.0)) return NULL;
    orc_muca *m = (orc_muca *)calloc(1, sizeof(orc_muca));
    m->n = n; m->e0 = e0; m->de = de;
    m->lnr = (double *)calloc((size_t)n + 1, sizeof(double));
    m->a = (double *)calloc((size_t)n, sizeof(double));
    for (int k = 0; k < n; ++k) {
        m->a[k] = a[k];
        m->lnr[k + 1] = m->lnr[k] + a[k] * de;
    }
    return m;
}

void orc_muca_free(orc_muca *m)
{
    if (!m) return;
    free(m->lnr); free(m->a); free(m);
}

double orc_muca_lnrho(const orc_muca *m, double E)
{
    int k = (int)floor((E - m->e0) / m->de);
    if (k < 0) k = 0;
    if (k > m->n - 1) k = m->n - 1;
    return m->lnr[k] + m->a[k] * (E - (m->e0 + k * m->de));
}

/* One class of a multicanonical heat-bath pass: proposals as in
 * group_update (heat-bath at slope a0, tag TAG_HB), then Metropolis-Hastings
 * for the weight 1/rho~ in link order.  Optional trace per link (update
 * order): energy before, dE, u, exponent, accepted. */
static void muca_class(orc_lat *t, const orc_muca *m, int cls, double a0, double *tr_E,
                       double *tr_dE, double *tr_u, double *tr_x, int *tr_acc)
{
    const orc_geom *g = t->g;
    int c0 = g->class_start[cls], c1 = g->class_start[cls + 1];
    double phi[8];
    for (int i = c0; i < c1; ++i) {
        int l = g->class_links[i];
        int n = staples(t, l, phi);
        double Sr = 0.0, Si = 0.0;
        for (int j = 0; j < n; ++j) { Sr += cos(phi[j]); Si += sin(phi[j]); }
        double alpha = atan2(Si, Sr), Sabs = sqrt(Sr * Sr + Si * Si);
        double th = t->theta[l], thn, X;
        int att = orc_vonmises(-a0 * Sabs, t->key, (uint32_t)l, t->sweep, TAG_HB, &X);
        if (att < 0) { thn = th; t->caps += 1.0; }
        else thn = wrap_angle(X - alpha);
        t->prop[l] = thn;
        t->dEl[l] = local_energy(n, phi, thn) - local_energy(n, phi, th);
    }
    for (int i = c0; i < c1; ++i) {
        int l = g->class_links[i];
        double d = t->dEl[l];
        double x = a0 * d - (orc_muca_lnrho(m, t->E + d) - orc_muca_lnrho(m, t->E));
        uint32_t ctr[4] = {(uint32_t)l, t->sweep, TAG_MUCA, 0u}, w[4];
        orc_philox4x32_10(ctr, t->key, w);
        double u = orc_uniform(w[0]);
        int acc = u < exp(x);
        if (tr_E) {
            tr_E[i - c0] = t->E; tr_dE[i - c0] = d; tr_u[i - c0] = u; tr_x[i - c0] = x;
            tr_acc[i - c0] = acc;
        }
        if (acc) { t->theta[l] = t->prop[l]; t->E += d; t->hb_acc += 1.0; }
        t->hb_tot += 1.0;
    }
}

/* n composite multicanonical sweeps: heat-bath pass (classes in order),
 * n_or overrelaxation passes (always taken), fresh-energy resync.  E_out
 * (nullable) receives the energy after each sweep. */
void orc_lat_muca_sweep(orc_lat *t, const orc_muca *m, double a0, int n_sweeps, double *E_out)
{
    const orc_geom *g = t->g;
    double lo = t->E_lo, w = t->dE;
    for (int s = 0; s < n_sweeps; ++s) {
        for (int cls = 0; cls < 2 * g->d; ++cls) muca_class(t, m, cls, a0, 0, 0, 0, 0, 0);
        t->E_lo = -1e300; t->dE = 2e300;   /* overrelaxation keeps E: no window */
        for (int k = 0; k < t->n_or; ++k) pass(t, 1, 0.0, TAG_HB);
        t->E_lo = lo; t->dE = w;
        double fresh = orc_energy(t);
        double drift = fabs(fresh - t->E);
        if (drift > t->max_drift) t->max_drift = drift;
        t->E = fresh;
        t->sweep += 1u;
        if (E_out) E_out[s] = t->E;
    }
}

/* One multicanonical heat-bath class with its per-link trace (tests);
 * returns the number of links of the class. */
int orc_lat_muca_class_trace(orc_lat *t, const orc_muca *m, int cls, double a0, double *E_before,
                             double *dE, double *u, double *x, int *accepted)
{
    if (cls < 0 || cls >= 2 * t->g->d) return 0;
    muca_class(t, m, cls, a0, E_before, dE, u, x, accepted);
    return t->g->class_start[cls + 1] - t->g->class_start[cls];
}

/* Per-link staple modulus |S| and angle alpha (for invariance checks). */
void orc_lat_staple(const orc_lat *t, int l, double out[2])
{
    double phi[8];
    int n = staples(t, l, phi);
    double Sr = 0.0, Si = 0.0;
    for (int j = 0; j < n; ++j) { Sr += cos(phi[j]); Si += sin(phi[j]); }
    out[0] = sqrt(Sr * Sr + Si * Si);
    out[1] = atan2(Si, Sr);
}

/* |S| of every link slot (0 where the link does not exist). */
void orc_lat_staple_moduli(const orc_lat *t, double *out)
{
    double st[2];
    for (int l = 0; l < t->g->nslot; ++l) {
        out[l] = 0.0;
        if (!t->g->exists[l]) continue;
        orc_lat_staple(t, l, st);
        out[l] = st[0];
    }
}

/* ------------------------------------------------------------------------
 * Whole LLR runs over many independent (interval, replica) lattices, each
 * on its own thread: hot start, approach, then n_rm Robbins-Monro
 * iterations (Algorithm 1).  Used for CPU timing and statistical tests.
 * ---------------------------------------------------------------------- */
typedef struct {
    const orc_geom *g;
    int n_lat, n_threads, next_index;
    uint64_t seed;
    const int *interval_id, *replica_id;
    const double *E_lo, *dE;
    double *a;               /* [n_lat] in: a^(0); out: final a */
    double *a_hist;          /* [n_lat][n_rm] or NULL */
    int n_or, block, n_therm, n_meas, n_rm, rm_offset, max_approach;
    double beta_up, beta_dn;
    int *status;             /* [n_lat] 0 ok, -1 window not reached */
    double *updates;         /* [n_lat] link updates done */
} orc_batch;

static void *batch_worker(void *arg)
{
    void **pa = (void **)arg;
    orc_batch *b = (orc_batch *)pa[0];
    int tid = (int)(intptr_t)pa[1];
    for (int i = tid; i < b->n_lat; i += b->n_threads) {
        orc_lat *t = orc_lat_new(b->g, b->seed, b->interval_id[i], b->replica_id[i], b->E_lo[i],
                                 b->dE[i], b->n_or, b->block, b->beta_up, b->beta_dn);
        orc_lat_hot_start(t);
        int used = orc_lat_approach(t, b->max_approach);
        b->status[i] = used < 0 ? -1 : 0;
        double a = b->a[i];
        if (used >= 0)
            for (int n = 0; n < b->n_rm; ++n) {
                a = orc_lat_rm_step(t, a, b->n_therm, b->n_meas, n + b->rm_offset, NULL);
                if (b->a_hist) b->a_hist[(size_t)i * b->n_rm + n] = a;
            }
        b->a[i] = a;
        double per_sweep = 0.0;
        for (int l = 0; l < b->g->nslot; ++l) per_sweep += b->g->exists[l];
        b->updates[i] = per_sweep * (1 + b->n_or) * ((double)t->sweep);
        orc_lat_free(t);
    }
    return NULL;
}

int orc_batch_run(const orc_geom *g, int n_lat, uint64_t seed, const int *interval_id,
                  const int *replica_id, const double *E_lo, const double *dE, double *a,
                  double *a_hist, int n_or, int block, int n_therm, int n_meas, int n_rm,
                  int rm_offset, int max_approach, double beta_up, double beta_dn,
                  int n_threads, int *status, double *updates)
{
    orc_batch b = {g, n_lat, n_threads > 0 ? n_threads : 1, 0, seed, interval_id, replica_id,
                   E_lo, dE, a, a_hist, n_or, block, n_therm, n_meas, n_rm, rm_offset,
                   max_approach, beta_up, beta_dn, status, updates};
    pthread_t th[256];
    void *args[256][2];
    int nt = b.n_threads > 256 ? 256 : b.n_threads;
    b.n_threads = nt;
    for (int i = 0; i < nt; ++i) {
        args[i][0] = &b; args[i][1] = (void *)(intptr_t)i;
        pthread_create(&th[i], NULL, batch_worker, args[i]);
    }
    for (int i = 0; i < nt; ++i) pthread_join(th[i], NULL);
    return 0;
}

/* Run n_sweeps composite sweeps at slope a[i] on existing lattices, one
 * host thread per lattice group (CPU timing of the same work). */
typedef struct {
    orc_lat **lats;
    const double *a;
    int n, n_sweeps, n_threads, tid;
} orc_sweeps_job;

static void *sweeps_worker(void *arg)
{
    orc_sweeps_job *j = (orc_sweeps_job *)arg;
    for (int i = j->tid; i < j->n; i += j->n_threads) orc_lat_sweep(j->lats[i], j->a[i], j->n_sweeps);
    return NULL;
}

void orc_batch_sweeps(orc_lat **lats, const double *a, int n, int n_sweeps, int n_threads)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    orc_sweeps_job jobs[256];
    for (int t = 0; t < n_threads; ++t) {
        jobs[t].lats = lats; jobs[t].a = a; jobs[t].n = n; jobs[t].n_sweeps = n_sweeps;
        jobs[t].n_threads = n_threads; jobs[t].tid = t;
        pthread_create(&th[t], NULL, sweeps_worker, &jobs[t]);
    }
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
}

/* approach on existing lattices in parallel; status[i] = sweeps used or -1 */
typedef struct {
    orc_lat **lats;
    int *status;
    int n, max_sweeps, n_threads, tid;
} orc_approach_job;

static void *approach_worker(void *arg)
{
    orc_approach_job *j = (orc_approach_job *)arg;
    for (int i = j->tid; i < j->n; i += j->n_threads)
        j->status[i] = orc_lat_approach(j->lats[i], j->max_sweeps);
    return NULL;
}

void orc_batch_approach(orc_lat **lats, int *status, int n, int max_sweeps, int n_threads)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    orc_approach_job jobs[256];
    for (int t = 0; t < n_threads; ++t) {
        jobs[t].lats = lats; jobs[t].status = status; jobs[t].n = n;
        jobs[t].max_sweeps = max_sweeps; jobs[t].n_threads = n_threads; jobs[t].tid = t;
        pthread_create(&th[t], NULL, approach_worker, &jobs[t]);
    }
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
}
