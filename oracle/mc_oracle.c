/*
 * mc_oracle.c -- plain, slow FP64 CPU oracle of the Monte Carlo packet
 * transport of Kerzendorf & Sim (2014), Sects. 2.3-2.8.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file's library.  It shares no
 * code, header, table or constant with the CUDA library: everything below is
 * written from the paper's text (and, where the paper is silent, from the
 * readings listed in the design notes), one step after another, in the
 * paper's order and notation.
 *
 * Units are CGS at the interface.  Internally a radius is carried as
 * x = r / (c t_exp), so that in homologous expansion v/c = x and the Doppler
 * factor of Sect. 2.5 is D = 1 - mu x.  Path lengths are in the same unit;
 * an optical depth per unit x is kappa' = sigma_T n_e c t_exp.
 *
 * Floating point: IEEE binary64 with +, -, *, / and sqrt only (each
 * correctly rounded), compiled without FMA contraction.  The logarithm and
 * exponential are this file's own series (named below), so that the result
 * of every operation is fixed by its operands.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------ constants */
/* CODATA 2018, CGS. */
#define C_LIGHT 2.99792458e10        /* cm s^-1 */
#define H_PLANCK 6.62607015e-27      /* erg s */
#define K_BOLTZ 1.380649e-16         /* erg K^-1 */
#define SIGMA_SB 5.670374419e-5      /* erg cm^-2 s^-1 K^-4 */
#define SIGMA_T 6.6524587321e-25     /* cm^2 */
#define M_ELECTRON 9.1093837015e-28  /* g */
#define E_CHARGE 4.803204712570263e-10 /* esu */
#define EV_ERG 1.602176634e-12       /* erg */
#define PI_D 3.14159265358979323846
#define ZETA5 1.0369277551433699263  /* Riemann zeta(5) */

#define ORC_INF (1.0 / 0.0)

/* packet fates */
#define ORC_IN_FLIGHT 0
#define ORC_ESCAPED 1
#define ORC_REABSORBED 2
#define ORC_CAPPED 3

/* per-packet counters */
#define ORC_CNT_SEGMENTS 0
#define ORC_CNT_LINE_CHECKS 1
#define ORC_CNT_RESONANCES 2
#define ORC_CNT_LINE_INTERACTIONS 3
#define ORC_CNT_E_SCATTERS 4
#define ORC_CNT_SHELL_CROSSINGS 5
#define ORC_NCOUNT 6

/* run statistics */
#define ORC_ST_ESCAPED 0
#define ORC_ST_REABSORBED 1
#define ORC_ST_CAPPED 2
#define ORC_ST_SEGMENTS 3
#define ORC_ST_LINE_CHECKS 4
#define ORC_ST_RESONANCES 5
#define ORC_ST_LINE_INTERACTIONS 6
#define ORC_ST_E_SCATTERS 7
#define ORC_ST_SHELL_CROSSINGS 8
#define ORC_NSTATS 9

/* ------------------------------------------------------------ Philox4x32-10
 * Counter-based generator of Salmon, Moraes, Dror & Shaw (SC'11, "Parallel
 * random numbers: as easy as 1, 2, 3"): ten rounds, each two 32x32->64
 * multiplications whose halves are mixed with the other counter words and
 * the round key; the key is bumped by the two Weyl constants after each
 * round.  Key = (seed low 32 bits, seed high 32 bits); counter = (block,
 * packet id, iteration, stream).
 */
static void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Draw stream of one packet: uniform number d uses Philox block d/2, words
 * (0,1) when d is even and (2,3) when d is odd; u53 = (wa >> 5) 2^26 + (wb >> 6). */
typedef struct {
    uint32_t key[2];
    uint32_t packet, iteration, stream;
    uint32_t d;
    uint32_t cached_block;
    int have_block;
    uint32_t words[4];
} orc_rng;

static void rng_init(orc_rng *r, uint64_t seed, uint32_t iteration, uint32_t packet, uint32_t stream)
{
    r->key[0] = (uint32_t)seed;
    r->key[1] = (uint32_t)(seed >> 32);
    r->packet = packet;
    r->iteration = iteration;
    r->stream = stream;
    r->d = 0;
    r->have_block = 0;
    r->cached_block = 0;
}

static uint64_t rng_next_u53(orc_rng *r)
{
    uint32_t block = r->d >> 1;
    if (!r->have_block || r->cached_block != block) {
        uint32_t ctr[4] = {block, r->packet, r->iteration, r->stream};
        philox4x32_10(ctr, r->key, r->words);
        r->cached_block = block;
        r->have_block = 1;
    }
    uint32_t wa, wb;
    if ((r->d & 1u) == 0) { wa = r->words[0]; wb = r->words[1]; }
    else { wa = r->words[2]; wb = r->words[3]; }
    r->d += 1;
    return ((uint64_t)(wa >> 5) << 26) | (uint64_t)(wb >> 6);
}

/* z in (0, 1] */
static double rng_open0(orc_rng *r) { return (double)(rng_next_u53(r) + 1) * 0x1.0p-53; }
/* z in [0, 1) */
static double rng_closed0(orc_rng *r) { return (double)rng_next_u53(r) * 0x1.0p-53; }

/* ------------------------------------------------------------ ln and exp
 * Natural logarithm by the series ln m = 2 atanh(s), s = (m-1)/(m+1)
 * (Abramowitz & Stegun 4.1.27), after reducing x = m 2^e with m in
 * [sqrt(1/2), sqrt(2)]; ln 2 is split into a 32-bit head and a tail so that
 * e * head is exact.  Valid for finite normal x > 0.
 */
#define LN2_HEAD 0x1.62e42fee00000p-1
#define LN2_TAIL 0x1.a39ef35793c76p-33
#define SQRT2_D 0x1.6a09e667f3bcdp+0
#define INV_LN2 0x1.71547652b82fep+0

double orc_log(double x)
{
    uint64_t b;
    memcpy(&b, &x, 8);
    int e = (int)((b >> 52) & 0x7ffu) - 1023;
    uint64_t mb = (b & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;
    double m;
    memcpy(&m, &mb, 8);
    if (m > SQRT2_D) { m = m * 0.5; e = e + 1; }
    double s = (m - 1.0) / (m + 1.0);
    double s2 = s * s;
    double p = 1.0 / 23.0;
    p = p * s2 + 1.0 / 21.0;
    p = p * s2 + 1.0 / 19.0;
    p = p * s2 + 1.0 / 17.0;
    p = p * s2 + 1.0 / 15.0;
    p = p * s2 + 1.0 / 13.0;
    p = p * s2 + 1.0 / 11.0;
    p = p * s2 + 1.0 / 9.0;
    p = p * s2 + 1.0 / 7.0;
    p = p * s2 + 1.0 / 5.0;
    p = p * s2 + 1.0 / 3.0;
    double two_s = 2.0 * s;
    double ln_m = two_s + two_s * (s2 * p);
    double de = (double)e;
    return de * LN2_HEAD + (de * LN2_TAIL + ln_m);
}

/* Exponential: Cody & Waite (1980) reduction x = n ln2 + r, |r| <= ln2/2,
 * then the Taylor series of e^r to degree 14, scaled by 2^n through the
 * exponent field.  Returns 0 below -708 (no subnormal results). */
double orc_exp(double x)
{
    if (x < -708.0) return 0.0;
    if (x > 709.0) return ORC_INF;
    double n = floor(x * INV_LN2 + 0.5);
    double r = (x - n * LN2_HEAD) - n * LN2_TAIL;
    double p = 1.0 / 87178291200.0;     /* 1/14! */
    p = p * r + 1.0 / 6227020800.0;     /* 1/13! */
    p = p * r + 1.0 / 479001600.0;
    p = p * r + 1.0 / 39916800.0;
    p = p * r + 1.0 / 3628800.0;
    p = p * r + 1.0 / 362880.0;
    p = p * r + 1.0 / 40320.0;
    p = p * r + 1.0 / 5040.0;
    p = p * r + 1.0 / 720.0;
    p = p * r + 1.0 / 120.0;
    p = p * r + 1.0 / 24.0;
    p = p * r + 1.0 / 6.0;
    p = p * r + 0.5;
    p = p * r + 1.0;
    p = p * r + 1.0;
    int ni = (int)n;
    if (ni < -1022) {                    /* split the scale to stay normal */
        uint64_t half_b = (uint64_t)(ni / 2 + 1023) << 52;
        uint64_t rest_b = (uint64_t)(ni - ni / 2 + 1023) << 52;
        double h, q;
        memcpy(&h, &half_b, 8);
        memcpy(&q, &rest_b, 8);
        return (p * h) * q;
    }
    uint64_t sb = (uint64_t)(ni + 1023) << 52;
    double scale;
    memcpy(&scale, &sb, 8);
    return p * scale;
}

void orc_log_array(int64_t n, const double *in, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_log(in[i]);
}

void orc_exp_array(int64_t n, const double *in, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_exp(in[i]);
}

/* ------------------------------------------------------------ Planck sampling
 * Comoving frequencies of injected packets follow B_nu(T_inner) (Sect. 2.4,
 * Eq. 10 and the text after it).  Sampling follows Carter & Cashwell (1975)
 * (also Bjorkman & Wood 2001): pick the series index l as the smallest l with
 * (90/pi^4) sum_{j<=l} j^-4 >= z0, then xi = -ln(z1 z2 z3 z4) / l and
 * nu = (k T / h) xi.  The partial sums are tabulated up to l = 1024. */
#define PLANCK_LMAX 1024
static double planck_cdf[PLANCK_LMAX + 1];
static int planck_ready = 0;
static pthread_mutex_t planck_lock = PTHREAD_MUTEX_INITIALIZER;

static void planck_table_init(void)
{
    pthread_mutex_lock(&planck_lock);
    if (!planck_ready) {
        double norm = 90.0 / (PI_D * PI_D * PI_D * PI_D);
        double s = 0.0;
        planck_cdf[0] = 0.0;
        for (int l = 1; l <= PLANCK_LMAX; ++l) {
            double dl = (double)l;
            s = s + 1.0 / (dl * dl * dl * dl);
            planck_cdf[l] = norm * s;
        }
        planck_ready = 1;
    }
    pthread_mutex_unlock(&planck_lock);
}

/* xi = h nu / (k T) for the five given uniforms */
static double planck_xi(double z0, double z1, double z2, double z3, double z4)
{
    int l = PLANCK_LMAX;
    for (int i = 1; i <= PLANCK_LMAX; ++i) {
        if (planck_cdf[i] >= z0) { l = i; break; }
    }
    double prod = ((z1 * z2) * z3) * z4;
    return -orc_log(prod) / (double)l;
}

/* ------------------------------------------------------------ model */
typedef struct {
    int32_t n_shells;
    const double *v_inner, *v_outer, *n_e; /* [S] cm/s, cm/s, cm^-3 */
    double t_exp;                          /* s */
    int32_t n_lines;
    const double *nu;                      /* [L] Hz, strictly descending */
    const double *tau;                     /* [S*L] shell-major Sobolev depths */
    int32_t line_mode;                     /* 0 scatter, 1 downbranch, 2 macro atom */
    const int32_t *line_row;               /* [L] branching row of each line (downbranch) */
    const uint32_t *dbr_offset;            /* [rows+1] */
    const uint32_t *dbr_line;              /* [nnz] emitting line of each entry */
    const double *dbr_cdf;                 /* [nnz] cumulative branching ratio */
    int32_t j_blue;                        /* 1: collect J_blue estimators */
    int32_t spec_bins;
    double spec_nu_lo, spec_nu_hi;
    uint64_t max_segments;
    double delta_t;                        /* s */
    int32_t n_virtual;                     /* N_v virtual packets per launch (Sect. 2.9), 0 = off */
    double tau_v_max;                      /* drop a v-packet once tau_v exceeds this (0 = never) */
    /* macro-atom internal jumps (line_mode 2), rows as the branching table */
    const double *ma_jump_p;               /* [rows] probability that the level jumps */
    const uint32_t *ma_jump_offset;        /* [rows+1] */
    const int32_t *ma_jump_target;         /* [n] level (row) jumped to */
    const double *ma_jump_cdf;             /* [n] cumulative target probability */
} orc_model;

typedef struct {
    double *j_est;      /* [S] sum E_cmf l D, l in units of c t_exp */
    double *nu_bar;     /* [S] sum E_cmf nu_cmf l D */
    double *j_blue;     /* [S*L] sum E_lab D_res^2 / nu_line, or NULL */
    double *spectrum;   /* [bins+2] sum E_lab per bin, then underflow, overflow */
    uint64_t stats[ORC_NSTATS];
    /* optional per-packet records, indexed from the first packet of the call */
    int32_t *status;
    double *nu_out;     /* lab frequency at the end */
    double *e_out;      /* lab energy at the end */
    uint64_t *counters; /* [count * ORC_NCOUNT] */
    double *spectrum_v; /* [bins+2] sum E_v,lab exp(-tau_v) per bin (Eq. 21), or NULL */
} orc_result;

/* Per-event trace for the invariant tests (small runs only). */
typedef struct {
    int32_t kind;        /* 1 electron, 2 line, 3 shell crossing, 4 escape, 5 reabsorb */
    int32_t line;        /* absorbing line (line events) */
    int32_t emit;        /* emitting line (line events) */
    int32_t shell;
    double x, mu_before, mu_after;
    double nu_lab_before, nu_lab_after, e_lab_before, e_lab_after;
    double e_cmf_before, e_cmf_after, nu_cmf_before, nu_cmf_after;
} orc_event;

typedef struct {
    orc_event *events;
    int64_t capacity, count;
} orc_trace;

/* ------------------------------------------------------------ geometry
 * Distance (in units of c t_exp) from x along mu to the boundary of shell
 * [x_in, x_out] (Sect. 2.6).  The outer boundary is always reachable; the
 * inner one only for mu < 0 with impact parameter below x_in.  Roots are taken
 * in the cancellation-free form.  *which = +1 outer, -1 inner.
 */
double orc_distance_shell(double x, double mu, double x_in, double x_out, int32_t *which)
{
    double p = x * mu;
    double disc_out = (x_out - x) * (x_out + x) + p * p;
    double root_out = sqrt(disc_out);
    double d_out;
    if (mu >= 0.0) d_out = ((x_out - x) * (x_out + x)) / (root_out + p);
    else d_out = root_out - p;
    if (!(d_out > 0.0)) d_out = 0.0; /* also the 0/0 of a tangent ray on the boundary */
    if (mu < 0.0) {
        double disc_in = (x_in - x) * (x_in + x) + p * p;
        if (disc_in >= 0.0) {
            double d_in = ((x - x_in) * (x + x_in)) / (sqrt(disc_in) - p);
            if (!(d_in > 0.0)) d_in = 0.0;
            *which = -1;
            return d_in;
        }
    }
    *which = 1;
    return d_out;
}

/* First line index j with nu[j] < nu_cmf (strict), L if none. */
static int32_t first_redward_line(const double *nu, int32_t L, double nu_cmf)
{
    int32_t lo = 0, hi = L;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (nu[mid] < nu_cmf) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* Downbranch emission: first entry k of the row with z < cdf[k]. */
static int32_t downbranch_pick(const orc_model *m, int32_t row, double z)
{
    uint32_t b = m->dbr_offset[row], e = m->dbr_offset[row + 1];
    for (uint32_t k = b; k < e; ++k) {
        if (z < m->dbr_cdf[k]) return (int32_t)m->dbr_line[k];
    }
    return (int32_t)m->dbr_line[e - 1];
}

int32_t orc_downbranch_pick(const orc_model *m, int32_t row, double z) { return downbranch_pick(m, row, z); }

/* Macro atom (Sect. 2.5, mode macroatom): activated in a level (row), the
 * atom makes internal transitions -- from its current level it jumps with
 * that level's probability ma_jump_p, to the target the level's jump CDF
 * picks -- until it deactivates through the current level's branching row
 * (the downbranch choice).  Draws, in order: per step one to decide whether
 * to jump, one for the target if it jumps; then one for the emitting line.
 * After ORC_MA_MAX_STEPS jumps the atom deactivates without the decision. */
#define ORC_MA_MAX_STEPS 1024
static int32_t macroatom_emit(const orc_model *m, int32_t row, orc_rng *r, uint32_t *jumps)
{
    uint32_t n = 0;
    while (n < ORC_MA_MAX_STEPS) {
        double za = rng_closed0(r);
        if (!(za < m->ma_jump_p[row])) break;
        double zb = rng_closed0(r);
        uint32_t b = m->ma_jump_offset[row], e = m->ma_jump_offset[row + 1];
        int32_t next = m->ma_jump_target[e - 1];
        for (uint32_t k = b; k < e; ++k) {
            if (zb < m->ma_jump_cdf[k]) { next = m->ma_jump_target[k]; break; }
        }
        row = next;
        n += 1;
    }
    if (jumps) *jumps = n;
    return downbranch_pick(m, row, rng_closed0(r));
}

/* n walks from level row, walk i drawing from the r-packet stream of packet i
 * (seed, iteration 0): emitting line and number of jumps of each. */
void orc_macroatom_walks(const orc_model *m, int32_t row, uint64_t seed, int64_t n, int32_t *line, uint32_t *jumps)
{
    for (int64_t i = 0; i < n; ++i) {
        orc_rng r;
        rng_init(&r, seed, 0u, (uint32_t)i, 0u);
        line[i] = macroatom_emit(m, row, &r, jumps ? &jumps[i] : NULL);
    }
}

/* ------------------------------------------------------------ one packet */
typedef struct {
    double x, mu, nu_lab, e_lab;
    int32_t shell, next_line, status;
    uint64_t cnt[ORC_NCOUNT];
} orc_packet;

typedef struct {
    double *x_in, *x_out, *kappa; /* kappa = sigma_T n_e c t_exp (per unit x) */
} orc_geom;

static void geom_init(const orc_model *m, orc_geom *g)
{
    int S = m->n_shells;
    g->x_in = (double *)malloc(sizeof(double) * S);
    g->x_out = (double *)malloc(sizeof(double) * S);
    g->kappa = (double *)malloc(sizeof(double) * S);
    for (int s = 0; s < S; ++s) {
        g->x_in[s] = m->v_inner[s] / C_LIGHT;
        g->x_out[s] = m->v_outer[s] / C_LIGHT;
        g->kappa[s] = ((SIGMA_T * m->n_e[s]) * C_LIGHT) * m->t_exp;
    }
}

static void geom_free(orc_geom *g) { free(g->x_in); free(g->x_out); free(g->kappa); }

/* Packet energy of Eqs. 9-10: E = 4 pi r_i^2 sigma T_i^4 dt / N. */
static double packet_energy(const orc_model *m, double t_inner, uint64_t n_packets)
{
    double r_i = m->v_inner[0] * m->t_exp;
    double lum = (((4.0 * PI_D) * r_i) * r_i) * SIGMA_SB * t_inner * t_inner * t_inner * t_inner;
    return (lum * m->delta_t) / (double)n_packets;
}

/* Injection at the inner boundary (Sect. 2.4). */
static void inject(const orc_model *m, const orc_geom *g, orc_rng *r, double e_cmf, double t_inner,
                   orc_packet *pk, double *nu_cmf_out)
{
    double z0 = rng_closed0(r);
    double z1 = rng_open0(r), z2 = rng_open0(r), z3 = rng_open0(r), z4 = rng_open0(r);
    double xi = planck_xi(z0, z1, z2, z3, z4);
    double nu_cmf = ((K_BOLTZ * t_inner) / H_PLANCK) * xi;
    double mu = sqrt(rng_open0(r));
    double x = g->x_in[0];
    double D = 1.0 - mu * x;
    pk->x = x;
    pk->mu = mu;
    pk->nu_lab = nu_cmf / D;
    pk->e_lab = e_cmf / D;
    pk->shell = 0;
    pk->next_line = first_redward_line(m->nu, m->n_lines, nu_cmf);
    pk->status = ORC_IN_FLIGHT;
    memset(pk->cnt, 0, sizeof(pk->cnt));
    if (nu_cmf_out) *nu_cmf_out = nu_cmf;
}

static void spectrum_add(const orc_model *m, double *spec, double nu_lab, double e_lab);

/* ------------------------------------------------------------ virtual packets
 * Sect. 2.9.  In the spectrum iteration, whenever an r-packet is about to
 * start a new trajectory (injection, or after an interaction), N_v virtual
 * packets leave the same point with the same comoving frequency and energy
 * but their own directions mu_v, uniform in (mu_min, 1] with
 * mu_min = -sqrt(1 - (r_inner/r)^2), so that none meets the inner boundary.
 * A v-packet never interacts: it flies to the outer boundary collecting the
 * optical depth tau_v of the Sobolev points it passes and of electron
 * scattering (kappa_e = sigma_T n_e D with D at each segment start, as for
 * r-packets), and adds exp(-tau_v) times its lab-frame energy to the bin of
 * its lab frequency (Eq. 21).  Comoving energies: Eq. 19 after an
 * interaction, Eq. 20 at injection.  Its direction draws come from Philox
 * stream 1, so the r-packet's own draws are untouched.
 */

/* tau_v along the ray from x, mu in shell s (lines from index j on), or
 * ORC_INF when the ray meets the inner boundary (only by rounding) or tau_v
 * exceeds tau_v_max (> 0). */
static double virtual_tau(const orc_model *m, const orc_geom *g, double x, double mu, int32_t s,
                          double nu_lab, int32_t j)
{
    const int32_t S = m->n_shells, L = m->n_lines;
    const double inv = 1.0 / nu_lab;
    double tau = 0.0;
    for (;;) {
        const double D = 1.0 - mu * x;
        const double nu_cmf = nu_lab * D;
        const double kv = g->kappa[s] * D;
        int32_t which;
        const double d_shell = orc_distance_shell(x, mu, g->x_in[s], g->x_out[s], &which);
        /* Sobolev points before the shell boundary (strict, as for r-packets) */
        while (j < L) {
            double d_line = (nu_cmf - m->nu[j]) * inv;
            if (d_line < 0.0) d_line = 0.0;
            if (!(d_line < d_shell)) break;
            tau += m->tau[(size_t)s * (size_t)L + (size_t)j];
            j += 1;
            if (m->tau_v_max > 0.0 && tau > m->tau_v_max) return ORC_INF;
        }
        tau += kv * d_shell;
        if (m->tau_v_max > 0.0 && tau > m->tau_v_max) return ORC_INF;
        const double xb = (which > 0) ? g->x_out[s] : g->x_in[s];
        double mun = (x * mu + d_shell) / xb;
        if (mun > 1.0) mun = 1.0;
        if (mun < -1.0) mun = -1.0;
        x = xb;
        mu = mun;
        s += which;
        if (s >= S) return tau;
        if (s < 0) return ORC_INF;
    }
}

double orc_virtual_tau(const orc_model *m, double x, double mu, int32_t shell, double nu_lab, int32_t next_line)
{
    orc_geom g;
    geom_init(m, &g);
    double tau = virtual_tau(m, &g, x, mu, shell, nu_lab, next_line);
    geom_free(&g);
    return tau;
}

/* N_v v-packets from radius x in shell s with comoving frequency nu_cmf and
 * comoving energy e_cmf of the r-packet about to be launched. */
static void spawn_virtual(const orc_model *m, const orc_geom *g, orc_rng *rv, double x, int32_t s,
                          double nu_cmf, double e_cmf, int32_t next_line, int injection, orc_result *res)
{
    const int32_t nv = m->n_virtual;
    const double ri = g->x_in[0] / x;
    double arg = 1.0 - ri * ri;
    if (arg < 0.0) arg = 0.0;
    const double mu_min = -sqrt(arg);
    for (int32_t i = 0; i < nv; ++i) {
        const double mu_v = mu_min + (1.0 - mu_min) * rng_open0(rv);
        const double D = 1.0 - mu_v * x;
        const double e_v = injection ? (e_cmf * (2.0 * mu_v)) / (double)nv
                                     : (e_cmf * (1.0 - mu_min)) / (2.0 * (double)nv);
        const double nu_lab = nu_cmf / D;
        const double tau = virtual_tau(m, g, x, mu_v, s, nu_lab, next_line);
        if (tau == ORC_INF) continue;
        spectrum_add(m, res->spectrum_v, nu_lab, (e_v / D) * orc_exp(-tau));
    }
}

static void trace_push(orc_trace *t, const orc_event *e)
{
    if (t && t->count < t->capacity) t->events[t->count] = *e;
    if (t) t->count += 1;
}

/* Transport one packet until it escapes, is reabsorbed or is capped
 * (Sect. 2.6), accumulating the estimators of Sect. 2.7 into res. */
static void transport(const orc_model *m, const orc_geom *g, orc_rng *r, orc_rng *rv, orc_packet *pk,
                      orc_result *res, orc_trace *trace)
{
    const int32_t S = m->n_shells, L = m->n_lines;
    const double *nu_line = m->nu;
    for (;;) {
        if (pk->cnt[ORC_CNT_SEGMENTS] >= m->max_segments) { pk->status = ORC_CAPPED; return; }
        pk->cnt[ORC_CNT_SEGMENTS] += 1;
        const int32_t s = pk->shell;
        const double x = pk->x, mu = pk->mu;
        /* Segment start: Doppler factor, comoving frequency and energy, and
         * the observer-frame Thomson opacity kappa_e = sigma_T n_e D (Eq. 11). */
        const double D = 1.0 - mu * x;
        const double nu_cmf = pk->nu_lab * D;
        const double e_cmf = pk->e_lab * D;
        const double k = g->kappa[s] * D;
        /* Optical depth to the next event: tau = -ln z, z in (0,1]. */
        double tau_rem = -orc_log(rng_open0(r));
        int32_t which;
        const double d_shell = orc_distance_shell(x, mu, g->x_in[s], g->x_out[s], &which);
        double d_e = (k > 0.0) ? tau_rem / k : ORC_INF;
        const double inv = 1.0 / pk->nu_lab;
        int32_t j = pk->next_line;
        int kind;          /* 1 electron, 2 line, 3 shell */
        double l;
        /* Walk the redward lines while a Sobolev resonance is the closest event. */
        for (;;) {
            double d_line;
            if (j >= L) {
                d_line = ORC_INF;
            } else {
                pk->cnt[ORC_CNT_LINE_CHECKS] += 1;
                d_line = (nu_cmf - nu_line[j]) * inv;
                if (d_line < 0.0) d_line = 0.0;
            }
            if (d_line < d_e && d_line < d_shell) {
                pk->cnt[ORC_CNT_RESONANCES] += 1;
                if (m->j_blue && res->j_blue) {
                    double d_res = nu_line[j] * inv;
                    res->j_blue[(size_t)s * (size_t)L + (size_t)j] += ((pk->e_lab * d_res) * d_res) / nu_line[j];
                }
                double tau_line = m->tau[(size_t)s * (size_t)L + (size_t)j];
                if (tau_line + k * d_line > tau_rem) { kind = 2; l = d_line; break; }
                tau_rem = tau_rem - tau_line;
                d_e = (k > 0.0) ? tau_rem / k : ORC_INF;
                j = j + 1;
                continue;
            }
            if (d_e < d_shell) { kind = 1; l = d_e; }
            else { kind = 3; l = d_shell; }
            break;
        }
        pk->next_line = j;
        /* Estimators, Eqs. 13-14 (segment-start comoving E, nu and D). */
        res->j_est[s] += (e_cmf * l) * D;
        res->nu_bar[s] += ((e_cmf * nu_cmf) * l) * D;

        orc_event ev;
        if (trace) {
            memset(&ev, 0, sizeof(ev));
            ev.shell = s;
            ev.mu_before = mu;
            ev.nu_lab_before = pk->nu_lab;
            ev.e_lab_before = pk->e_lab;
        }
        /* Move along the ray; the impact parameter squared q is conserved. */
        const double p = x * mu;
        if (kind == 3) {
            pk->cnt[ORC_CNT_SHELL_CROSSINGS] += 1;
            double xb = (which > 0) ? g->x_out[s] : g->x_in[s];
            double mun = (p + l) / xb;
            if (mun > 1.0) mun = 1.0;
            if (mun < -1.0) mun = -1.0;
            pk->x = xb;
            pk->mu = mun;
            pk->shell = s + which;
            if (trace) { ev.kind = 3; ev.x = xb; ev.mu_after = mun; ev.nu_lab_after = pk->nu_lab; ev.e_lab_after = pk->e_lab; }
            if (pk->shell >= S) {
                pk->status = ORC_ESCAPED;
                if (trace) { ev.kind = 4; trace_push(trace, &ev); }
                return;
            }
            if (pk->shell < 0) {
                pk->status = ORC_REABSORBED;
                if (trace) { ev.kind = 5; trace_push(trace, &ev); }
                return;
            }
            if (trace) trace_push(trace, &ev);
            continue;
        }
        double q = x * x - p * p;
        if (q < 0.0) q = 0.0;
        const double pl = p + l;
        const double xn = sqrt(q + pl * pl);
        double mun = pl / xn;
        if (mun > 1.0) mun = 1.0;
        if (mun < -1.0) mun = -1.0;
        pk->x = xn;
        const double D1 = 1.0 - mun * xn;
        if (kind == 1) {
            /* Thomson scattering: coherent in the comoving frame, isotropic. */
            pk->cnt[ORC_CNT_E_SCATTERS] += 1;
            const double nu_c = pk->nu_lab * D1;
            const double e_c = pk->e_lab * D1;
            const double mu2 = -1.0 + 2.0 * rng_closed0(r);
            const double D2 = 1.0 - mu2 * xn;
            pk->mu = mu2;
            pk->nu_lab = nu_c / D2;
            pk->e_lab = e_c / D2;
            if (rv) spawn_virtual(m, g, rv, xn, s, nu_c, e_c, j, 0, res);
            if (trace) {
                ev.kind = 1; ev.x = xn; ev.mu_after = mu2;
                ev.nu_cmf_before = nu_c; ev.nu_cmf_after = pk->nu_lab * D2;
                ev.e_cmf_before = e_c; ev.e_cmf_after = pk->e_lab * D2;
                ev.nu_lab_after = pk->nu_lab; ev.e_lab_after = pk->e_lab;
                trace_push(trace, &ev);
            }
        } else {
            /* Bound-bound absorption at the Sobolev point of line j, then
             * re-emission: resonance scattering (scatter) or direct
             * deactivation of the activated upper level (downbranch). */
            pk->cnt[ORC_CNT_LINE_INTERACTIONS] += 1;
            const double e_c = pk->e_lab * D1;
            int32_t emit = j;
            if (m->line_mode == 1) emit = downbranch_pick(m, m->line_row[j], rng_closed0(r));
            else if (m->line_mode == 2) emit = macroatom_emit(m, m->line_row[j], r, NULL);
            const double mu2 = -1.0 + 2.0 * rng_closed0(r);
            const double D2 = 1.0 - mu2 * xn;
            if (trace) {
                ev.kind = 2; ev.x = xn; ev.line = j; ev.emit = emit; ev.mu_after = mu2;
                ev.nu_cmf_before = pk->nu_lab * D1; ev.e_cmf_before = e_c;
            }
            pk->mu = mu2;
            pk->nu_lab = nu_line[emit] / D2;
            pk->e_lab = e_c / D2;
            pk->next_line = emit + 1;
            if (rv) spawn_virtual(m, g, rv, xn, s, nu_line[emit], e_c, emit + 1, 0, res);
            if (trace) {
                ev.nu_cmf_after = pk->nu_lab * D2; ev.e_cmf_after = pk->e_lab * D2;
                ev.nu_lab_after = pk->nu_lab; ev.e_lab_after = pk->e_lab;
                trace_push(trace, &ev);
            }
        }
    }
}

/* Direct binning of an escaping packet (Sect. 2.9): lab energy into the bin
 * of its lab frequency, bins uniform in nu over [nu_lo, nu_hi); below and
 * above the range into the two extra tallies. */
static void spectrum_add(const orc_model *m, double *spec, double nu_lab, double e_lab)
{
    int B = m->spec_bins;
    if (nu_lab < m->spec_nu_lo) { spec[B] += e_lab; return; }
    double dnu = (m->spec_nu_hi - m->spec_nu_lo) / (double)B;
    double t = (nu_lab - m->spec_nu_lo) / dnu;
    if (!(t >= 0.0 && t < (double)B)) { spec[B + 1] += e_lab; return; } /* overflow or NaN */
    int b = (int)floor(t);
    spec[b] += e_lab;
}

/* Run packets [first, first+count) of an iteration of n_packets packets. */
static void run_range(const orc_model *m, const orc_geom *g, uint64_t seed, uint32_t iteration,
                      uint64_t n_packets, double t_inner, uint64_t first, uint64_t count,
                      orc_result *res, uint64_t rec_base, orc_trace *trace)
{
    double e_cmf = packet_energy(m, t_inner, n_packets);
    for (uint64_t i = 0; i < count; ++i) {
        uint64_t pid = first + i;
        orc_rng r;
        rng_init(&r, seed, iteration, (uint32_t)pid, 0u);
        orc_packet pk;
        double nu_cmf0;
        inject(m, g, &r, e_cmf, t_inner, &pk, &nu_cmf0);
        orc_rng rv;
        const int virt = m->n_virtual > 0 && res->spectrum_v;
        if (virt) {
            rng_init(&rv, seed, iteration, (uint32_t)pid, 1u);
            spawn_virtual(m, g, &rv, g->x_in[0], 0, nu_cmf0, e_cmf, pk.next_line, 1, res);
        }
        transport(m, g, &r, virt ? &rv : NULL, &pk, res, trace);
        if (pk.status == ORC_ESCAPED) {
            res->stats[ORC_ST_ESCAPED] += 1;
            spectrum_add(m, res->spectrum, pk.nu_lab, pk.e_lab);
        } else if (pk.status == ORC_REABSORBED) {
            res->stats[ORC_ST_REABSORBED] += 1;
        } else {
            res->stats[ORC_ST_CAPPED] += 1;
        }
        res->stats[ORC_ST_SEGMENTS] += pk.cnt[ORC_CNT_SEGMENTS];
        res->stats[ORC_ST_LINE_CHECKS] += pk.cnt[ORC_CNT_LINE_CHECKS];
        res->stats[ORC_ST_RESONANCES] += pk.cnt[ORC_CNT_RESONANCES];
        res->stats[ORC_ST_LINE_INTERACTIONS] += pk.cnt[ORC_CNT_LINE_INTERACTIONS];
        res->stats[ORC_ST_E_SCATTERS] += pk.cnt[ORC_CNT_E_SCATTERS];
        res->stats[ORC_ST_SHELL_CROSSINGS] += pk.cnt[ORC_CNT_SHELL_CROSSINGS];
        uint64_t k = rec_base + i;
        if (res->status) res->status[k] = pk.status;
        if (res->nu_out) res->nu_out[k] = pk.nu_lab;
        if (res->e_out) res->e_out[k] = pk.e_lab;
        if (res->counters) memcpy(&res->counters[k * ORC_NCOUNT], pk.cnt, sizeof(pk.cnt));
    }
}

typedef struct {
    const orc_model *m;
    const orc_geom *g;
    uint64_t seed, n_packets, first, count, rec_base;
    uint32_t iteration;
    double t_inner;
    orc_result res;
} orc_job;

static void *job_main(void *arg)
{
    orc_job *jb = (orc_job *)arg;
    run_range(jb->m, jb->g, jb->seed, jb->iteration, jb->n_packets, jb->t_inner, jb->first,
              jb->count, &jb->res, jb->rec_base, NULL);
    return NULL;
}

static int valid_model(const orc_model *m)
{
    if (m->n_shells <= 0 || m->n_lines < 0 || m->spec_bins <= 0) return 0;
    if (!m->v_inner || !m->v_outer || !m->n_e || !m->tau || (m->n_lines > 0 && !m->nu)) return 0;
    if (m->line_mode < 0 || m->line_mode > 2) return 0;
    if (m->line_mode >= 1 && (!m->line_row || !m->dbr_offset || !m->dbr_line || !m->dbr_cdf)) return 0;
    if (m->line_mode == 2 && (!m->ma_jump_p || !m->ma_jump_offset || !m->ma_jump_target || !m->ma_jump_cdf))
        return 0;
    return 1;
}

/* Transport packets [first, first+count) of an iteration with n_packets
 * packets.  Estimators are ADDED to res (callers zero them).  With
 * n_threads > 1 the packet range is split into contiguous parts, each with its
 * own estimator copies, summed in part order at the end.  Returns 0 on success. */
int orc_run(const orc_model *m, uint64_t seed, uint32_t iteration, uint64_t n_packets, double t_inner,
            uint64_t first, uint64_t count, int32_t n_threads, orc_result *res)
{
    if (!valid_model(m) || n_packets == 0) return -1;
    planck_table_init();
    orc_geom g;
    geom_init(m, &g);
    if (n_threads <= 1 || count < (uint64_t)n_threads * 4) {
        run_range(m, &g, seed, iteration, n_packets, t_inner, first, count, res, 0, NULL);
        geom_free(&g);
        return 0;
    }
    const int S = m->n_shells, B = m->spec_bins;
    const size_t nJb = (m->j_blue && res->j_blue) ? (size_t)S * (size_t)m->n_lines : 0;
    orc_job *jobs = (orc_job *)calloc((size_t)n_threads, sizeof(orc_job));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    uint64_t per = count / (uint64_t)n_threads, rem = count % (uint64_t)n_threads, off = 0;
    for (int t = 0; t < n_threads; ++t) {
        orc_job *jb = &jobs[t];
        uint64_t c = per + ((uint64_t)t < rem ? 1 : 0);
        jb->m = m; jb->g = &g; jb->seed = seed; jb->iteration = iteration;
        jb->n_packets = n_packets; jb->t_inner = t_inner; jb->first = first + off; jb->count = c;
        jb->rec_base = 0;
        jb->res.j_est = (double *)calloc((size_t)S, sizeof(double));
        jb->res.nu_bar = (double *)calloc((size_t)S, sizeof(double));
        jb->res.spectrum = (double *)calloc((size_t)B + 2, sizeof(double));
        jb->res.j_blue = nJb ? (double *)calloc(nJb, sizeof(double)) : NULL;
        jb->res.spectrum_v = res->spectrum_v ? (double *)calloc((size_t)B + 2, sizeof(double)) : NULL;
        jb->res.status = res->status ? res->status + off : NULL;
        jb->res.nu_out = res->nu_out ? res->nu_out + off : NULL;
        jb->res.e_out = res->e_out ? res->e_out + off : NULL;
        jb->res.counters = res->counters ? res->counters + off * ORC_NCOUNT : NULL;
        off += c;
        pthread_create(&th[t], NULL, job_main, jb);
    }
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < n_threads; ++t) {
        orc_job *jb = &jobs[t];
        for (int s = 0; s < S; ++s) { res->j_est[s] += jb->res.j_est[s]; res->nu_bar[s] += jb->res.nu_bar[s]; }
        for (int b = 0; b < B + 2; ++b) res->spectrum[b] += jb->res.spectrum[b];
        if (res->spectrum_v)
            for (int b = 0; b < B + 2; ++b) res->spectrum_v[b] += jb->res.spectrum_v[b];
        for (size_t i = 0; i < nJb; ++i) res->j_blue[i] += jb->res.j_blue[i];
        for (int k = 0; k < ORC_NSTATS; ++k) res->stats[k] += jb->res.stats[k];
        free(jb->res.j_est); free(jb->res.nu_bar); free(jb->res.spectrum); free(jb->res.j_blue);
        free(jb->res.spectrum_v);
    }
    free(jobs); free(th);
    geom_free(&g);
    return 0;
}

/* Single-threaded run with an event trace (invariant tests). */
int orc_run_traced(const orc_model *m, uint64_t seed, uint32_t iteration, uint64_t n_packets,
                   double t_inner, uint64_t first, uint64_t count, orc_result *res, orc_trace *trace)
{
    if (!valid_model(m) || n_packets == 0) return -1;
    planck_table_init();
    orc_geom g;
    geom_init(m, &g);
    run_range(m, &g, seed, iteration, n_packets, t_inner, first, count, res, 0, trace);
    geom_free(&g);
    return 0;
}

/* Injection state of packets [first, first+count): comoving frequency,
 * direction, lab frequency and energy, first redward line. */
int orc_inject_packets(const orc_model *m, uint64_t seed, uint32_t iteration, uint64_t n_packets,
                       double t_inner, uint64_t first, uint64_t count, double *nu_cmf, double *mu,
                       double *nu_lab, double *e_lab, int32_t *next_line)
{
    if (!valid_model(m) || n_packets == 0) return -1;
    planck_table_init();
    orc_geom g;
    geom_init(m, &g);
    double e_cmf = packet_energy(m, t_inner, n_packets);
    for (uint64_t i = 0; i < count; ++i) {
        orc_rng r;
        rng_init(&r, seed, iteration, (uint32_t)(first + i), 0u);
        orc_packet pk;
        double nc;
        inject(m, &g, &r, e_cmf, t_inner, &pk, &nc);
        nu_cmf[i] = nc; mu[i] = pk.mu; nu_lab[i] = pk.nu_lab; e_lab[i] = pk.e_lab; next_line[i] = pk.next_line;
    }
    geom_free(&g);
    return 0;
}

/* Raw uniform draws of one packet's stream (z in [0,1) form), for the tests. */
void orc_uniforms(uint64_t seed, uint32_t iteration, uint32_t packet, uint32_t stream, int64_t n, double *out)
{
    orc_rng r;
    rng_init(&r, seed, iteration, packet, stream);
    for (int64_t i = 0; i < n; ++i) out[i] = rng_closed0(&r);
}

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) { philox4x32_10(ctr, key, out); }

/* xi samples of the Planck sampler for given uniforms (5 per sample). */
void orc_planck_xi(int64_t n, const double *z, double *xi)
{
    planck_table_init();
    for (int64_t i = 0; i < n; ++i) xi[i] = planck_xi(z[5 * i], z[5 * i + 1], z[5 * i + 2], z[5 * i + 3], z[5 * i + 4]);
}

/* ------------------------------------------------------------ plasma
 * Level populations, Sect. 2.3: Boltzmann excitation (Eq. 4) for the ground
 * and metastable levels and the dilute-lte form (Eq. 5, weight W) for the
 * other levels.  The partition function is Z = sum_k w_k g_k exp(-eps_k/kT_R),
 * so that the populations of an ion sum to its density.  lte_excitation != 0
 * sets w_k = 1 for every level (Eq. 4).  n has layout [S][I][K].
 */
void orc_level_populations(int32_t S, int32_t I, int32_t K, const double *t_rad, const double *w,
                           const double *energy_ev, const double *g, const uint8_t *metastable,
                           const double *n_ion, int32_t lte_excitation, double *n)
{
    double *wgb = (double *)malloc(sizeof(double) * (size_t)K);
    for (int32_t s = 0; s < S; ++s) {
        const double kT = K_BOLTZ * t_rad[s];
        for (int32_t i = 0; i < I; ++i) {
            double Z = 0.0;
            for (int32_t k = 0; k < K; ++k) {
                size_t a = (size_t)i * K + k;
                double wk = (lte_excitation || metastable[a]) ? 1.0 : w[s];
                double eps = energy_ev[a] * EV_ERG;
                double b = orc_exp(-(eps / kT));
                wgb[k] = (wk * g[a]) * b;
                Z = Z + wgb[k];
            }
            double N = n_ion[(size_t)s * I + i];
            for (int32_t k = 0; k < K; ++k) n[((size_t)s * I + i) * K + k] = (wgb[k] * N) / Z;
        }
    }
    free(wgb);
}

/* Sobolev optical depth, Eq. 12:
 *   tau = (pi e^2 / m_e c) f lambda t_exp n_l (1 - g_l n_u / (g_u n_l)),
 * lambda = c / nu.  tau has layout [S][L].  A line with n_l = 0 gets tau = 0. */
void orc_sobolev_tau(int32_t S, int32_t L, int32_t I, int32_t K, const double *nu, const double *f,
                     const int32_t *ion, const int32_t *lower, const int32_t *upper, const double *g,
                     const double *n, double t_exp, double *tau)
{
    const double sob = ((PI_D * E_CHARGE) * E_CHARGE) / (M_ELECTRON * C_LIGHT);
    for (int32_t s = 0; s < S; ++s) {
        for (int32_t j = 0; j < L; ++j) {
            size_t lev_l = (size_t)ion[j] * K + lower[j];
            size_t lev_u = (size_t)ion[j] * K + upper[j];
            double n_l = n[(size_t)s * I * K + lev_l];
            double n_u = n[(size_t)s * I * K + lev_u];
            double t = 0.0;
            if (n_l > 0.0) {
                double lambda = C_LIGHT / nu[j];
                double stim = 1.0 - (g[lev_l] * n_u) / (g[lev_u] * n_l);
                t = ((((sob * f[j]) * lambda) * t_exp) * n_l) * stim;
            }
            tau[(size_t)s * L + j] = t;
        }
    }
}

double orc_sobolev_constant(void) { return ((PI_D * E_CHARGE) * E_CHARGE) / (M_ELECTRON * C_LIGHT); }

/* ------------------------------------------------------------ radiation field
 * Geometric dilution at the shell centre (Sect. 2.8):
 * W = (1 - sqrt(1 - (r_inner/r)^2)) / 2, r the mid-radius of the shell. */
void orc_geometric_dilution(int32_t S, const double *v_inner, const double *v_outer, double *w)
{
    double x_i = v_inner[0] / C_LIGHT;
    for (int32_t s = 0; s < S; ++s) {
        double x_mid = (v_inner[s] / C_LIGHT + v_outer[s] / C_LIGHT) * 0.5;
        double rr = x_i / x_mid;
        w[s] = 0.5 * (1.0 - sqrt(1.0 - rr * rr));
    }
}

/* Factor turning a raw J sum (E l D with l in units of c t_exp) into the
 * estimator of Eq. 13: c t_exp / (4 pi dt V), V the shell volume. */
void orc_estimator_norm(int32_t S, const double *v_inner, const double *v_outer, double t_exp,
                        double delta_t, double *norm)
{
    for (int32_t s = 0; s < S; ++s) {
        double ri = v_inner[s] * t_exp, ro = v_outer[s] * t_exp;
        double V = ((4.0 / 3.0) * PI_D) * (((ro * ro) * ro) - ((ri * ri) * ri));
        norm[s] = (C_LIGHT * t_exp) / (((4.0 * PI_D) * delta_t) * V);
    }
}

/* Radiation-field update from the estimators, Eqs. 15-16:
 *   T_R = (h/k) (pi^4 / (360 zeta(5))) nu_bar / J,  W = pi J / (sigma T_R^4).
 * Shells whose J sum is zero keep their previous T_R and W. */
void orc_update_radiation_field(int32_t S, const double *j_raw, const double *nu_bar_raw,
                                const double *norm, double *t_rad, double *w)
{
    const double c_tr = (H_PLANCK / K_BOLTZ) * ((PI_D * PI_D * PI_D * PI_D) / (360.0 * ZETA5));
    for (int32_t s = 0; s < S; ++s) {
        if (!(j_raw[s] > 0.0)) continue;
        double T = c_tr * (nu_bar_raw[s] / j_raw[s]);
        double J = j_raw[s] * norm[s];
        t_rad[s] = T;
        w[s] = (PI_D * J) / (SIGMA_SB * (((T * T) * T) * T));
    }
}

int32_t orc_abi_version(void) { return 1; }

/* ------------------------------------------------------------ inner boundary
 * Sect. 2.8.  Eq. 18: first guess of T_inner from the requested luminosity
 * at the outer boundary, L_o = 4 pi r_i^2 sigma T_i^4.  The emitted
 * luminosity is the lab-frame energy of the escaping packets per unit time
 * (every bin of the spectrum, including the two outside the range).  After an
 * iteration T_inner moves so that the emitted luminosity would match the
 * requested one if it scaled like T_inner^4: T <- T (L_o / L_emitted)^(1/4);
 * with no escaping energy T_inner is kept.
 */
double orc_t_inner_from_luminosity(double r_inner, double l_outer)
{
    double x = l_outer / ((((4.0 * PI_D) * r_inner) * r_inner) * SIGMA_SB);
    return sqrt(sqrt(x));
}

double orc_emitted_luminosity(const double *spectrum, int32_t n_bins_total, double delta_t)
{
    double s = 0.0;
    for (int32_t b = 0; b < n_bins_total; ++b) s += spectrum[b];
    return s / delta_t;
}

double orc_t_inner_update(double t_inner, double l_requested, double l_emitted)
{
    if (!(l_emitted > 0.0)) return t_inner;
    return t_inner * sqrt(sqrt(l_requested / l_emitted));
}

/* ------------------------------------------------------------ ionization
 * Sect. 2.3.  Per shell, the ratio of successive ionization stages of an
 * element, Phi'_{e,j} = N_{e,j+1} n_e / N_{e,j}, is the Saha-Boltzmann value
 * (lte mode, Eq. 2)
 *   Phi = 2 Z_{j+1}/Z_j (2 pi m_e k T_R / h^2)^(3/2) exp(-chi_j / k T_R)
 * or the modified nebular value (nebular mode, Eq. 3)
 *   Phi' = W [delta zeta_j + W (1 - zeta_j)] (T_e / T_R)^(1/2) Phi,  T_e = 0.9 T_R.
 * Z_j is the LTE partition function sum_k g_k exp(-eps_k / k T_R) of a stage
 * with levels, 1 for a stage without (ion_of[e*J + j] < 0).  For a trial n_e
 * the stage fractions follow from the ratios; n_e itself is the root of
 * charge conservation n_e = sum_e N_e sum_j j f_{e,j}(n_e) (the right side
 * falls as n_e grows, so the root is unique), found by bisection on ln n_e
 * with the geometric midpoint sqrt(lo hi).
 * Outputs: n_ion[S*I] for the stages with levels, n_e[S].
 */
#define ORC_ION_MAX_STAGES 16
static void stage_fractions(int32_t J, const double *phi, double n_e, double *f)
{
    double r = 1.0, sum = 1.0;
    f[0] = 1.0;
    for (int32_t j = 1; j < J; ++j) {
        r = r * (phi[j - 1] / n_e);
        f[j] = r;
        sum += r;
    }
    for (int32_t j = 0; j < J; ++j) f[j] = f[j] / sum;
}

int orc_ionization(int32_t S, int32_t I, int32_t K, int32_t E, int32_t J, const int32_t *ion_of,
                   const double *energy_ev, const double *g, const double *chi_ev, const double *zeta,
                   double delta, const double *n_element, const double *t_rad, const double *w,
                   int32_t mode, double *n_ion, double *n_e)
{
    if (J < 2 || J > ORC_ION_MAX_STAGES || (mode != 1 && mode != 2)) return -1;
    double *phi = (double *)malloc(sizeof(double) * (size_t)E * (size_t)(J - 1));
    double Z[ORC_ION_MAX_STAGES], f[ORC_ION_MAX_STAGES];
    for (int32_t s = 0; s < S; ++s) {
        const double T = t_rad[s], W = w[s];
        const double kT = K_BOLTZ * T;
        const double x = ((2.0 * PI_D) * M_ELECTRON * kT) / (H_PLANCK * H_PLANCK);
        const double saha = x * sqrt(x);
        const double neb = (mode == 2) ? sqrt(0.9) : 1.0;  /* (T_e / T_R)^(1/2) */
        double max_charge = 0.0;
        for (int32_t e = 0; e < E; ++e) {
            for (int32_t j = 0; j < J; ++j) {
                int32_t a = ion_of[e * J + j];
                double z = 1.0;
                if (a >= 0) {
                    z = 0.0;
                    for (int32_t k = 0; k < K; ++k) {
                        size_t lv = (size_t)a * K + k;
                        z = z + g[lv] * orc_exp(-((energy_ev[lv] * EV_ERG) / kT));
                    }
                }
                Z[j] = z;
            }
            for (int32_t j = 0; j + 1 < J; ++j) {
                size_t t = (size_t)e * (J - 1) + j;
                double p = ((2.0 * Z[j + 1]) / Z[j]) * saha * orc_exp(-((chi_ev[t] * EV_ERG) / kT));
                if (mode == 2) p = ((W * (delta * zeta[t] + W * (1.0 - zeta[t]))) * neb) * p;
                phi[t] = p;
            }
            max_charge += n_element[(size_t)s * E + e] * (double)(J - 1);
        }
        /* bisection on ln n_e: charge(lo) > lo, charge(hi) <= hi */
        double lo = max_charge * 1e-40, hi = max_charge;
        for (int it = 0; it < 200 && max_charge > 0.0; ++it) {
            double mid = sqrt(lo * hi);
            if (!(mid > lo && mid < hi)) break;
            double charge = 0.0;
            for (int32_t e = 0; e < E; ++e) {
                stage_fractions(J, &phi[(size_t)e * (J - 1)], mid, f);
                double ce = 0.0;
                for (int32_t j = 1; j < J; ++j) ce += (double)j * f[j];
                charge += n_element[(size_t)s * E + e] * ce;
            }
            if (charge > mid) lo = mid; else hi = mid;
        }
        const double ne = (max_charge > 0.0) ? sqrt(lo * hi) : 0.0;
        n_e[s] = ne;
        for (int32_t e = 0; e < E; ++e) {
            if (ne > 0.0) stage_fractions(J, &phi[(size_t)e * (J - 1)], ne, f);
            else { f[0] = 1.0; for (int32_t j = 1; j < J; ++j) f[j] = 0.0; }
            for (int32_t j = 0; j < J; ++j) {
                int32_t a = ion_of[e * J + j];
                if (a >= 0) n_ion[(size_t)s * I + a] = n_element[(size_t)s * E + e] * f[j];
            }
        }
    }
    free(phi);
    return 0;
}
