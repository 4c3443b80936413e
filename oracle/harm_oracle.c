/*
 * harm_oracle.c -- plain FP64 CPU oracle of the facet-to-IQ echo.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's CPU
 * baseline leg may load this code. It shares nothing with the CUDA path: no
 * headers, tables, helpers or generators. It evaluates every quantity directly
 * from its definition, in double precision, with no blocking, tiling, fusion,
 * offset decomposition or recurrence.
 *
 * What it computes (paper sections / equations cited per function):
 *   - Philox4x32-10 counter RNG (Salmon, Moraes, Dror & Shaw, SC'11) and the
 *     Box-Muller draw of the intra-facet speckle R + iI with R, I ~ N(0, 1/2)
 *     (Sec. III-A, Eq. 7 and the sentence after Eq. 8).
 *   - The resolved sea surface as a linear superposition of waves (the "linear
 *     surface" option of Sec. III, CWM off), JONSWAP frequency spectrum with
 *     cos^2s spreading on a 16 x 16 (omega, theta) grid.
 *   - Per-pulse platform state with light-time (Eq. 3 transmit/receive times).
 *   - The field contribution of a facet (Eq. 3, Eq. 4, Eq. 16): area, NRCS,
 *     speckle, Tx and Rx antenna gains, 1/(r_t r_r) spreading and the two-way
 *     phase exp(-i K0 (r_t + r_r + v_c t)).
 *   - The range-slice sum (Eq. 17) in its box form (taps = 1) and its
 *     Kaiser-windowed sinc form (taps = 2m), accumulated per bin with a
 *     Neumaier compensated sum (Neumaier 1974).
 *
 * Parity unpinned against the paper: the JONSWAP/spreading wave table and the
 * closed-form NRCS are not given by the paper; they are pinned only against
 * textbook closed forms and invariants in the tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_C 299792458.0
#define OR_G 9.80665
#define OR_PI 3.14159265358979323846
#define OR_MAXC 16

typedef struct {
    double pos0[3];
    double vel[3];
    double len_az, len_el;
} or_antenna;

typedef struct {
    double f0, fs, prf;
    int n_pulses, n_range;
    or_antenna tx;
    int n_channels;
    or_antenna rx[OR_MAXC];
    int nx, ny;
    double facet;
    int n_omega, n_theta;
    double u10, fetch, wind_dir, spread_s, gamma;
    uint64_t wave_seed;
    double cur_u, cur_v;
    double sigma0_base, wind_mod;
    int epoch_pulses;
    uint64_t speckle_seed;
    int static_surface;
    int taps;
    double beta;
    /* optional per-cell NRCS base and current (cells of cell_m, origin at the
       patch corner); NULL pointers mean uniform values above */
    int ncx, ncy;
    double cell;
    const double *cell_sigma0; /* [ncy][ncx] */
    const double *cell_uv;     /* [ncy][ncx][2] */
} or_scene;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: 10 rounds of the Philox S-box with a Weyl key schedule.     */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
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

/* Counter layout: (id, 0, word2, 0); key = (seed low word, seed high word XOR
   stream), where stream separates independent uses of one seed (0 for the
   speckle, 0x57415645 for the wave phases). */
#define OR_STREAM_SPECKLE 0x00000000u
#define OR_STREAM_WAVE 0x57415645u

static void philox_draw(uint64_t seed, uint32_t id, uint32_t word2, uint32_t stream, uint32_t out[4])
{
    uint32_t ctr[4] = {id, 0u, word2, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) ^ stream};
    or_philox4x32_10(ctr, key, out);
}

/* Intra-facet speckle R + iI of facet f in coherence epoch e (Eq. 7 at f_s = 0,
   R, I ~ N(0, 1/2) so that <s s*> = 1): Box-Muller on two Philox words. */
void or_speckle(uint64_t seed, uint64_t f, uint32_t epoch, double *re, double *im)
{
    uint32_t w[4];
    philox_draw(seed, (uint32_t)f, epoch, OR_STREAM_SPECKLE, w);
    double u1 = ((double)w[0] + 1.0) * (1.0 / 4294967296.0); /* (0, 1] */
    double u2 = (double)w[1] * (1.0 / 4294967296.0);         /* [0, 1) */
    double rad = sqrt(-log(u1));
    *re = rad * cos(2.0 * OR_PI * u2);
    *im = rad * sin(2.0 * OR_PI * u2);
}

/* ------------------------------------------------------------------------ */
/* Sea state: JONSWAP spectrum, cos^2s spreading, 2-D linear wave grid.      */
/* ------------------------------------------------------------------------ */
void or_jonswap_params(double u10, double fetch, double *omega_p, double *alpha)
{
    double xt = OR_G * fetch / (u10 * u10); /* dimensionless fetch */
    *omega_p = 22.0 * (OR_G / u10) * pow(xt, -1.0 / 3.0);
    *alpha = 0.076 * pow(xt, -0.22);
}

/* JONSWAP frequency spectrum S(omega) [m^2 s] (Hasselmann et al. 1973). */
double or_jonswap(double omega, double u10, double fetch, double gamma)
{
    double wp, alpha;
    or_jonswap_params(u10, fetch, &wp, &alpha);
    double sigma = (omega <= wp) ? 0.07 : 0.09;
    double r = exp(-(omega - wp) * (omega - wp) / (2.0 * sigma * sigma * wp * wp));
    double pm = alpha * OR_G * OR_G * pow(omega, -5.0) * exp(-1.25 * pow(wp / omega, 4.0));
    return pm * pow(gamma, r);
}

/* cos^{2s} directional spreading D(dtheta), normalised to unit integral over
   one turn. */
double or_spreading(double dtheta, double s)
{
    double ns = pow(2.0, 2.0 * s - 1.0) * tgamma(s + 1.0) * tgamma(s + 1.0) /
                (OR_PI * tgamma(2.0 * s + 1.0));
    return ns * pow(cos(0.5 * dtheta), 2.0 * s);
}

/* Wave component table: n_omega log-spaced frequency bins on [0.7, 2.5] omega_p
   (geometric bin centres), n_theta directions centred on the wind, deep-water
   dispersion k = omega^2 / g, amplitude a = sqrt(2 S dω D dθ) and a uniform
   random phase drawn by Philox (wave stream) per component. */
int or_wave_table(const or_scene *s, double *kx, double *ky, double *om, double *amp, double *ph)
{
    int no = s->n_omega, nt = s->n_theta;
    if (no <= 0 || nt <= 0) return 0;
    double wp, alpha;
    or_jonswap_params(s->u10, s->fetch, &wp, &alpha);
    double lo = 0.7 * wp, hi = 2.5 * wp;
    double dth = 2.0 * OR_PI / nt;
    for (int i = 0; i < no; ++i) {
        double e0 = lo * pow(hi / lo, (double)i / no);
        double e1 = lo * pow(hi / lo, (double)(i + 1) / no);
        double w = sqrt(e0 * e1);
        double dw = e1 - e0;
        double sw = or_jonswap(w, s->u10, s->fetch, s->gamma);
        double k = w * w / OR_G;
        for (int j = 0; j < nt; ++j) {
            int m = i * nt + j;
            double th = s->wind_dir - OR_PI + (j + 0.5) * dth;
            double d = or_spreading(th - s->wind_dir, s->spread_s);
            kx[m] = k * cos(th);
            ky[m] = k * sin(th);
            om[m] = w;
            amp[m] = sqrt(2.0 * sw * dw * d * dth);
            uint32_t r[4];
            philox_draw(s->wave_seed, (uint32_t)m, 0u, OR_STREAM_WAVE, r);
            ph[m] = 2.0 * OR_PI * ((double)r[0] * (1.0 / 4294967296.0));
        }
    }
    return no * nt;
}

/* Surface height and slopes at rest position (x, y), time t, by direct summation
   of the wave components. */
void or_surface(int nw, const double *kx, const double *ky, const double *om, const double *amp,
                const double *ph, double x, double y, double t, double out[3])
{
    double eta = 0.0, ex = 0.0, ey = 0.0;
    for (int m = 0; m < nw; ++m) {
        double arg = kx[m] * x + ky[m] * y - om[m] * t + ph[m];
        double c = cos(arg), sn = sin(arg);
        eta += amp[m] * c;
        ex -= amp[m] * kx[m] * sn;
        ey -= amp[m] * ky[m] * sn;
    }
    out[0] = eta;
    out[1] = ex;
    out[2] = ey;
}

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */
static double norm3(const double v[3]) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

static void antenna_pos(const or_antenna *a, double t, double p[3])
{
    for (int i = 0; i < 3; ++i) p[i] = a->pos0[i] + a->vel[i] * t;
}

typedef struct {
    double t;         /* pulse transmit time t_n */
    double ts;        /* scene (bounce) time at the scene centre */
    double trx;       /* receive time */
    double ptx[3], prx[3];
    double rt_ref, rr_ref; /* ranges to the scene centre */
    double atx[3], etx[3]; /* Tx antenna azimuth / elevation axes */
    double arx[3], erx[3]; /* Rx antenna axes */
} or_pulse;

/* Antenna frame steered to the scene centre: boresight b from the phase centre
   to the origin, azimuth axis a = velocity projected normal to b, elevation axis
   e = b x a. */
static void antenna_frame(const double p[3], const double v[3], double a[3], double e[3])
{
    double r = norm3(p);
    double b[3] = {-p[0] / r, -p[1] / r, -p[2] / r};
    double vb = v[0] * b[0] + v[1] * b[1] + v[2] * b[2];
    double t[3] = {v[0] - vb * b[0], v[1] - vb * b[1], v[2] - vb * b[2]};
    double tn = norm3(t);
    for (int i = 0; i < 3; ++i) a[i] = t[i] / tn;
    e[0] = b[1] * a[2] - b[2] * a[1];
    e[1] = b[2] * a[0] - b[0] * a[2];
    e[2] = b[0] * a[1] - b[1] * a[0];
}

/* Pulse n, channel c: transmit at t_n; the scene is sampled at the bounce time
   t_s = t_n + R_t / c at the scene centre; the receive time solves
   t_r = t_s + |P_rx(t_r) - 0| / c by three fixed-point steps from t_r = t_s
   (Eq. 3's transmit and receive times, evaluated at the scene centre). */
void or_pulse_state(const or_scene *s, int n, int c, or_pulse *g)
{
    g->t = (double)n / s->prf;
    antenna_pos(&s->tx, g->t, g->ptx);
    g->rt_ref = norm3(g->ptx);
    g->ts = g->t + g->rt_ref / OR_C;
    double trx = g->ts;
    double p[3];
    for (int it = 0; it < 3; ++it) {
        antenna_pos(&s->rx[c], trx, p);
        trx = g->ts + norm3(p) / OR_C;
    }
    g->trx = trx;
    antenna_pos(&s->rx[c], trx, g->prx);
    g->rr_ref = norm3(g->prx);
    antenna_frame(g->ptx, s->tx.vel, g->atx, g->etx);
    antenna_frame(g->prx, s->rx[c].vel, g->arx, g->erx);
}

/* Exposed for the tests: flat array of the pulse state. */
void or_pulse_state_flat(const or_scene *s, int n, int c, double *o)
{
    or_pulse g;
    or_pulse_state(s, n, c, &g);
    o[0] = g.t; o[1] = g.ts; o[2] = g.trx;
    for (int i = 0; i < 3; ++i) {
        o[3 + i] = g.ptx[i]; o[6 + i] = g.prx[i];
        o[11 + i] = g.atx[i]; o[14 + i] = g.etx[i];
        o[17 + i] = g.arx[i]; o[20 + i] = g.erx[i];
    }
    o[9] = g.rt_ref; o[10] = g.rr_ref;
}

static double sinc(double x)
{
    if (x == 0.0) return 1.0;
    double px = OR_PI * x;
    return sin(px) / px;
}

/* Antenna gain, applied as a field weight (Eq. 16): sinc^2 in azimuth times
   sinc^2 in elevation, with direction cosines u = d.a, v = d.e of the unit
   vector d from the phase centre to the facet. */
double or_pattern(double len_az, double len_el, double lambda, const double d[3],
                  const double a[3], const double e[3])
{
    double u = d[0] * a[0] + d[1] * a[1] + d[2] * a[2];
    double v = d[0] * e[0] + d[1] * e[1] + d[2] * e[2];
    double sa = sinc(len_az * u / lambda);
    double se = sinc(len_el * v / lambda);
    return sa * sa * se * se;
}

/* Modified Bessel function I0 by its power series sum_k ((x/2)^k / k!)^2. */
double or_bessel_i0(double x)
{
    double sum = 1.0, term = 1.0, q = 0.25 * x * x;
    for (int k = 1; k < 500; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

/* Kaiser-windowed sinc interpolation weight with half-width m:
   h(x) = sinc(x) I0(beta sqrt(1 - (x/m)^2)) / I0(beta) for |x| < m, else 0. */
double or_kaiser_sinc(double x, int m, double beta)
{
    if (fabs(x) >= (double)m) return 0.0;
    double q = x / (double)m;
    return sinc(x) * or_bessel_i0(beta * sqrt(1.0 - q * q)) / or_bessel_i0(beta);
}

/* Closed-form bistatic NRCS of a facet: Q = k_s - k_i with k_i = r_t (Tx to
   facet) and k_s = -r_r (facet to Rx); the wind term uses the angle between the
   wind direction and the horizontal part of Q (the bistatic angle of Eq. 12);
   the tilt factor is max(0, n.Q) / (|n| Q_z) for the facet normal n. */
double or_sigma0(const or_scene *s, double base, const double rt_hat[3], const double rr_hat[3],
                 double slope_x, double slope_y)
{
    if (s->static_surface) return base;
    double q[3] = {-(rt_hat[0] + rr_hat[0]), -(rt_hat[1] + rr_hat[1]), -(rt_hat[2] + rr_hat[2])};
    double qh = sqrt(q[0] * q[0] + q[1] * q[1]);
    double cphi = 0.0;
    if (qh > 0.0) cphi = (cos(s->wind_dir) * q[0] + sin(s->wind_dir) * q[1]) / qh;
    double nvec[3] = {-slope_x, -slope_y, 1.0};
    double ndotq = nvec[0] * q[0] + nvec[1] * q[1] + nvec[2] * q[2];
    double tilt = (ndotq > 0.0 ? ndotq : 0.0) / (norm3(nvec) * q[2]);
    return base * (1.0 + s->wind_mod * cphi) * tilt;
}

static int cell_index(const or_scene *s, double x, double y)
{
    double lx = s->nx * s->facet, ly = s->ny * s->facet;
    int cx = (int)floor((x + 0.5 * lx) / s->cell);
    int cy = (int)floor((y + 0.5 * ly) / s->cell);
    if (cx < 0) cx = 0;
    if (cx >= s->ncx) cx = s->ncx - 1;
    if (cy < 0) cy = 0;
    if (cy >= s->ncy) cy = s->ncy - 1;
    return cy * s->ncx + cx;
}

/* Range-window start per channel: the reference bistatic range at the middle
   pulse minus half the window. */
double or_range_start(const or_scene *s, int c)
{
    or_pulse g;
    or_pulse_state(s, s->n_pulses / 2, c, &g);
    return g.rt_ref + g.rr_ref - 0.5 * s->n_range * (OR_C / s->fs);
}

/* One facet's complex contribution at pulse state g (Eq. 3, 4, 16) and its
   fractional range-bin position p. state = (eta, eta_x, eta_y). */
static void contribution_full(const or_scene *s, const or_pulse *g, int n, int c, int64_t f,
                              const double state[3], double r0, double *sre, double *sim, double *p,
                              double *sumx, double *sumy, int *cell)
{
    double lambda = OR_C / s->f0;
    double k0 = 2.0 * OR_PI / lambda;
    int ix = (int)(f % s->nx), iy = (int)(f / s->nx);
    double x = (ix + 0.5 - 0.5 * s->nx) * s->facet;
    double y = (iy + 0.5 - 0.5 * s->ny) * s->facet;
    double xf[3] = {x, y, state[0]};
    double dt[3] = {xf[0] - g->ptx[0], xf[1] - g->ptx[1], xf[2] - g->ptx[2]};
    double dr[3] = {xf[0] - g->prx[0], xf[1] - g->prx[1], xf[2] - g->prx[2]};
    double rt = norm3(dt), rr = norm3(dr);
    double ut[3] = {dt[0] / rt, dt[1] / rt, dt[2] / rt};
    double ur[3] = {dr[0] / rr, dr[1] / rr, dr[2] / rr};
    double gt = or_pattern(s->tx.len_az, s->tx.len_el, lambda, ut, g->atx, g->etx);
    double gr = or_pattern(s->rx[c].len_az, s->rx[c].len_el, lambda, ur, g->arx, g->erx);
    double base = s->sigma0_base, cu = s->cur_u, cv = s->cur_v;
    if (s->cell_sigma0 || s->cell_uv) {
        int ci = cell_index(s, x, y);
        if (s->cell_sigma0) base = s->cell_sigma0[ci];
        if (s->cell_uv) {
            cu = s->cell_uv[2 * ci];
            cv = s->cell_uv[2 * ci + 1];
        }
    }
    double sig = or_sigma0(s, base, ut, ur, state[1], state[2]);
    double area = s->facet * s->facet;
    double amp = sqrt(sig * area) * gt * gr * (g->rt_ref * g->rr_ref) / (rt * rr);
    uint32_t e = s->epoch_pulses > 0 ? (uint32_t)(n / s->epoch_pulses) : 0u;
    double zr, zi;
    or_speckle(s->speckle_seed, (uint64_t)f, e, &zr, &zi);
    double vc = cu * (ut[0] + ur[0]) + cv * (ut[1] + ur[1]);
    double phase = -k0 * (rt + rr + vc * g->t);
    if (sumx) *sumx = ut[0] + ur[0];
    if (sumy) *sumy = ut[1] + ur[1];
    if (cell) *cell = (s->ncx > 0) ? cell_index(s, x, y) : -1;
    double cph = cos(phase), sph = sin(phase);
    double ar = amp * zr, ai = amp * zi;
    *sre = ar * cph - ai * sph;
    *sim = ar * sph + ai * cph;
    *p = (rt + rr - r0) / (OR_C / s->fs);
}

static void contribution(const or_scene *s, const or_pulse *g, int n, int c, int64_t f,
                         const double state[3], double r0, double *sre, double *sim, double *p)
{
    contribution_full(s, g, n, c, f, state, r0, sre, sim, p, NULL, NULL, NULL);
}

/* Neumaier compensated add of v into (sum, comp). */
static void neumaier(double *sum, double *comp, double v)
{
    double t = *sum + v;
    if (fabs(*sum) >= fabs(v))
        *comp += (*sum - t) + v;
    else
        *comp += (v - t) + *sum;
    *sum = t;
}

/* Spread one contribution onto the range bins (Eq. 17 box when taps == 1,
   Kaiser-windowed sinc of half-width taps/2 otherwise). */
static void spread(const or_scene *s, double sre, double sim, double p, double *sr, double *cr,
                   double *si, double *ci)
{
    int nr = s->n_range;
    if (s->taps == 1) {
        double fk = floor(p);
        if (fk < 0.0 || fk >= nr) return;
        int k = (int)fk;
        neumaier(&sr[k], &cr[k], sre);
        neumaier(&si[k], &ci[k], sim);
        return;
    }
    int m = s->taps / 2;
    double fk0 = floor(p);
    if (fk0 < -(double)m - 1.0 || fk0 > (double)nr + m) return;
    int k0 = (int)fk0;
    for (int k = k0 - m + 1; k <= k0 + m; ++k) {
        if (k < 0 || k >= nr) continue;
        double h = or_kaiser_sinc((double)k - p, m, s->beta);
        neumaier(&sr[k], &cr[k], h * sre);
        neumaier(&si[k], &ci[k], h * sim);
    }
}

/* Speckle epoch of pulse n. */
uint32_t or_epoch(const or_scene *s, int n)
{
    return s->epoch_pulses > 0 ? (uint32_t)(n / s->epoch_pulses) : 0u;
}

/* Facet states (eta, eta_x, eta_y) of all facets at pulse n (scene time t_s at
   the scene centre), written to out[3][nf]. Zero for a static surface. */
void or_facet_states(const or_scene *s, int n, int nw, const double *kx, const double *ky,
                     const double *om, const double *amp, const double *ph, double *out)
{
    int64_t nf = (int64_t)s->nx * s->ny;
    or_pulse g;
    or_pulse_state(s, n, 0, &g);
    if (s->static_surface || nw == 0) {
        memset(out, 0, sizeof(double) * 3 * nf);
        return;
    }
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < nf; ++f) {
        int ix = (int)(f % s->nx), iy = (int)(f / s->nx);
        double x = (ix + 0.5 - 0.5 * s->nx) * s->facet;
        double y = (iy + 0.5 - 0.5 * s->ny) * s->facet;
        double st[3];
        or_surface(nw, kx, ky, om, amp, ph, x, y, g.ts, st);
        out[f] = st[0];
        out[nf + f] = st[1];
        out[2 * nf + f] = st[2];
    }
}

/* Facet states of the listed facets at pulse n: out[3][count] in list order. */
static void list_states(const or_scene *s, int n, int nw, const double *kx, const double *ky, const double *om,
                        const double *amp, const double *ph, int64_t count, const int64_t *facets, double *out)
{
    or_pulse g;
    or_pulse_state(s, n, 0, &g);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < count; ++q) {
        double st[3] = {0.0, 0.0, 0.0};
        if (!s->static_surface && nw > 0) {
            int64_t f = facets[q];
            int ix = (int)(f % s->nx), iy = (int)(f / s->nx);
            double x = (ix + 0.5 - 0.5 * s->nx) * s->facet;
            double y = (iy + 0.5 - 0.5 * s->ny) * s->facet;
            or_surface(nw, kx, ky, om, amp, ph, x, y, g.ts, st);
        }
        out[q] = st[0];
        out[count + q] = st[1];
        out[2 * count + q] = st[2];
    }
}

/* IQ of the listed pulses: iq[c][i][k][2] for pulse pulses[i], all channels,
   summing the facets listed in facets[0..n_fac) (all facets when facets is
   NULL). */
int or_echo(const or_scene *s, int n_list, const int *pulses, int64_t n_fac, const int64_t *facets,
            double *iq)
{
    int nc = s->n_channels, nr = s->n_range;
    int64_t nf = (int64_t)s->nx * s->ny;
    int nw = (s->static_surface ? 0 : s->n_omega * s->n_theta);
    double *kx = NULL, *ky = NULL, *om = NULL, *amp = NULL, *ph = NULL;
    if (nw > 0) {
        kx = malloc(sizeof(double) * nw); ky = malloc(sizeof(double) * nw);
        om = malloc(sizeof(double) * nw); amp = malloc(sizeof(double) * nw);
        ph = malloc(sizeof(double) * nw);
        or_wave_table(s, kx, ky, om, amp, ph);
    }
    int64_t nsum = facets ? n_fac : nf;
    /* states of the summed facets only: st[3][nsum] in list order */
    double *st = malloc(sizeof(double) * 3 * (nsum > 0 ? nsum : 1));
    double r0[OR_MAXC];
    for (int c = 0; c < nc; ++c) r0[c] = or_range_start(s, c);
    for (int i = 0; i < n_list; ++i) {
        int n = pulses[i];
        if (facets)
            list_states(s, n, nw, kx, ky, om, amp, ph, nsum, facets, st);
        else
            or_facet_states(s, n, nw, kx, ky, om, amp, ph, st);
#pragma omp parallel for schedule(dynamic, 1)
        for (int c = 0; c < nc; ++c) {
            or_pulse g;
            or_pulse_state(s, n, c, &g);
            double *sr = calloc(nr, sizeof(double)), *cr = calloc(nr, sizeof(double));
            double *si = calloc(nr, sizeof(double)), *ci = calloc(nr, sizeof(double));
            for (int64_t q = 0; q < nsum; ++q) {
                int64_t f = facets ? facets[q] : q;
                double state[3] = {st[q], st[nsum + q], st[2 * nsum + q]};
                double sre, sim, p;
                contribution(s, &g, n, c, f, state, r0[c], &sre, &sim, &p);
                spread(s, sre, sim, p, sr, cr, si, ci);
            }
            double *row = iq + ((int64_t)c * n_list + i) * nr * 2;
            for (int k = 0; k < nr; ++k) {
                row[2 * k] = sr[k] + cr[k];
                row[2 * k + 1] = si[k] + ci[k];
            }
            free(sr); free(cr); free(si); free(ci);
        }
    }
    free(st);
    free(kx); free(ky); free(om); free(amp); free(ph);
    return 0;
}

/* One facet's contribution (complex value and bin position) for tests:
   out = {re, im, p}. */
void or_contribution(const or_scene *s, int n, int c, int64_t f, const double state[3], double *out)
{
    or_pulse g;
    or_pulse_state(s, n, c, &g);
    double r0 = or_range_start(s, c);
    contribution(s, &g, n, c, f, state, r0, &out[0], &out[1], &out[2]);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Adjoint of the echo with respect to the per-cell NRCS base and current, for
   the misfit L = sum |IQ - target|^2 with residual r = IQ - target given as
   resid[c][i][k][2] for the listed pulses. Chain rule on each contribution s
   spread with weights h(k - p): with g = sum_k h(k - p) r[k] (the transposed
   spread, a gather over the same bins),
     dL/dsigma_cell += Re(conj(g) s) / sigma_cell          (s ~ sqrt(sigma))
     dL/du_cell     += 2 K0 t_n (r_t + r_r)_x Im(conj(g) s) (phase -K0 v_c t_n)
     dL/dv_cell     += 2 K0 t_n (r_t + r_r)_y Im(conj(g) s)
   (Eq. 3 and Eq. 4). The current does not move range bins, so h does not
   depend on it. Gradients are added into g_sigma[ncells] / g_uv[ncells][2]. */
int or_adjoint(const or_scene *s, int n_list, const int *pulses, const double *resid, double *g_sigma,
               double *g_uv)
{
    if (s->ncx <= 0 || s->ncy <= 0) return -1;
    int nc = s->n_channels, nr = s->n_range;
    int64_t nf = (int64_t)s->nx * s->ny;
    int ncell = s->ncx * s->ncy;
    int nw = (s->static_surface ? 0 : s->n_omega * s->n_theta);
    double *kx = NULL, *ky = NULL, *om = NULL, *amp = NULL, *ph = NULL;
    if (nw > 0) {
        kx = malloc(sizeof(double) * nw); ky = malloc(sizeof(double) * nw);
        om = malloc(sizeof(double) * nw); amp = malloc(sizeof(double) * nw);
        ph = malloc(sizeof(double) * nw);
        or_wave_table(s, kx, ky, om, amp, ph);
    }
    double lambda = OR_C / s->f0;
    double k0 = 2.0 * OR_PI / lambda;
    double *st = malloc(sizeof(double) * 3 * nf);
    double r0[OR_MAXC];
    for (int c = 0; c < nc; ++c) r0[c] = or_range_start(s, c);
    /* per-channel partial gradients, summed in channel order at the end */
    double *part = calloc((size_t)nc * ncell * 3, sizeof(double));
    for (int i = 0; i < n_list; ++i) {
        int n = pulses[i];
        or_facet_states(s, n, nw, kx, ky, om, amp, ph, st);
#pragma omp parallel for schedule(dynamic, 1)
        for (int c = 0; c < nc; ++c) {
            or_pulse g;
            or_pulse_state(s, n, c, &g);
            const double *row = resid + ((int64_t)c * n_list + i) * nr * 2;
            double *pc = part + (size_t)c * ncell * 3;
            for (int64_t f = 0; f < nf; ++f) {
                double state[3] = {st[f], st[nf + f], st[2 * nf + f]};
                double sre, sim, p, sx, sy;
                int cell;
                contribution_full(s, &g, n, c, f, state, r0[c], &sre, &sim, &p, &sx, &sy, &cell);
                double gr = 0.0, gi = 0.0;
                if (s->taps == 1) {
                    double fk = floor(p);
                    if (fk >= 0.0 && fk < nr) {
                        gr = row[2 * (int)fk];
                        gi = row[2 * (int)fk + 1];
                    }
                } else {
                    int m = s->taps / 2;
                    double fk0 = floor(p);
                    if (fk0 >= -(double)m - 1.0 && fk0 <= (double)nr + m) {
                        int kk0 = (int)fk0;
                        for (int k = kk0 - m + 1; k <= kk0 + m; ++k) {
                            if (k < 0 || k >= nr) continue;
                            double h = or_kaiser_sinc((double)k - p, m, s->beta);
                            gr += h * row[2 * k];
                            gi += h * row[2 * k + 1];
                        }
                    }
                }
                double re_gs = gr * sre + gi * sim;
                double im_gs = gr * sim - gi * sre;
                double sig = s->cell_sigma0 ? s->cell_sigma0[cell] : s->sigma0_base;
                if (sig > 0.0) pc[3 * cell] += re_gs / sig;
                pc[3 * cell + 1] += 2.0 * k0 * g.t * sx * im_gs;
                pc[3 * cell + 2] += 2.0 * k0 * g.t * sy * im_gs;
            }
        }
    }
    for (int c = 0; c < nc; ++c)
        for (int q = 0; q < ncell; ++q) {
            if (g_sigma) g_sigma[q] += part[((size_t)c * ncell + q) * 3];
            if (g_uv) {
                g_uv[2 * q] += part[((size_t)c * ncell + q) * 3 + 1];
                g_uv[2 * q + 1] += part[((size_t)c * ncell + q) * 3 + 2];
            }
        }
    free(part);
    free(st);
    free(kx); free(ky); free(om); free(amp); free(ph);
    return 0;
}
