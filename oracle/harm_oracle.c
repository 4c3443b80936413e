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
 *   - Surface and scattering variants of Sec. III: the Choppy Wave Model
 *     (horizontal displacement of the grid points along the waves' orbits),
 *     heterogeneous sea states built from four overlapping homogeneous tiles
 *     (Eq. 1, Eq. 2), the order-1 autoregressive speckle (Eq. 10) with the
 *     intra-facet Doppler shift of Eq. 7, and antenna gains looked up in u-v
 *     grids (Sec. III-B).
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

/* Complex antenna gain on a regular u-v grid (direction cosines along the
   antenna's azimuth and elevation axes); g == NULL selects the analytic
   sinc^2 pattern. */
typedef struct {
    int nu, nv;
    double u0, du, v0, dv;
    const double *g; /* [nv][nu][2] */
} or_lut;

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
    /* variants of Sec. III (all off when zero / NULL) */
    double tau_s;      /* AR(1) speckle correlation time (Eq. 10); 0 = independent epochs */
    double doppler_hz; /* intra-facet Doppler shift f_s (Eq. 7) */
    int cwm;           /* Choppy Wave Model horizontal displacement */
    double het_l;      /* heterogeneous sea state: TL tile size L (Eq. 1, 2) */
    int het_ncx, het_ncy;       /* corner grid, corner (cx, cy) at the patch corner + (cx, cy) L */
    const double *het_u10;      /* [het_ncy][het_ncx] wind speed of corner spectrum S_i */
    const double *het_dir;      /* [het_ncy][het_ncx] wind direction of corner spectrum S_i */
    or_lut lut[1 + OR_MAXC];    /* [0] transmitter, [1 + c] receive channel c */
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

/* AR(1) memory of the speckle between consecutive epochs (Eq. 10): beta =
   exp(-T_e / tau_s) for the epoch duration T_e; tau_s = 0 gives beta = 0
   (independent epochs). */
double or_speckle_beta(const or_scene *s)
{
    if (!(s->tau_s > 0.0) || s->epoch_pulses <= 0) return 0.0;
    return exp(-((double)s->epoch_pulses / s->prf) / s->tau_s);
}

/* Speckle of facet f in epoch e under the order-1 autoregressive model of
   Eq. 10, applied to R and I alike: s_0 = w_0 and s_e = beta s_(e-1) +
   sqrt(1 - beta^2) w_e, where w_e is the independent draw of or_speckle for
   epoch e (R', I' of variance 1/2, so E|s_e|^2 = 1 for every e). The
   recurrence is run from epoch 0. */
void or_speckle_ar1(uint64_t seed, uint64_t f, uint32_t epoch, double beta, double *re, double *im)
{
    if (beta == 0.0) {
        or_speckle(seed, f, epoch, re, im);
        return;
    }
    double zr, zi;
    or_speckle(seed, f, 0u, &zr, &zi);
    double q = sqrt(1.0 - beta * beta);
    for (uint32_t e = 1; e <= epoch; ++e) {
        double wr, wi;
        or_speckle(seed, f, e, &wr, &wi);
        zr = beta * zr + q * wr;
        zi = beta * zi + q * wi;
    }
    *re = zr;
    *im = zi;
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
static int wave_table_for(const or_scene *s, double u10, double wind_dir, uint32_t word2, double *kx,
                          double *ky, double *om, double *amp, double *ph)
{
    int no = s->n_omega, nt = s->n_theta;
    if (no <= 0 || nt <= 0) return 0;
    double wp, alpha;
    or_jonswap_params(u10, s->fetch, &wp, &alpha);
    double lo = 0.7 * wp, hi = 2.5 * wp;
    double dth = 2.0 * OR_PI / nt;
    for (int i = 0; i < no; ++i) {
        double e0 = lo * pow(hi / lo, (double)i / no);
        double e1 = lo * pow(hi / lo, (double)(i + 1) / no);
        double w = sqrt(e0 * e1);
        double dw = e1 - e0;
        double sw = or_jonswap(w, u10, s->fetch, s->gamma);
        double k = w * w / OR_G;
        for (int j = 0; j < nt; ++j) {
            int m = i * nt + j;
            double th = wind_dir - OR_PI + (j + 0.5) * dth;
            double d = or_spreading(th - wind_dir, s->spread_s);
            kx[m] = k * cos(th);
            ky[m] = k * sin(th);
            om[m] = w;
            amp[m] = sqrt(2.0 * sw * dw * d * dth);
            uint32_t r[4];
            philox_draw(s->wave_seed, (uint32_t)m, word2, OR_STREAM_WAVE, r);
            ph[m] = 2.0 * OR_PI * ((double)r[0] * (1.0 / 4294967296.0));
        }
    }
    return no * nt;
}

int or_wave_table(const or_scene *s, double *kx, double *ky, double *om, double *amp, double *ph)
{
    return wave_table_for(s, s->u10, s->wind_dir, 0u, kx, ky, om, amp, ph);
}

/* Wave table of the homogeneous tile T2L_i centred on corner i = cy * ncx + cx
   of a heterogeneous sea state (Eq. 1): the corner's own spectrum S_i (wind
   speed and direction; fetch, peak enhancement and spreading of the scene) and
   its own random phases (Philox word 2 = 1 + i), uncorrelated with every other
   corner. */
int or_wave_table_corner(const or_scene *s, int corner, double *kx, double *ky, double *om, double *amp,
                         double *ph)
{
    return wave_table_for(s, s->het_u10[corner], s->het_dir[corner], 1u + (uint32_t)corner, kx, ky, om, amp, ph);
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

/* Choppy Wave Model (Sec. III; Nouguier, Guerin & Chapron, JGR 2009): the
   grid point at rest position (x, y) moves horizontally by
   D = -sum_j a_j (k_j / |k_j|) sin(theta_j) while its height is the linear
   eta = sum_j a_j cos(theta_j), theta_j = k_j . (x, y) - omega_j t + phi_j.
   out = (eta, deta/dx, deta/dy, D_x, D_y, dD_x/dx, dD_x/dy, dD_y/dy), every
   derivative taken with respect to the rest position (dD_y/dx = dD_x/dy). */
void or_surface_cwm(int nw, const double *kx, const double *ky, const double *om, const double *amp,
                    const double *ph, double x, double y, double t, double out[8])
{
    for (int q = 0; q < 8; ++q) out[q] = 0.0;
    for (int m = 0; m < nw; ++m) {
        double arg = kx[m] * x + ky[m] * y - om[m] * t + ph[m];
        double c = cos(arg), sn = sin(arg);
        double k = sqrt(kx[m] * kx[m] + ky[m] * ky[m]);
        double ux = kx[m] / k, uy = ky[m] / k;
        out[0] += amp[m] * c;
        out[1] -= amp[m] * kx[m] * sn;
        out[2] -= amp[m] * ky[m] * sn;
        out[3] -= amp[m] * ux * sn;
        out[4] -= amp[m] * uy * sn;
        out[5] -= amp[m] * ux * kx[m] * c;
        out[6] -= amp[m] * ux * ky[m] * c;
        out[7] -= amp[m] * uy * ky[m] * c;
    }
}

/* The wave sets of a scene: one table for a homogeneous sea state, one per
   corner of the TL-tile grid for a heterogeneous one. */
typedef struct {
    int n_sets, nw;
    double *kx, *ky, *om, *amp, *ph; /* [n_sets][nw] */
} or_waves;

static void waves_build(const or_scene *s, or_waves *W)
{
    W->nw = s->static_surface ? 0 : s->n_omega * s->n_theta;
    W->n_sets = s->het_ncx > 0 ? s->het_ncx * s->het_ncy : 1;
    size_t n = (size_t)W->n_sets * (W->nw > 0 ? W->nw : 1);
    W->kx = calloc(n, sizeof(double));
    W->ky = calloc(n, sizeof(double));
    W->om = calloc(n, sizeof(double));
    W->amp = calloc(n, sizeof(double));
    W->ph = calloc(n, sizeof(double));
    if (W->nw == 0) return;
    for (int i = 0; i < W->n_sets; ++i) {
        size_t o = (size_t)i * W->nw;
        if (s->het_ncx > 0)
            or_wave_table_corner(s, i, W->kx + o, W->ky + o, W->om + o, W->amp + o, W->ph + o);
        else
            or_wave_table(s, W->kx + o, W->ky + o, W->om + o, W->amp + o, W->ph + o);
    }
}

static void waves_free(or_waves *W)
{
    free(W->kx); free(W->ky); free(W->om); free(W->amp); free(W->ph);
}

/* TL tile of a rest position: the corner grid starts at the patch corner with
   step L; positions on the last corner line belong to the tile before it. */
static void hetero_tile(const or_scene *s, double x, double y, int *tx, int *ty)
{
    double lx = s->nx * s->facet, ly = s->ny * s->facet;
    int ix = (int)floor((x + 0.5 * lx) / s->het_l);
    int iy = (int)floor((y + 0.5 * ly) / s->het_l);
    if (ix < 0) ix = 0;
    if (ix > s->het_ncx - 2) ix = s->het_ncx - 2;
    if (iy < 0) iy = 0;
    if (iy > s->het_ncy - 2) iy = s->het_ncy - 2;
    *tx = ix;
    *ty = iy;
}

/* Weight W^i of corner i = (cx, cy) at rest position (x, y) (Eq. 2):
   sqrt(1 - w_x - w_y + w_x w_y) with w_x = |x_i - x| / L, w_y = |y_i - y| / L,
   for the four corners of the position's TL tile; zero for every other corner. */
double or_hetero_weight(const or_scene *s, int cx, int cy, double x, double y)
{
    int tx, ty;
    hetero_tile(s, x, y, &tx, &ty);
    if (cx < tx || cx > tx + 1 || cy < ty || cy > ty + 1) return 0.0;
    double xc = -0.5 * s->nx * s->facet + cx * s->het_l;
    double yc = -0.5 * s->ny * s->facet + cy * s->het_l;
    double wx = fabs(xc - x) / s->het_l, wy = fabs(yc - y) / s->het_l;
    double v = 1.0 - wx - wy + wx * wy;
    return v > 0.0 ? sqrt(v) : 0.0;
}

/* State of the facet at rest position (x, y) at scene time t: the 8 fields of
   or_surface_cwm. A heterogeneous sea state sums the four overlapping
   homogeneous tiles with the weights of Eq. 2 (Eq. 1), applied alike to every
   field (the weights are constants of the position, so the slopes and the
   displacement gradient are combined with the same weights). Without the CWM
   the horizontal displacement and its gradient are zero (linear surface). */
void or_facet_state(const or_scene *s, const or_waves *W, double x, double y, double t, double out[8])
{
    for (int q = 0; q < 8; ++q) out[q] = 0.0;
    if (W->nw == 0) return;
    if (s->het_ncx > 0) {
        int tx, ty;
        hetero_tile(s, x, y, &tx, &ty);
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                int cx = tx + dx, cy = ty + dy;
                double w = or_hetero_weight(s, cx, cy, x, y);
                if (w == 0.0) continue;
                size_t o = (size_t)(cy * s->het_ncx + cx) * W->nw;
                double tmp[8];
                or_surface_cwm(W->nw, W->kx + o, W->ky + o, W->om + o, W->amp + o, W->ph + o, x, y, t, tmp);
                for (int q = 0; q < 8; ++q) out[q] += w * tmp[q];
            }
    } else {
        or_surface_cwm(W->nw, W->kx, W->ky, W->om, W->amp, W->ph, x, y, t, out);
    }
    if (!s->cwm)
        for (int q = 3; q < 8; ++q) out[q] = 0.0;
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

/* Complex gain at direction cosines (u, v) from a u-v grid (Sec. III-B: the
   patterns are converted to u-v grids and looked up per facet and pulse):
   bilinear interpolation between the four surrounding nodes; zero outside the
   grid. out = (re, im). */
void or_lut_gain(const or_lut *L, double u, double v, double out[2])
{
    out[0] = out[1] = 0.0;
    double fu = (u - L->u0) / L->du, fv = (v - L->v0) / L->dv;
    if (!(fu >= 0.0 && fu <= (double)(L->nu - 1) && fv >= 0.0 && fv <= (double)(L->nv - 1))) return;
    int iu = (int)floor(fu), iv = (int)floor(fv);
    if (iu > L->nu - 2) iu = L->nu - 2;
    if (iv > L->nv - 2) iv = L->nv - 2;
    double a = fu - iu, b = fv - iv;
    const double *g00 = L->g + 2 * ((size_t)iv * L->nu + iu);
    const double *g10 = g00 + 2;
    const double *g01 = g00 + 2 * (size_t)L->nu;
    const double *g11 = g01 + 2;
    for (int q = 0; q < 2; ++q)
        out[q] = (1.0 - a) * (1.0 - b) * g00[q] + a * (1.0 - b) * g10[q] + (1.0 - a) * b * g01[q] + a * b * g11[q];
}

/* Gain of one antenna for the unit direction d from its phase centre: the u-v
   grid when one is set, else the analytic sinc^2 pattern (real). */
static void antenna_gain(const or_lut *L, double len_az, double len_el, double lambda, const double d[3],
                         const double a[3], const double e[3], double out[2])
{
    if (L->g) {
        double u = d[0] * a[0] + d[1] * a[1] + d[2] * a[2];
        double v = d[0] * e[0] + d[1] * e[1] + d[2] * e[2];
        or_lut_gain(L, u, v, out);
    } else {
        out[0] = or_pattern(len_az, len_el, lambda, d, a, e);
        out[1] = 0.0;
    }
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
double or_sigma0_normal(const or_scene *s, double base, const double rt_hat[3], const double rr_hat[3],
                        const double nvec[3])
{
    if (s->static_surface) return base;
    double q[3] = {-(rt_hat[0] + rr_hat[0]), -(rt_hat[1] + rr_hat[1]), -(rt_hat[2] + rr_hat[2])};
    double qh = sqrt(q[0] * q[0] + q[1] * q[1]);
    double cphi = 0.0;
    if (qh > 0.0) cphi = (cos(s->wind_dir) * q[0] + sin(s->wind_dir) * q[1]) / qh;
    double ndotq = nvec[0] * q[0] + nvec[1] * q[1] + nvec[2] * q[2];
    double tilt = (ndotq > 0.0 ? ndotq : 0.0) / (norm3(nvec) * q[2]);
    return base * (1.0 + s->wind_mod * cphi) * tilt;
}

/* The same for a facet of the linear surface with slopes (slope_x, slope_y):
   normal n = (-slope_x, -slope_y, 1). */
double or_sigma0(const or_scene *s, double base, const double rt_hat[3], const double rr_hat[3],
                 double slope_x, double slope_y)
{
    double nvec[3] = {-slope_x, -slope_y, 1.0};
    return or_sigma0_normal(s, base, rt_hat, rr_hat, nvec);
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

/* One facet's complex contribution at pulse state g (Eq. 3, 4, 7, 16) and its
   fractional range-bin position p. state = the 8 fields of or_facet_state. The
   facet sits at its rest position moved by the horizontal displacement (zero
   without the CWM) and lifted to eta; its normal is the cross product of the
   tangents (1 + dD_x/dx, dD_x/dy, deta/dx) and (dD_x/dy, 1 + dD_y/dy, deta/dy)
   of the displaced surface, and its area is the facet area times the normal's
   vertical component (the horizontal area of the displaced facet; 1 for the
   linear surface). */
static void contribution_full(const or_scene *s, const or_pulse *g, int n, int c, int64_t f,
                              const double state[8], double r0, double *sre, double *sim, double *p,
                              double *sumx, double *sumy, int *cell)
{
    double lambda = OR_C / s->f0;
    double k0 = 2.0 * OR_PI / lambda;
    int ix = (int)(f % s->nx), iy = (int)(f / s->nx);
    double x = (ix + 0.5 - 0.5 * s->nx) * s->facet;
    double y = (iy + 0.5 - 0.5 * s->ny) * s->facet;
    double xf[3] = {x + state[3], y + state[4], state[0]};
    double dt[3] = {xf[0] - g->ptx[0], xf[1] - g->ptx[1], xf[2] - g->ptx[2]};
    double dr[3] = {xf[0] - g->prx[0], xf[1] - g->prx[1], xf[2] - g->prx[2]};
    double rt = norm3(dt), rr = norm3(dr);
    double ut[3] = {dt[0] / rt, dt[1] / rt, dt[2] / rt};
    double ur[3] = {dr[0] / rr, dr[1] / rr, dr[2] / rr};
    double gt[2], gr[2];
    antenna_gain(&s->lut[0], s->tx.len_az, s->tx.len_el, lambda, ut, g->atx, g->etx, gt);
    antenna_gain(&s->lut[1 + c], s->rx[c].len_az, s->rx[c].len_el, lambda, ur, g->arx, g->erx, gr);
    double base = s->sigma0_base, cu = s->cur_u, cv = s->cur_v;
    if (s->cell_sigma0 || s->cell_uv) {
        int ci = cell_index(s, x, y);
        if (s->cell_sigma0) base = s->cell_sigma0[ci];
        if (s->cell_uv) {
            cu = s->cell_uv[2 * ci];
            cv = s->cell_uv[2 * ci + 1];
        }
    }
    double tx_[3] = {1.0 + state[5], state[6], state[1]};
    double ty_[3] = {state[6], 1.0 + state[7], state[2]};
    double nvec[3] = {tx_[1] * ty_[2] - tx_[2] * ty_[1], tx_[2] * ty_[0] - tx_[0] * ty_[2],
                      tx_[0] * ty_[1] - tx_[1] * ty_[0]};
    double sig = or_sigma0_normal(s, base, ut, ur, nvec);
    double area = s->facet * s->facet * (nvec[2] > 0.0 ? nvec[2] : 0.0);
    double amp = sqrt(sig * area) * (g->rt_ref * g->rr_ref) / (rt * rr);
    uint32_t e = s->epoch_pulses > 0 ? (uint32_t)(n / s->epoch_pulses) : 0u;
    double zr, zi;
    or_speckle_ar1(s->speckle_seed, (uint64_t)f, e, or_speckle_beta(s), &zr, &zi);
    double vc = cu * (ut[0] + ur[0]) + cv * (ut[1] + ur[1]);
    double phase = -k0 * (rt + rr + vc * g->t) + 2.0 * OR_PI * s->doppler_hz * g->t;
    if (sumx) *sumx = ut[0] + ur[0];
    if (sumy) *sumy = ut[1] + ur[1];
    if (cell) *cell = (s->ncx > 0) ? cell_index(s, x, y) : -1;
    /* field weight G_t G_r (complex for u-v grids) times the speckle */
    double gre = gt[0] * gr[0] - gt[1] * gr[1], gim = gt[0] * gr[1] + gt[1] * gr[0];
    double wr = zr * gre - zi * gim, wi = zr * gim + zi * gre;
    double cph = cos(phase), sph = sin(phase);
    double ar = amp * wr, ai = amp * wi;
    *sre = ar * cph - ai * sph;
    *sim = ar * sph + ai * cph;
    *p = (rt + rr - r0) / (OR_C / s->fs);
}

static void contribution(const or_scene *s, const or_pulse *g, int n, int c, int64_t f,
                         const double state[8], double r0, double *sre, double *sim, double *p)
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

/* Facet states (the 8 fields of or_facet_state) of all facets at pulse n, at
   the scene time t_s of the scene centre, written to out[8][nf]. Zero for a
   static surface. */
static void facet_states_w(const or_scene *s, const or_waves *W, int n, double *out)
{
    int64_t nf = (int64_t)s->nx * s->ny;
    or_pulse g;
    or_pulse_state(s, n, 0, &g);
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < nf; ++f) {
        int ix = (int)(f % s->nx), iy = (int)(f / s->nx);
        double x = (ix + 0.5 - 0.5 * s->nx) * s->facet;
        double y = (iy + 0.5 - 0.5 * s->ny) * s->facet;
        double st[8];
        or_facet_state(s, W, x, y, g.ts, st);
        for (int q = 0; q < 8; ++q) out[q * nf + f] = st[q];
    }
}

void or_facet_states(const or_scene *s, int n, double *out)
{
    or_waves W;
    waves_build(s, &W);
    facet_states_w(s, &W, n, out);
    waves_free(&W);
}

/* Facet states of the listed facets at pulse n: out[8][count] in list order. */
static void list_states(const or_scene *s, const or_waves *W, int n, int64_t count, const int64_t *facets,
                        double *out)
{
    or_pulse g;
    or_pulse_state(s, n, 0, &g);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < count; ++q) {
        int64_t f = facets[q];
        int ix = (int)(f % s->nx), iy = (int)(f / s->nx);
        double x = (ix + 0.5 - 0.5 * s->nx) * s->facet;
        double y = (iy + 0.5 - 0.5 * s->ny) * s->facet;
        double st[8];
        or_facet_state(s, W, x, y, g.ts, st);
        for (int k = 0; k < 8; ++k) out[k * count + q] = st[k];
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
    or_waves W;
    waves_build(s, &W);
    int64_t nsum = facets ? n_fac : nf;
    /* states of the summed facets only: st[8][nsum] in list order */
    double *st = malloc(sizeof(double) * 8 * (nsum > 0 ? nsum : 1));
    double r0[OR_MAXC];
    for (int c = 0; c < nc; ++c) r0[c] = or_range_start(s, c);
    for (int i = 0; i < n_list; ++i) {
        int n = pulses[i];
        if (facets)
            list_states(s, &W, n, nsum, facets, st);
        else
            facet_states_w(s, &W, n, st);
#pragma omp parallel for schedule(dynamic, 1)
        for (int c = 0; c < nc; ++c) {
            or_pulse g;
            or_pulse_state(s, n, c, &g);
            double *sr = calloc(nr, sizeof(double)), *cr = calloc(nr, sizeof(double));
            double *si = calloc(nr, sizeof(double)), *ci = calloc(nr, sizeof(double));
            for (int64_t q = 0; q < nsum; ++q) {
                int64_t f = facets ? facets[q] : q;
                double state[8];
                for (int k = 0; k < 8; ++k) state[k] = st[k * nsum + q];
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
    waves_free(&W);
    return 0;
}

/* Bin positions of every facet at the listed pulses (for the parity of the
   accumulator's integer bins): p_out[i][c][f] is the fractional range-bin
   position p = (r_t + r_r - R0_c) / dr of facet f's contribution to channel c at
   pulse pulses[i] (the p that `spread` turns into taps k = floor(p) - 3 ...
   floor(p) + 4), and cell_out[f] its cell index (-1 without per-cell fields). */
int or_bin_positions(const or_scene *s, int n_list, const int *pulses, double *p_out, int *cell_out)
{
    int nc = s->n_channels;
    int64_t nf = (int64_t)s->nx * s->ny;
    or_waves W;
    waves_build(s, &W);
    double *st = malloc(sizeof(double) * 8 * (nf > 0 ? nf : 1));
    double r0[OR_MAXC];
    for (int c = 0; c < nc; ++c) r0[c] = or_range_start(s, c);
    for (int i = 0; i < n_list; ++i) {
        int n = pulses[i];
        facet_states_w(s, &W, n, st);
        for (int c = 0; c < nc; ++c) {
            or_pulse g;
            or_pulse_state(s, n, c, &g);
            double *row = p_out + ((int64_t)i * nc + c) * nf;
#pragma omp parallel for schedule(static)
            for (int64_t f = 0; f < nf; ++f) {
                double state[8];
                for (int k = 0; k < 8; ++k) state[k] = st[k * nf + f];
                double sre, sim, p;
                int cell;
                contribution_full(s, &g, n, c, f, state, r0[c], &sre, &sim, &p, NULL, NULL, &cell);
                row[f] = p;
                if (i == 0 && c == 0 && cell_out) cell_out[f] = cell;
            }
        }
    }
    free(st);
    waves_free(&W);
    return 0;
}

/* Philox words of the speckle draws of count (facet, epoch) pairs:
   out[4 q .. 4 q + 3] for counter (facet[q], 0, epoch[q], 0) under the speckle
   key (the words or_speckle turns into a draw). */
void or_speckle_words(uint64_t seed, int64_t count, const uint32_t *facet, const uint32_t *epoch, uint32_t *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < count; ++q) philox_draw(seed, facet[q], epoch[q], OR_STREAM_SPECKLE, out + 4 * q);
}

/* One facet's contribution (complex value and bin position) for tests:
   out = {re, im, p}. */
void or_contribution(const or_scene *s, int n, int c, int64_t f, const double state[8], double *out)
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

/* Threads of later parallel regions (timing only; results do not depend on it). */
void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
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
    or_waves W;
    waves_build(s, &W);
    double lambda = OR_C / s->f0;
    double k0 = 2.0 * OR_PI / lambda;
    double *st = malloc(sizeof(double) * 8 * nf);
    double r0[OR_MAXC];
    for (int c = 0; c < nc; ++c) r0[c] = or_range_start(s, c);
    /* per-channel partial gradients, summed in channel order at the end */
    double *part = calloc((size_t)nc * ncell * 3, sizeof(double));
    for (int i = 0; i < n_list; ++i) {
        int n = pulses[i];
        facet_states_w(s, &W, n, st);
#pragma omp parallel for schedule(dynamic, 1)
        for (int c = 0; c < nc; ++c) {
            or_pulse g;
            or_pulse_state(s, n, c, &g);
            const double *row = resid + ((int64_t)c * n_list + i) * nr * 2;
            double *pc = part + (size_t)c * ncell * 3;
            for (int64_t f = 0; f < nf; ++f) {
                double state[8];
                for (int k = 0; k < 8; ++k) state[k] = st[k * nf + f];
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
    waves_free(&W);
    return 0;
}
