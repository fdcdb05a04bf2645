/*
 * mc_oracle.c -- plain, slow CPU oracle for the checkerboard local-update sweep of
 * Demchik & Strelchenko, "Monte Carlo simulations on Graphics Processing Units"
 * (arXiv:0903.3053).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The CUDA
 * product path shares no code, header or table with this file.
 *
 * What it computes, step by step and in the paper's order:
 *   - Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
 *     easy as 1, 2, 3", SC'11), the counter-based stream that replaces the
 *     paper's RANMAR (Sec. 2.2), keyed by (seed) with counters (site, sweep,
 *     tag, chain).
 *   - 2D Ising model, Eq. (1), Metropolis single-spin updates on the red/black
 *     checkerboard (Sec. 2.3), one colour after the other (Sec. 2.1).
 *   - 4D SU(2) Wilson gauge theory, Eqs. (2)-(3), heat-bath link replacement of
 *     Eqs. (5)-(7) with the staple of Eq. (6), links parametrised as in Eq. (4),
 *     odd sites before even sites and mu = 0..3 within each (Sec. 2.4).
 *     Links are held as FP64 2x2 complex matrices -- deliberately a different
 *     formulation from the quaternion arithmetic of the GPU path.
 *
 * Readings of the paper that the paper leaves open are marked READING.
 * Every floating-point quantity is FP64.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al. SC'11, Sec. 3): 10 rounds of two 32x32->64     */
/* multiplications, the "S-box" being the hi/lo halves of the products, with a */
/* Weyl-sequence key schedule.                                                 */
/* ------------------------------------------------------------------------- */
static const uint32_t PHILOX_MUL0 = 0xD2511F53u;
static const uint32_t PHILOX_MUL1 = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL0 = 0x9E3779B9u; /* golden ratio */
static const uint32_t PHILOX_WEYL1 = 0xBB67AE85u; /* sqrt(3) - 1 */

ORC_API void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_WEYL0;
            k1 += PHILOX_WEYL1;
        }
        uint64_t prod0 = (uint64_t)PHILOX_MUL0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)PHILOX_MUL1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* A run of n consecutive 32-bit words of one stream: word j is word (j & 3)
 * of the block with counter (j >> 2, c1, c2, c3) and key (seed low, seed
 * high) -- how every per-position draw below takes its random words. */
ORC_API void orc_philox_words(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, long n, uint32_t *out)
{
    for (long j = 0; j < n; j += 4) {
        uint32_t ctr[4] = {(uint32_t)(j >> 2), c1, c2, c3};
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        for (long i = j; i < n && i < j + 4; ++i)
            out[i] = r[i - j];
    }
}

/* Stream layout shared (as a specification, not as code) with the GPU path.
 * key = (seed low 32 bits, seed high 32 bits); counter = (c0, c1, c2, c3) with
 * c3 = chain id and c2's top byte a tag naming what the numbers are for.    */
#define TAG_ISING_INIT 0x01000000u
#define TAG_ISING_METRO 0x02000000u
#define TAG_SU2_INIT 0x11000000u
#define TAG_SU2_HB 0x12000000u
#define TAG_SU2_DIR 0x13000000u

static void philox_block(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                         uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Integer random word -> float in (0, 1]: the paper maps its 24-bit RANMAR
 * integers to [0, 1) (Sec. 2.2); READING: the same 24-bit resolution, shifted
 * by one step so that log() never sees 0. */
static double uniform01(uint32_t r) { return (double)((r >> 8) + 1u) * (1.0 / 16777216.0); }

/* ========================================================================= */
/* 2D Ising model, Eq. (1): H = - sum_<ij> s_i s_j, s = +-1, periodic torus. */
/* Spins are int8, row-major s[y*Lx + x].                                    */
/* ========================================================================= */

/* Metropolis acceptance exp(-beta*dE) for dE = 2*s_i*h_i > 0, i.e. dE = 4 and 8,
 * as 32-bit integer thresholds: T = floor(exp(-beta*dE) * 2^32), clamped to
 * 2^32 - 1.  A move with dE > 0 is accepted iff the site's random word r < T.
 * out[0] is the threshold for dE = 4, out[1] for dE = 8. */
ORC_API void orc_ising_thresholds(double beta, uint32_t out[2])
{
    for (int k = 0; k < 2; ++k) {
        double dE = 4.0 * (double)(k + 1);
        double t = exp(-beta * dE) * 4294967296.0;
        if (t >= 4294967295.0)
            out[k] = 0xFFFFFFFFu;
        else
            out[k] = (uint32_t)floor(t);
    }
}

/* Site (x, y) has colour c = (x + y) & 1 (red/black partition, Sec. 2.3) and
 * index i = y*(Lx/2) + x/2 within its colour class (READING: the paper gives no
 * indexing; this one makes the random word of a site independent of how spins
 * are packed in memory). */
static uint32_t colour_index(int x, int y, int Lx) { return (uint32_t)y * (uint32_t)(Lx / 2) + (uint32_t)(x >> 1); }

/* Random word of site i of colour c: word (i & 3) of the Philox block with
 * counter (i >> 2, c1, tag | c, chain). */
static uint32_t site_word(uint64_t seed, uint32_t chain, uint32_t c1, uint32_t tag, int c, uint32_t i)
{
    uint32_t out[4];
    philox_block(seed, i >> 2, c1, tag | (uint32_t)c, chain, out);
    return out[i & 3u];
}

/* Lattice initialisation, hot or cold (Sec. 2.1): cold = all +1; hot = each
 * spin +1 iff the top bit of its random word (sweep field 0, tag INIT) is 1. */
ORC_API void orc_ising_init(int8_t *s, int Lx, int Ly, uint64_t seed, uint32_t chain, int hot)
{
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            int8_t v = 1;
            if (hot) {
                int c = (x + y) & 1;
                uint32_t r = site_word(seed, chain, 0u, TAG_ISING_INIT, c, colour_index(x, y, Lx));
                v = (r >> 31) ? (int8_t)1 : (int8_t)-1;
            }
            s[y * Lx + x] = v;
        }
}

/* Local field h = sum of the four nearest neighbours on the periodic torus. */
static int ising_field(const int8_t *s, int Lx, int Ly, int x, int y)
{
    int xp = (x + 1) % Lx, xm = (x + Lx - 1) % Lx;
    int yp = (y + 1) % Ly, ym = (y + Ly - 1) % Ly;
    return s[y * Lx + xp] + s[y * Lx + xm] + s[yp * Lx + x] + s[ym * Lx + x];
}

/* One Metropolis sweep number `sweep` (Sec. 2.3, Sec. 2.1): first every site of
 * colour 0 ("even"), then every site of colour 1 ("odd") -- READING: the paper
 * names even and odd kernels without fixing their order.  For each site,
 * dE = 2 s_i h_i; the flip is taken when dE <= 0 and otherwise when the site's
 * random word is below the threshold for that dE (Metropolis min(1, e^{-beta dE})).
 * Within one colour no site is a neighbour of another, so the visiting order
 * inside a colour does not matter. */
ORC_API void orc_ising_sweep(int8_t *s, int Lx, int Ly, const uint32_t thr[2], uint64_t seed,
                             uint32_t chain, uint32_t sweep)
{
    for (int c = 0; c < 2; ++c)
        for (int y = 0; y < Ly; ++y)
            for (int x = 0; x < Lx; ++x) {
                if (((x + y) & 1) != c)
                    continue;
                uint32_t r = site_word(seed, chain, sweep, TAG_ISING_METRO, c, colour_index(x, y, Lx));
                int local = s[y * Lx + x] * ising_field(s, Lx, Ly, x, y); /* dE / 2 */
                int flip;
                if (local <= 0)
                    flip = 1;
                else if (local == 2)
                    flip = r < thr[0];
                else /* local == 4 */
                    flip = r < thr[1];
                if (flip)
                    s[y * Lx + x] = (int8_t)(-s[y * Lx + x]);
            }
}

/* Observables of Eq. (1): E = H = -sum over each bond once, M = sum of spins. */
ORC_API void orc_ising_observe(const int8_t *s, int Lx, int Ly, int64_t *E, int64_t *M)
{
    int64_t e = 0, m = 0;
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            int v = s[y * Lx + x];
            e -= (int64_t)v * (s[y * Lx + (x + 1) % Lx] + s[((y + 1) % Ly) * Lx + x]);
            m += v;
        }
    *E = e;
    *M = m;
}

/* n consecutive sweeps numbered first_sweep .. first_sweep + n - 1, recording
 * E and M after every sweep (the "statistics run" of Sec. 2.3) when the series
 * pointers are non-NULL. */
ORC_API void orc_ising_run(int8_t *s, int Lx, int Ly, double beta, uint64_t seed, uint32_t chain,
                           uint32_t first_sweep, int n, int64_t *E_series, int64_t *M_series)
{
    uint32_t thr[2];
    orc_ising_thresholds(beta, thr);
    for (int k = 0; k < n; ++k) {
        orc_ising_sweep(s, Lx, Ly, thr, seed, chain, first_sweep + (uint32_t)k);
        if (E_series && M_series)
            orc_ising_observe(s, Lx, Ly, &E_series[k], &M_series[k]);
    }
}

/* ========================================================================= */
/* 4D SU(2) gauge theory (Sec. 2.4).                                          */
/* Extents L[mu], mu = 0 is time (L_t), mu = 1, 2, 3 are x, y, z (L_1..L_3).   */
/* Site index s = x1 + L1*(x2 + L2*(x3 + L3*x0)); link (s, mu).               */
/* Links enter and leave this file as quaternions q = (U0, U1, U2, U3) of     */
/* Eq. (4), U = U0*I + i*sigma_j*U_j, doubles, array [s][mu][4].              */
/* Inside, each link is a 2x2 complex matrix.                                 */
/* ========================================================================= */

typedef struct {
    double complex m00, m01, m10, m11;
} mat2;

static mat2 mat_from_quat(const double q[4])
{
    /* Eq. (4) with sigma_1 = [[0,1],[1,0]], sigma_2 = [[0,-i],[i,0]],
     * sigma_3 = [[1,0],[0,-1]]. */
    mat2 u;
    u.m00 = q[0] + I * q[3];
    u.m01 = q[2] + I * q[1];
    u.m10 = -q[2] + I * q[1];
    u.m11 = q[0] - I * q[3];
    return u;
}

static void quat_from_mat(mat2 u, double q[4])
{
    q[0] = creal(u.m00);
    q[3] = cimag(u.m00);
    q[2] = creal(u.m01);
    q[1] = cimag(u.m01);
}

static mat2 mat_mul(mat2 a, mat2 b)
{
    mat2 c;
    c.m00 = a.m00 * b.m00 + a.m01 * b.m10;
    c.m01 = a.m00 * b.m01 + a.m01 * b.m11;
    c.m10 = a.m10 * b.m00 + a.m11 * b.m10;
    c.m11 = a.m10 * b.m01 + a.m11 * b.m11;
    return c;
}

static mat2 mat_dag(mat2 a)
{
    mat2 c;
    c.m00 = conj(a.m00);
    c.m01 = conj(a.m10);
    c.m10 = conj(a.m01);
    c.m11 = conj(a.m11);
    return c;
}

static mat2 mat_add(mat2 a, mat2 b)
{
    mat2 c = {a.m00 + b.m00, a.m01 + b.m01, a.m10 + b.m10, a.m11 + b.m11};
    return c;
}

static mat2 mat_scale(mat2 a, double f)
{
    mat2 c = {a.m00 * f, a.m01 * f, a.m10 * f, a.m11 * f};
    return c;
}

static double complex mat_det(mat2 a) { return a.m00 * a.m11 - a.m01 * a.m10; }
static double complex mat_trace(mat2 a) { return a.m00 + a.m11; }

typedef struct {
    int L[4];
    long nsites;
    mat2 *U; /* [s][mu] */
} su2_lattice;

static long site_index(const int L[4], const int x[4])
{
    return (long)x[1] + (long)L[1] * ((long)x[2] + (long)L[2] * ((long)x[3] + (long)L[3] * (long)x[0]));
}

static void site_coords(const int L[4], long s, int x[4])
{
    x[1] = (int)(s % L[1]);
    s /= L[1];
    x[2] = (int)(s % L[2]);
    s /= L[2];
    x[3] = (int)(s % L[3]);
    s /= L[3];
    x[0] = (int)s;
}

/* Neighbour site x + step*e_mu on the hypertorus. */
static long shift(const int L[4], long s, int mu, int step)
{
    int x[4];
    site_coords(L, s, x);
    x[mu] = ((x[mu] + step) % L[mu] + L[mu]) % L[mu];
    return site_index(L, x);
}

static mat2 *link(su2_lattice *lat, long s, int mu) { return &lat->U[s * 4 + mu]; }

static void load_lattice(su2_lattice *lat, const int L[4], const double *q)
{
    memcpy(lat->L, L, sizeof(int) * 4);
    lat->nsites = (long)L[0] * L[1] * L[2] * L[3];
    lat->U = (mat2 *)malloc(sizeof(mat2) * (size_t)lat->nsites * 4);
    for (long k = 0; k < lat->nsites * 4; ++k)
        lat->U[k] = mat_from_quat(&q[4 * k]);
}

static void store_lattice(su2_lattice *lat, double *q)
{
    for (long k = 0; k < lat->nsites * 4; ++k)
        quat_from_mat(lat->U[k], &q[4 * k]);
}

static void free_lattice(su2_lattice *lat) { free(lat->U); }

/* Staple of Eq. (6): the sum, over the six directions nu != mu, of the two
 * paths from x to x + mu that close a plaquette with U_mu(x):
 *   U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu).
 * READING: Eq. (6) prints the sum as "nu (mu < nu)"; with that restriction a
 * link in direction 3 would have no staple, so the sum is taken over nu != mu.
 * The local Boltzmann weight of U_mu(x) is then exp(beta/2 Re Tr(U W^dag)). */
static mat2 staple(su2_lattice *lat, long s, int mu)
{
    mat2 W = {0, 0, 0, 0};
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu)
            continue;
        long s_pnu = shift(lat->L, s, nu, +1);
        long s_pmu = shift(lat->L, s, mu, +1);
        long s_mnu = shift(lat->L, s, nu, -1);
        long s_mnu_pmu = shift(lat->L, s_mnu, mu, +1);
        mat2 up = mat_mul(mat_mul(*link(lat, s, nu), *link(lat, s_pnu, mu)), mat_dag(*link(lat, s_pmu, nu)));
        mat2 down = mat_mul(mat_mul(mat_dag(*link(lat, s_mnu, nu)), *link(lat, s_mnu, mu)), *link(lat, s_mnu_pmu, nu));
        W = mat_add(W, mat_add(up, down));
    }
    return W;
}

#define KP_TRIES 8      /* "8 attempts per start" of the update kernels (Sec. 2.4) */
#define CREUTZ_TRIES 64 /* READING: cap of the fallback sampler; the paper has none */
#define HB_FAILED 255

/* Draw a0 in [-1, 1] with density proportional to sqrt(1 - a0^2) exp(alpha a0)
 * (the heat-bath distribution of the real part of X = U W^dag / k, Eq. (5)).
 *   tries 0..7  : Kennedy & Pendleton, Phys. Lett. B 156 (1985) 393:
 *                 lambda^2 = -(ln u1 + cos^2(2 pi u2) ln u3) / (2 alpha) is a
 *                 Gamma(3/2) variate, accepted with probability sqrt(1 - lambda^2)
 *                 (u4^2 <= 1 - lambda^2); a0 = 1 - 2 lambda^2.
 *   tries 8..71 : Creutz, Phys. Rev. D 21 (1980) 2308: a0 from the inverse CDF
 *                 of exp(alpha a0) on [-1, 1], written with log1p/expm1 so that
 *                 small alpha stays accurate, accepted with probability
 *                 sqrt(1 - a0^2) (u2^2 <= 1 - a0^2).
 * Try t uses the Philox block (c0, c1, c2base | t, c3).  Returns the first
 * accepted try, or HB_FAILED when every try was rejected.  If `forced` >= 0 the
 * draw of try `forced` is returned whatever its test says.  If `margins` is
 * non-NULL every try is evaluated and margins[t] receives the signed distance
 * of try t's acceptance test from its threshold (>= 0 means accepted). */
static int heatbath_a0(double alpha, uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2base, uint32_t c3,
                       int forced, double *a0_out, double *margins)
{
    int chosen = HB_FAILED;
    double a0_chosen = 0.0;
    for (int t = 0; t < KP_TRIES + CREUTZ_TRIES; ++t) {
        uint32_t r[4];
        philox_block(seed, c0, c1, c2base | (uint32_t)t, c3, r);
        double u1 = uniform01(r[0]), u2 = uniform01(r[1]);
        double a0, margin;
        if (t < KP_TRIES) {
            if (alpha > 0.0) {
                double u3 = uniform01(r[2]), u4 = uniform01(r[3]);
                double cs = cos(2.0 * M_PI * u2);
                double lam2 = -(log(u1) + cs * cs * log(u3)) / (2.0 * alpha);
                a0 = 1.0 - 2.0 * lam2;
                margin = (1.0 - lam2) - u4 * u4;
            } else {
                a0 = 0.0;
                margin = -1.0; /* the Gamma variate is undefined at alpha = 0: reject */
            }
        } else {
            if (alpha > 0.0) {
                double c = -expm1(-2.0 * alpha); /* 1 - e^{-2 alpha} */
                a0 = 1.0 + log1p(-(1.0 - u1) * c) / alpha;
            } else {
                a0 = 2.0 * u1 - 1.0; /* alpha = 0: the factor exp(alpha a0) is flat */
            }
            margin = (1.0 - a0 * a0) - u2 * u2;
        }
        if (margins)
            margins[t] = margin;
        if (chosen == HB_FAILED && (forced >= 0 ? t == forced : margin >= 0.0)) {
            chosen = t;
            a0_chosen = a0;
            if (!margins)
                break;
        }
    }
    *a0_out = a0_chosen;
    return chosen;
}

/* Uniform direction on the 2-sphere from the Philox block (c0, c1, c2, c3):
 * cos(theta) = 2 u1 - 1, phi = 2 pi u2. */
static void sphere_direction(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double n[3])
{
    uint32_t r[4];
    philox_block(seed, c0, c1, c2, c3, r);
    double ct = 2.0 * uniform01(r[0]) - 1.0;
    double phi = 2.0 * M_PI * uniform01(r[1]);
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    n[0] = st * cos(phi);
    n[1] = st * sin(phi);
    n[2] = ct;
}

#define NOT_FORCED (-1)

/* Heat-bath replacement of one link, Eqs. (5)-(7).  With W the staple of
 * Eq. (6), k = sqrt(det W) and V = W / k in SU(2), the new link is
 * U = X V with X = a0 I + i sqrt(1 - a0^2) n.sigma, a0 from heatbath_a0 at
 * alpha = beta k and n uniform on S^2: then Re Tr(U W^dag) / 2 = k a0, so X is
 * drawn from exp(beta/2 Re Tr(U W^dag)) times Haar measure.  READING of Eq. (5)
 * "U -> w W with w normalising": w = X / k.  The result is projected back onto
 * SU(2) (U / sqrt(det U)) after the update.  When every try is rejected the
 * link is left as it is; that stays exact because the failure probability
 * depends on alpha only, not on the link.
 * `forced` (NOT_FORCED, a try index or HB_FAILED) makes the update follow the
 * decision of another run; each try on which this FP64 run decides otherwise
 * is then classified as near its threshold (|margin| < eps, counted in *near)
 * or not (counted in *bad).  Returns the try whose draw was taken. */
static int heatbath_link(su2_lattice *lat, long s, int mu, int parity, double beta, uint64_t seed,
                         uint32_t chain, uint32_t sweep, int forced, double eps, long *near, long *bad)
{
    mat2 W = staple(lat, s, mu);
    double k = sqrt(fmax(0.0, creal(mat_det(W))));
    mat2 V;
    if (k > 0.0)
        V = mat_scale(W, 1.0 / k);
    else {
        mat2 one = {1, 0, 0, 1};
        V = one;
    }
    double alpha = beta * k;
    uint32_t eo = (uint32_t)(s >> 1); /* index of the site within its parity class */
    uint32_t sel = ((uint32_t)parity << 12) | ((uint32_t)mu << 8);
    double a0;
    int t;
    if (forced == NOT_FORCED) {
        t = heatbath_a0(alpha, seed, eo, sweep, TAG_SU2_HB | sel, chain, -1, &a0, NULL);
    } else {
        double margins[KP_TRIES + CREUTZ_TRIES];
        int own = heatbath_a0(alpha, seed, eo, sweep, TAG_SU2_HB | sel, chain, -1, &a0, margins);
        if (own != forced) {
            /* the other run rejected every try before `forced` and accepted it */
            int ok = 1;
            int last = forced == HB_FAILED ? KP_TRIES + CREUTZ_TRIES - 1 : forced;
            for (int u = 0; u <= last; ++u) {
                int other_accepts = (u == forced);
                int mine_accepts = margins[u] >= 0.0;
                if (other_accepts != mine_accepts && fabs(margins[u]) >= eps)
                    ok = 0;
            }
            if (ok)
                ++*near;
            else
                ++*bad;
        }
        t = forced;
        if (t != HB_FAILED)
            heatbath_a0(alpha, seed, eo, sweep, TAG_SU2_HB | sel, chain, forced, &a0, NULL);
    }
    if (t == HB_FAILED)
        return t;
    double n[3];
    sphere_direction(seed, eo, sweep, TAG_SU2_DIR | sel, chain, n);
    double r = sqrt(fmax(0.0, 1.0 - a0 * a0));
    double xq[4] = {a0, r * n[0], r * n[1], r * n[2]};
    mat2 X = mat_from_quat(xq);
    mat2 U = mat_mul(X, V);
    double complex d = mat_det(U);
    *link(lat, s, mu) = mat_scale(U, 1.0 / sqrt(creal(d)));
    return t;
}

static int site_parity(const int L[4], long s)
{
    int x[4];
    site_coords(L, s, x);
    return (x[0] + x[1] + x[2] + x[3]) & 1;
}

/* Size of the per-sweep try record: one byte per link, [s][mu]. */
ORC_API long orc_su2_nlinks(const int L[4]) { return 4L * L[0] * L[1] * L[2] * L[3]; }

/* Lattice initialisation (Sec. 2.4): cold = identity links; hot = Haar-random
 * links, the normalised 4-vector of four Box-Muller normals from one Philox
 * block per link (counter (s, 0, tag INIT | mu, chain)). */
ORC_API void orc_su2_init(double *q, const int L[4], uint64_t seed, uint32_t chain, int hot)
{
    long ns = (long)L[0] * L[1] * L[2] * L[3];
    for (long s = 0; s < ns; ++s)
        for (int mu = 0; mu < 4; ++mu) {
            double *v = &q[(s * 4 + mu) * 4];
            if (!hot) {
                v[0] = 1.0;
                v[1] = v[2] = v[3] = 0.0;
                continue;
            }
            uint32_t r[4];
            philox_block(seed, (uint32_t)s, 0u, TAG_SU2_INIT | (uint32_t)mu, chain, r);
            double u1 = uniform01(r[0]), u2 = uniform01(r[1]), u3 = uniform01(r[2]), u4 = uniform01(r[3]);
            double ra = sqrt(-2.0 * log(u1)), rb = sqrt(-2.0 * log(u3));
            double g[4] = {ra * cos(2.0 * M_PI * u2), ra * sin(2.0 * M_PI * u2), rb * cos(2.0 * M_PI * u4),
                           rb * sin(2.0 * M_PI * u4)};
            double nrm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2] + g[3] * g[3]);
            for (int c = 0; c < 4; ++c)
                v[c] = g[c] / nrm;
        }
}

/* One heat-bath sweep number `sweep` in the order of Sec. 2.4: for each
 * direction mu = 0..3 the odd sites (parity 1), then for each mu the even sites
 * (parity 0).  Within one (parity, mu) phase no updated link enters another
 * updated link's staple, so the order inside a phase does not matter.
 *   tries_out     : optional [s][mu] bytes, accepted try per link (255 = none).
 *   forced_tries  : optional [s][mu] bytes; where given, the update takes that
 *                   try's draw -- but only after checking that every decision
 *                   this FP64 run would take differently lies within `eps` of
 *                   its threshold.  Such links are counted in *n_near; any
 *                   other disagreement is counted in *n_bad.
 * Returns the number of links whose update found no accepted try. */
ORC_API long orc_su2_sweep(double *q, const int L[4], double beta, uint64_t seed, uint32_t chain, uint32_t sweep,
                           uint8_t *tries_out, const uint8_t *forced_tries, double eps, long *n_near,
                           long *n_bad)
{
    su2_lattice lat;
    load_lattice(&lat, L, q);
    long failures = 0, near = 0, bad = 0;
    const int parity_order[2] = {1, 0}; /* odd sites first */
    for (int pi = 0; pi < 2; ++pi) {
        int p = parity_order[pi];
        for (int mu = 0; mu < 4; ++mu)
            for (long s = 0; s < lat.nsites; ++s) {
                if (site_parity(L, s) != p)
                    continue;
                int forced = forced_tries ? (int)forced_tries[s * 4 + mu] : NOT_FORCED;
                int t = heatbath_link(&lat, s, mu, p, beta, seed, chain, sweep, forced, eps, &near, &bad);
                if (t == HB_FAILED)
                    ++failures;
                if (tries_out)
                    tries_out[s * 4 + mu] = (uint8_t)t;
            }
    }
    store_lattice(&lat, q);
    free_lattice(&lat);
    if (n_near)
        *n_near = near;
    if (n_bad)
        *n_bad = bad;
    return failures;
}

/* Overrelaxation, the second half of the "heat-bath algorithm with
 * overrelaxation" of Sec. 2.4 (the method of Creutz, Phys. Rev. D 36 (1987)
 * 515): the link is replaced by its reflection within the SU(2) matrices of
 * equal local action,
 *   U' = V U^dag V,  V = W / sqrt(det W),
 * so that Re Tr(U' W^dag) = k Re Tr(V U^dag) = Re Tr(U W^dag): the move is
 * microcanonical, needs no random number and is its own inverse (X = U V^dag
 * goes to X^dag).  A link whose staple vanishes is left unchanged.  The link is
 * reprojected (U / sqrt(det U)) like a heat-bath update.
 * READING: the paper names the combination but not the number of reflections
 * per heat-bath step; here a compound sweep is one heat-bath sweep followed by
 * n_or overrelaxation sweeps (a run-time parameter, like the paper's "number of
 * link updates per one MC sweep"), each in the heat-bath's phase order. */
static void overrelax_link(su2_lattice *lat, long s, int mu)
{
    mat2 W = staple(lat, s, mu);
    double k = sqrt(fmax(0.0, creal(mat_det(W))));
    if (!(k > 0.0))
        return;
    mat2 V = mat_scale(W, 1.0 / k);
    mat2 U = mat_mul(mat_mul(V, mat_dag(*link(lat, s, mu))), V);
    *link(lat, s, mu) = mat_scale(U, 1.0 / sqrt(creal(mat_det(U))));
}

/* One overrelaxation sweep in the phase order of orc_su2_sweep. */
ORC_API void orc_su2_overrelax(double *q, const int L[4])
{
    su2_lattice lat;
    load_lattice(&lat, L, q);
    const int parity_order[2] = {1, 0};
    for (int pi = 0; pi < 2; ++pi)
        for (int mu = 0; mu < 4; ++mu)
            for (long s = 0; s < lat.nsites; ++s)
                if (site_parity(L, s) == parity_order[pi])
                    overrelax_link(&lat, s, mu);
    store_lattice(&lat, q);
    free_lattice(&lat);
}

/* Plaquette averages of Eqs. (2)-(3): (1/2) Tr U_munu(x) with
 * U_munu(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag, averaged over all
 * 6 N plaquettes (out[0]), the 3 N spatial ones, mu, nu in {1,2,3} (out[1]) and
 * the 3 N temporal ones with mu = 0 (out[2]) -- the two double-precision
 * averages each measuring thread of Sec. 2.4 produces. */
ORC_API void orc_su2_plaquette(const double *q, const int L[4], double out[3])
{
    su2_lattice lat;
    load_lattice(&lat, L, q);
    double sum_s = 0.0, sum_t = 0.0;
    for (long s = 0; s < lat.nsites; ++s)
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                long s_pmu = shift(L, s, mu, +1), s_pnu = shift(L, s, nu, +1);
                mat2 P = mat_mul(mat_mul(*link(&lat, s, mu), *link(&lat, s_pmu, nu)),
                                 mat_mul(mat_dag(*link(&lat, s_pnu, mu)), mat_dag(*link(&lat, s, nu))));
                double h = 0.5 * creal(mat_trace(P));
                if (mu == 0)
                    sum_t += h;
                else
                    sum_s += h;
            }
    out[0] = (sum_s + sum_t) / (6.0 * (double)lat.nsites);
    out[1] = sum_s / (3.0 * (double)lat.nsites);
    out[2] = sum_t / (3.0 * (double)lat.nsites);
    free_lattice(&lat);
}

/* Polyakov loop (an observable the paper does not measure; it pairs with the
 * finite-temperature lattices L_t x L_s^3 of Sec. 2.4): for every spatial site
 * x, (1/2) Tr of the ordered product U_0(0, x) U_0(1, x) ... U_0(L_0 - 1, x) of
 * the time-direction links, averaged over the L_1 L_2 L_3 spatial sites.
 * Gauge invariant; changes sign under the centre transformation that flips
 * every U_0 on one time slice. */
ORC_API double orc_su2_polyakov(const double *q, const int L[4])
{
    su2_lattice lat;
    load_lattice(&lat, L, q);
    long nspace = (long)L[1] * L[2] * L[3];
    double sum = 0.0;
    for (long xs = 0; xs < nspace; ++xs) {
        /* canonical index s = x1 + L1 (x2 + L2 (x3 + L3 x0)): the spatial part is xs, time adds x0 * nspace */
        mat2 P = {1, 0, 0, 1};
        for (int t = 0; t < L[0]; ++t)
            P = mat_mul(P, *link(&lat, xs + (long)t * nspace, 0));
        sum += 0.5 * creal(mat_trace(P));
    }
    free_lattice(&lat);
    return sum / (double)nspace;
}

/* Wilson action of Eq. (2), S = beta sum_x sum_{mu<nu} [1 - (1/2) Tr U_munu]. */
ORC_API double orc_su2_action(const double *q, const int L[4], double beta)
{
    double P[3];
    orc_su2_plaquette(q, L, P);
    double ns = (double)L[0] * L[1] * L[2] * L[3];
    return beta * 6.0 * ns * (1.0 - P[0]);
}

/* The staple W of Eq. (6) for link (s, mu), returned as the quaternion of the
 * 2x2 matrix W (a sum of SU(2) matrices is a real multiple of one). */
ORC_API void orc_su2_staple(const double *q, const int L[4], long s, int mu, double out[4])
{
    su2_lattice lat;
    load_lattice(&lat, L, q);
    quat_from_mat(staple(&lat, s, mu), out);
    free_lattice(&lat);
}

/* n draws of the heat-bath a0 sampler at fixed alpha, draw i using counters
 * (i, 0, TAG_SU2_HB | t, 0xFFFFFFFF); tries[i] receives the accepted try. */
ORC_API void orc_su2_sample_a0(double alpha, uint64_t seed, long n, double *out, uint8_t *tries)
{
    for (long i = 0; i < n; ++i) {
        double a0;
        int t = heatbath_a0(alpha, seed, (uint32_t)i, 0u, TAG_SU2_HB, 0xFFFFFFFFu, -1, &a0, NULL);
        out[i] = a0;
        if (tries)
            tries[i] = (uint8_t)t;
    }
}

/* Quaternion of the product of the two SU(2) matrices of quaternions a and b,
 * computed through the 2x2 complex representation of Eq. (4). */
ORC_API void orc_su2_mul(const double a[4], const double b[4], double out[4])
{
    quat_from_mat(mat_mul(mat_from_quat(a), mat_from_quat(b)), out);
}

/* ========================================================================= */
/* Sampled checks of one sweep at any lattice size.                           */
/* ========================================================================= */

/* Expected post-sweep spin of each listed site (index y*Lx + x), given the
 * configurations before (pre) and after (post) sweep number `sweep`: colour-0
 * sites are updated against the pre-sweep colour-1 spins, colour-1 sites
 * against the post-sweep colour-0 spins (Sec. 2.3 checkerboard order). */
ORC_API void orc_ising_check_sites(const int8_t *pre, const int8_t *post, int Lx, int Ly, double beta,
                                   uint64_t seed, uint32_t chain, uint32_t sweep, const int64_t *sites, long n,
                                   int8_t *out)
{
    uint32_t thr[2];
    orc_ising_thresholds(beta, thr);
    for (long k = 0; k < n; ++k) {
        int x = (int)(sites[k] % Lx), y = (int)(sites[k] / Lx);
        int c = (x + y) & 1;
        const int8_t *nb = c == 0 ? pre : post;
        int xp = (x + 1) % Lx, xm = (x + Lx - 1) % Lx, yp = (y + 1) % Ly, ym = (y + Ly - 1) % Ly;
        int h = nb[y * Lx + xp] + nb[y * Lx + xm] + nb[yp * Lx + x] + nb[ym * Lx + x];
        int v = pre[y * Lx + x];
        int local = v * h;
        uint32_t r = site_word(seed, chain, sweep, TAG_ISING_METRO, c, colour_index(x, y, Lx));
        int flip = local <= 0 || (local == 2 ? r < thr[0] : r < thr[1]);
        out[k] = (int8_t)(flip ? -v : v);
    }
}

/* Position of phase (parity p, direction mu) in the sweep: odd sites first. */
static int phase_index(int p, int mu) { return (p == 1 ? 0 : 4) + mu; }

/* Expected post-sweep value of each listed link (index 4 s + mu), given the
 * quaternion configurations before and after sweep number `sweep`: for a link
 * of phase k, every link of an earlier phase holds its post-sweep value and
 * every other link its pre-sweep value, which is exactly the lattice the
 * update saw.  forced_tries (per listed link, or NULL) as in orc_su2_sweep.
 * Returns the number of listed links whose every try was rejected. */
ORC_API long orc_su2_check_links(const double *pre, const double *post, const int L[4], double beta, uint64_t seed,
                                 uint32_t chain, uint32_t sweep, const int64_t *links, long n,
                                 const uint8_t *forced_tries, double eps, double *out, long *n_near, long *n_bad)
{
    su2_lattice lat;
    load_lattice(&lat, L, pre);
    long failures = 0, near = 0, bad = 0;
    for (int ph = 0; ph < 8; ++ph) {
        int p = ph < 4 ? 1 : 0, mu = ph & 3;
        /* lattice as seen by phase ph */
        for (long s = 0; s < lat.nsites; ++s)
            for (int nu = 0; nu < 4; ++nu) {
                const double *src = phase_index(site_parity(L, s), nu) < ph ? post : pre;
                lat.U[s * 4 + nu] = mat_from_quat(&src[(s * 4 + nu) * 4]);
            }
        for (long k = 0; k < n; ++k) {
            long s = (long)(links[k] >> 2);
            int m = (int)(links[k] & 3);
            if (m != mu || site_parity(L, s) != p)
                continue;
            int forced = forced_tries ? (int)forced_tries[k] : NOT_FORCED;
            int t = heatbath_link(&lat, s, mu, p, beta, seed, chain, sweep, forced, eps, &near, &bad);
            if (t == HB_FAILED)
                ++failures;
            quat_from_mat(*link(&lat, s, mu), &out[k * 4]);
        }
    }
    free_lattice(&lat);
    if (n_near)
        *n_near = near;
    if (n_bad)
        *n_bad = bad;
    return failures;
}
