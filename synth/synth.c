/*
 * Seeded synthetic inputs for the Wilson-Dirac multigrid solver.
 *
 * This file holds NO arithmetic of the multigrid method itself.  It makes the
 * inputs that both the CPU oracle and the CUDA path consume:
 *   - Philox4x32-10 counter-based random numbers (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11);
 *   - Gaussian complex fields (Marsaglia polar method);
 *   - SU(3) gauge links from a quenched Wilson-gauge Monte Carlo: hot start,
 *     Cabibbo-Marinari updates over the SU(2) subgroups (0,1), (1,2), (0,2),
 *     Kennedy-Pendleton SU(2) heatbath (Phys. Lett. B156 (1985) 393) and
 *     SU(2) over-relaxation, checkerboarded by parity per direction;
 *   - random SU(3) gauge transformations and point sources.
 *
 * Bitwise reproducibility across x86-64 and aarch64: the file is compiled with
 * -ffp-contract=off (no fused multiply-add), uses only +, -, *, /, sqrt and
 * frexp/ldexp (all exact or correctly rounded in IEEE-754), and computes
 * logarithms with its own series (synth_log) instead of libm.  Every random
 * draw is addressed by a counter, so results do not depend on thread count.
 *
 * Layouts (shared with the C-ABI boundary):
 *   site index  = x + L0*(y + L1*(z + L2*t))
 *   links       U[mu][site][a][b], complex double as (re, im) pairs
 *   spinor      psi[site][spin 4][colour 3], complex double
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYNTH_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                       */
/* ------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static inline void philox_round(uint32_t c[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

SYNTH_API void synth_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        philox_round(c, k);
        if (r < 9) { k[0] += PHILOX_W0; k[1] += PHILOX_W1; }
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* A stream of uniforms addressed by (seed, a, b, c); d counts draws. */
typedef struct {
    uint32_t key[2];
    uint32_t ctr[4];
    uint32_t buf[4];
    int left;
} rng_t;

static void rng_init(rng_t* g, uint64_t seed, uint32_t a, uint32_t b, uint32_t c) {
    g->key[0] = (uint32_t)seed; g->key[1] = (uint32_t)(seed >> 32);
    g->ctr[0] = a; g->ctr[1] = b; g->ctr[2] = c; g->ctr[3] = 0;
    g->left = 0;
}

/* uniform double in the open interval (0,1), 53 random bits */
static double rng_uniform(rng_t* g) {
    if (g->left == 0) {
        synth_philox4x32_10(g->ctr, g->key, g->buf);
        g->ctr[3] += 1;
        g->left = 2;
    }
    int i = (2 - g->left) * 2;
    g->left -= 1;
    uint64_t u = (((uint64_t)g->buf[i] << 32) | g->buf[i + 1]) >> 11;
    return ((double)u + 0.5) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------ */
/* logarithm from + - * / only: x = m 2^e, m in [1/sqrt2, sqrt2),     */
/* ln m = 2 atanh(z), z = (m-1)/(m+1), |z| <= 0.1716, series in z^2.   */
/* ------------------------------------------------------------------ */
SYNTH_API double synth_log(double x) {
    int e;
    double m = frexp(x, &e);
    if (m < 0.70710678118654752440) { m = m * 2.0; e -= 1; }
    double z = (m - 1.0) / (m + 1.0);
    double z2 = z * z;
    double term = z, sum = 0.0;
    for (int k = 0; k < 14; ++k) {
        sum = sum + term / (double)(2 * k + 1);
        term = term * z2;
    }
    return 2.0 * sum + (double)e * 0.69314718055994530942;
}

/* standard normal pair by the Marsaglia polar method */
static void rng_normal2(rng_t* g, double* n0, double* n1) {
    for (;;) {
        double u = 2.0 * rng_uniform(g) - 1.0;
        double v = 2.0 * rng_uniform(g) - 1.0;
        double s = u * u + v * v;
        if (s >= 1.0 || s == 0.0) continue;
        double f = sqrt(-2.0 * synth_log(s) / s);
        *n0 = u * f; *n1 = v * f;
        return;
    }
}

/* ------------------------------------------------------------------ */
/* Gaussian complex fields: each real component ~ N(0,1)               */
/* stream tag: field draws use ctr = (index, stream, tag)               */
/* ------------------------------------------------------------------ */
SYNTH_API void synth_gaussian(double* out, int64_t n_complex, uint64_t seed, uint32_t stream) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_complex; ++i) {
        rng_t g;
        rng_init(&g, seed, (uint32_t)i, (uint32_t)(i >> 32) ^ 0x5A5A0000u, stream);
        double a, b;
        rng_normal2(&g, &a, &b);
        out[2 * i] = a; out[2 * i + 1] = b;
    }
}

/* ------------------------------------------------------------------ */
/* 3x3 complex helpers (row-major, interleaved re/im)                 */
/* ------------------------------------------------------------------ */
typedef struct { double re, im; } cplx;
typedef struct { cplx e[3][3]; } su3;

static inline cplx cmul(cplx a, cplx b) { cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static inline cplx cmulc(cplx a, cplx b) { /* a * conj(b) */ cplx r = {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im}; return r; }
static inline cplx cadd(cplx a, cplx b) { cplx r = {a.re + b.re, a.im + b.im}; return r; }
static inline cplx cconj(cplx a) { cplx r = {a.re, -a.im}; return r; }

static void su3_mul(su3* r, const su3* a, const su3* b) {        /* r = a b   */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx s = cmul(a->e[i][0], b->e[0][j]);
            s = cadd(s, cmul(a->e[i][1], b->e[1][j]));
            s = cadd(s, cmul(a->e[i][2], b->e[2][j]));
            r->e[i][j] = s;
        }
}
static void su3_mul_nd(su3* r, const su3* a, const su3* b) {     /* r = a b^dag */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx s = cmulc(a->e[i][0], b->e[j][0]);
            s = cadd(s, cmulc(a->e[i][1], b->e[j][1]));
            s = cadd(s, cmulc(a->e[i][2], b->e[j][2]));
            r->e[i][j] = s;
        }
}
static void su3_mul_dn(su3* r, const su3* a, const su3* b) {     /* r = a^dag b */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx s = cmul(cconj(a->e[0][i]), b->e[0][j]);
            s = cadd(s, cmul(cconj(a->e[1][i]), b->e[1][j]));
            s = cadd(s, cmul(cconj(a->e[2][i]), b->e[2][j]));
            r->e[i][j] = s;
        }
}
static void su3_acc(su3* r, const su3* a) {
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) r->e[i][j] = cadd(r->e[i][j], a->e[i][j]);
}

/* Gram-Schmidt rows 0,1; row 2 = conj(row0 x row1): the nearest-in-form SU(3) */
static void su3_reunitarize(su3* u) {
    double n = 0;
    for (int j = 0; j < 3; ++j) n += u->e[0][j].re * u->e[0][j].re + u->e[0][j].im * u->e[0][j].im;
    n = 1.0 / sqrt(n);
    for (int j = 0; j < 3; ++j) { u->e[0][j].re *= n; u->e[0][j].im *= n; }
    cplx d = {0, 0};                                   /* d = <row0, row1> */
    for (int j = 0; j < 3; ++j) d = cadd(d, cmul(cconj(u->e[0][j]), u->e[1][j]));
    for (int j = 0; j < 3; ++j) {
        cplx t = cmul(d, u->e[0][j]);
        u->e[1][j].re -= t.re; u->e[1][j].im -= t.im;
    }
    n = 0;
    for (int j = 0; j < 3; ++j) n += u->e[1][j].re * u->e[1][j].re + u->e[1][j].im * u->e[1][j].im;
    n = 1.0 / sqrt(n);
    for (int j = 0; j < 3; ++j) { u->e[1][j].re *= n; u->e[1][j].im *= n; }
    for (int j = 0; j < 3; ++j) {
        int a = (j + 1) % 3, b = (j + 2) % 3;
        cplx c = cmul(u->e[0][a], u->e[1][b]);
        cplx e = cmul(u->e[0][b], u->e[1][a]);
        cplx x = {c.re - e.re, c.im - e.im};
        u->e[2][j] = cconj(x);
    }
}

static void su3_random(su3* u, rng_t* g) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) rng_normal2(g, &u->e[i][j].re, &u->e[i][j].im);
    su3_reunitarize(u);
}

/* ------------------------------------------------------------------ */
/* lattice geometry                                                   */
/* ------------------------------------------------------------------ */
typedef struct { int L[4]; int64_t V; } geom_t;

static void geom_init(geom_t* g, const int* L) {
    for (int m = 0; m < 4; ++m) g->L[m] = L[m];
    g->V = (int64_t)L[0] * L[1] * L[2] * L[3];
}
static inline void geom_coords(const geom_t* g, int64_t s, int c[4]) {
    for (int m = 0; m < 4; ++m) { c[m] = (int)(s % g->L[m]); s /= g->L[m]; }
}
static inline int64_t geom_index(const geom_t* g, const int c[4]) {
    return c[0] + (int64_t)g->L[0] * (c[1] + (int64_t)g->L[1] * (c[2] + (int64_t)g->L[2] * c[3]));
}
static inline int64_t geom_shift(const geom_t* g, int64_t s, int mu, int dir) {
    int c[4];
    geom_coords(g, s, c);
    c[mu] = (c[mu] + dir + g->L[mu]) % g->L[mu];
    return geom_index(g, c);
}

static inline su3* link(double* U, const geom_t* g, int mu, int64_t s) {
    return (su3*)(U + 18 * (mu * g->V + s));
}

/* Staple sum A so that the local Wilson action is -(beta/3) Re tr(U_mu(x) A). */
static void staple(su3* A, double* U, const geom_t* g, int mu, int64_t s) {
    memset(A, 0, sizeof(*A));
    int64_t sp = geom_shift(g, s, mu, +1);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        su3 t1, t2;
        /* upper: U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag */
        int64_t sn = geom_shift(g, s, nu, +1);
        su3_mul_nd(&t1, link(U, g, nu, sp), link(U, g, mu, sn));
        su3_mul_nd(&t2, &t1, link(U, g, nu, s));
        su3_acc(A, &t2);
        /* lower: U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) = (U_mu(x-nu) U_nu(x+mu-nu))^dag U_nu(x-nu) */
        int64_t sm = geom_shift(g, s, nu, -1);
        int64_t spm = geom_shift(g, sp, nu, -1);
        su3 t3;
        su3_mul(&t1, link(U, g, mu, sm), link(U, g, nu, spm));
        su3_mul_dn(&t3, &t1, link(U, g, nu, sm));
        su3_acc(A, &t3);
    }
}

/* 2x2 complex matrix as quaternion helpers for the SU(2) subgroup update */
typedef struct { cplx e[2][2]; } su2m;

static void su2_mul(su2m* r, const su2m* a, const su2m* b) {
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            r->e[i][j] = cadd(cmul(a->e[i][0], b->e[0][j]), cmul(a->e[i][1], b->e[1][j]));
}
static void su2_from_q(su2m* r, const double q[4]) {
    /* q0 + i(q1 s1 + q2 s2 + q3 s3) */
    r->e[0][0].re = q[0]; r->e[0][0].im = q[3];
    r->e[0][1].re = q[2]; r->e[0][1].im = q[1];
    r->e[1][0].re = -q[2]; r->e[1][0].im = q[1];
    r->e[1][1].re = q[0]; r->e[1][1].im = -q[3];
}
static void su2_dag(su2m* r, const su2m* a) {
    for (int i = 0; i < 2; ++i) for (int j = 0; j < 2; ++j) r->e[i][j] = cconj(a->e[j][i]);
}

/* Kennedy-Pendleton draw of x0 with density ~ sqrt(1-x0^2) exp(alpha x0),
 * then a uniform direction for (x1,x2,x3) on the sphere of radius sqrt(1-x0^2).
 * The cos^2(2 pi r) factor is drawn as u^2/(u^2+v^2) for (u,v) uniform in the
 * unit disc, and the direction by Marsaglia's disc method, so only sqrt and
 * synth_log are needed. */
static void kp_draw(double x[4], double alpha, rng_t* g) {
    double lam2;
    for (int trial = 0; trial < 100000; ++trial) {
        double r1 = rng_uniform(g), r3 = rng_uniform(g);
        double u, v, s;
        do { u = 2.0 * rng_uniform(g) - 1.0; v = 2.0 * rng_uniform(g) - 1.0; s = u * u + v * v; } while (s >= 1.0 || s == 0.0);
        double c2 = (u * u) / s;
        lam2 = -(synth_log(r1) + c2 * synth_log(r3)) / (2.0 * alpha);
        double r4 = rng_uniform(g);
        if (r4 * r4 <= 1.0 - lam2) break;
    }
    x[0] = 1.0 - 2.0 * lam2;
    double rad = 1.0 - x[0] * x[0];
    rad = rad > 0 ? sqrt(rad) : 0.0;
    double u, v, s;
    do { u = 2.0 * rng_uniform(g) - 1.0; v = 2.0 * rng_uniform(g) - 1.0; s = u * u + v * v; } while (s >= 1.0 || s == 0.0);
    double f = 2.0 * sqrt(1.0 - s);
    x[1] = rad * u * f; x[2] = rad * v * f; x[3] = rad * (1.0 - 2.0 * s);
}

static const int SUBGROUP[3][2] = {{0, 1}, {1, 2}, {0, 2}};

/* One Cabibbo-Marinari update of link U (heatbath if hb, else over-relaxation). */
static void update_link(su3* U, const su3* A, double beta, int hb, rng_t* g) {
    for (int sg = 0; sg < 3; ++sg) {
        int i = SUBGROUP[sg][0], j = SUBGROUP[sg][1];
        su3 W;
        su3_mul(&W, U, A);
        cplx w00 = W.e[i][i], w01 = W.e[i][j], w10 = W.e[j][i], w11 = W.e[j][j];
        double q[4];
        q[0] = 0.5 * (w00.re + w11.re);
        q[1] = 0.5 * (w01.im + w10.im);
        q[2] = 0.5 * (w01.re - w10.re);
        q[3] = 0.5 * (w00.im - w11.im);
        double k = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        if (!(k > 1e-14)) continue;
        for (int a = 0; a < 4; ++a) q[a] /= k;
        su2m v, vd, r;
        su2_from_q(&v, q);
        su2_dag(&vd, &v);
        if (hb) {
            double x[4];
            kp_draw(x, 2.0 * beta * k / 3.0, g);
            su2m xm;
            su2_from_q(&xm, x);
            su2_mul(&r, &xm, &vd);
        } else {
            su2_mul(&r, &vd, &vd);
        }
        /* U <- R U, R = embedding of r in rows/cols (i,j) */
        for (int c = 0; c < 3; ++c) {
            cplx ui = U->e[i][c], uj = U->e[j][c];
            U->e[i][c] = cadd(cmul(r.e[0][0], ui), cmul(r.e[0][1], uj));
            U->e[j][c] = cadd(cmul(r.e[1][0], ui), cmul(r.e[1][1], uj));
        }
    }
}

/* ------------------------------------------------------------------ */
/* public gauge API                                                   */
/* ------------------------------------------------------------------ */
SYNTH_API void synth_gauge_hot(double* U, const int* L, uint64_t seed) {
    geom_t g; geom_init(&g, L);
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < g.V; ++s)
        for (int mu = 0; mu < 4; ++mu) {
            rng_t r; rng_init(&r, seed, (uint32_t)s, (uint32_t)mu | 0x10000000u, 0xFFFFFFFFu);
            su3_random(link(U, &g, mu, s), &r);
        }
}

SYNTH_API void synth_gauge_unit(double* U, const int* L) {
    geom_t g; geom_init(&g, L);
    memset(U, 0, sizeof(double) * 18 * 4 * g.V);
    for (int64_t s = 0; s < 4 * g.V; ++s)
        for (int a = 0; a < 3; ++a) U[18 * s + 2 * (3 * a + a)] = 1.0;
}

/* One compound sweep number `sweep`: 1 heatbath + n_or over-relaxation passes,
 * each pass over (parity, mu) checkerboards, then reunitarisation. */
SYNTH_API void synth_gauge_sweep(double* U, const int* L, double beta, int n_or, uint64_t seed, int sweep) {
    geom_t g; geom_init(&g, L);
    for (int pass = 0; pass <= n_or; ++pass) {
        int hb = (pass == 0);
        for (int par = 0; par < 2; ++par)
            for (int mu = 0; mu < 4; ++mu) {
#pragma omp parallel for schedule(static)
                for (int64_t s = 0; s < g.V; ++s) {
                    int c[4]; geom_coords(&g, s, c);
                    if (((c[0] + c[1] + c[2] + c[3]) & 1) != par) continue;
                    su3 A; staple(&A, U, &g, mu, s);
                    rng_t r;
                    rng_init(&r, seed, (uint32_t)s, (uint32_t)mu | ((uint32_t)pass << 4), (uint32_t)sweep);
                    update_link(link(U, &g, mu, s), &A, beta, hb, &r);
                }
            }
    }
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < 4 * g.V; ++s) su3_reunitarize((su3*)(U + 18 * s));
}

/* average plaquette (1/3) Re tr U_p over all 6 V plaquettes, fixed summation order */
SYNTH_API double synth_plaquette(const double* Uc, const int* L) {
    geom_t g; geom_init(&g, L);
    double* U = (double*)Uc;
    double total = 0.0;
    for (int64_t s = 0; s < g.V; ++s)
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                su3 t1, t2, t3;
                int64_t smu = geom_shift(&g, s, mu, +1), snu = geom_shift(&g, s, nu, +1);
                su3_mul(&t1, link(U, &g, mu, s), link(U, &g, nu, smu));
                su3_mul_nd(&t2, &t1, link(U, &g, mu, snu));
                su3_mul_nd(&t3, &t2, link(U, &g, nu, s));
                total += (t3.e[0][0].re + t3.e[1][1].re + t3.e[2][2].re) / 3.0;
            }
    return total / (6.0 * (double)g.V);
}

/* Random SU(3) gauge transformation Omega[site][3][3]. */
SYNTH_API void synth_random_su3_field(double* Om, int64_t n, uint64_t seed) {
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n; ++s) {
        rng_t r; rng_init(&r, seed, (uint32_t)s, 0x20000000u, 0xEEEEEEEEu);
        su3_random((su3*)(Om + 18 * s), &r);
    }
}
