/*
 * CPU oracle for the adaptive multigrid Wilson-Dirac solver of Babich et al.,
 * "Adaptive multigrid algorithm for the lattice Wilson-Dirac operator"
 * (arXiv:1005.3043).  TEST INFRASTRUCTURE ONLY: it is called by tests/, by the
 * package's smoke check and by the benchmark's CPU-baseline leg, never by the
 * product path.  Plain, slow, FP64 (complex double), written from the paper:
 * every function names the passage it restates.  It shares no code with the
 * CUDA library.
 *
 * Conventions (the paper is silent on them; the readings are listed with the
 * design notes):
 *  - site = x + L0*(y + L1*(z + L2*t)); mu = 0..3 is x, y, z, t.
 *  - spinor psi[site][spin 4][colour 3]; links U[mu][site][a][b].
 *  - gamma matrices in the DeGrand-Rossi (chiral) basis, gamma5 = diag(1,1,-1,-1);
 *    chirality + is spins {0,1}, chirality - is spins {2,3}.
 *  - periodic in x,y,z; antiperiodic in t when tap != 0 (factor -1 on every hop
 *    that crosses the t = L3-1 <-> 0 face).
 *  - aggregates are hypercubic blocks B[4]; coarse site X = (x/B0, ...) with the
 *    same lexicographic order; coarse dof a = s*Nv + i, s = 0 (+), 1 (-).
 *  - coarse operator A[X][d][a][b], d = 0 on-site, d = 1+2mu for X+mu, d = 2+2mu
 *    for X-mu:  (D_c y)[X] = sum_d A[X][d] y[X+d].
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;
#define OR_API __attribute__((visibility("default")))

enum { OR_OK = 0, OR_ERR_ARG = -1, OR_ERR_NUMERIC = -5, OR_ERR_NOT_CONVERGED = -4 };

/* ------------------------------------------------------------------ */
/* Dirac matrices (DeGrand-Rossi basis), gamma[mu][row][col]           */
/* ------------------------------------------------------------------ */
static cplx GAMMA[4][4][4];
static int gamma_ready = 0;

static void init_gamma(void) {
    if (gamma_ready) return;
    memset(GAMMA, 0, sizeof(GAMMA));
    /* gamma_1 (x) */
    GAMMA[0][0][3] = I;  GAMMA[0][1][2] = I;  GAMMA[0][2][1] = -I; GAMMA[0][3][0] = -I;
    /* gamma_2 (y) */
    GAMMA[1][0][3] = -1; GAMMA[1][1][2] = 1;  GAMMA[1][2][1] = 1;  GAMMA[1][3][0] = -1;
    /* gamma_3 (z) */
    GAMMA[2][0][2] = I;  GAMMA[2][1][3] = -I; GAMMA[2][2][0] = -I; GAMMA[2][3][1] = I;
    /* gamma_4 (t) */
    GAMMA[3][0][2] = 1;  GAMMA[3][1][3] = 1;  GAMMA[3][2][0] = 1;  GAMMA[3][3][1] = 1;
    gamma_ready = 1;
}

OR_API void or_gamma_matrices(double* out /* [4][4][4] complex */) {
    init_gamma();
    memcpy(out, GAMMA, sizeof(GAMMA));
}

/* ------------------------------------------------------------------ */
/* geometry                                                           */
/* ------------------------------------------------------------------ */
static int64_t vol(const int* L) { return (int64_t)L[0] * L[1] * L[2] * L[3]; }

static void coords(const int* L, int64_t s, int c[4]) {
    for (int m = 0; m < 4; ++m) { c[m] = (int)(s % L[m]); s /= L[m]; }
}
static int64_t index_of(const int* L, const int c[4]) {
    return c[0] + (int64_t)L[0] * (c[1] + (int64_t)L[1] * (c[2] + (int64_t)L[2] * c[3]));
}
/* neighbour of s in direction mu, dir = +1/-1; *sign = -1 when the hop
 * crosses the antiperiodic t face */
static int64_t neighbour(const int* L, int tap, int64_t s, int mu, int dir, double* sign) {
    int c[4];
    coords(L, s, c);
    *sign = 1.0;
    int n = c[mu] + dir;
    if (n == L[mu]) { n = 0; if (tap && mu == 3) *sign = -1.0; }
    if (n < 0) { n = L[mu] - 1; if (tap && mu == 3) *sign = -1.0; }
    c[mu] = n;
    return index_of(L, c);
}

/* ------------------------------------------------------------------ */
/* The 12x12 (spin x colour) blocks of eq. (2).                        */
/*   D_{x,y} = (4+m) delta_{x,y}                                      */
/*     - sum_mu [ (1-gamma_mu)/2 U^mu_x delta_{x+mu,y}                 */
/*              + (1+gamma_mu)/2 U^{mu dag}_{x-mu} delta_{x-mu,y} ]     */
/* hop_block(.., dir=+1) is the block multiplying psi(x+mu),           */
/* hop_block(.., dir=-1) the block multiplying psi(x-mu).               */
/* ------------------------------------------------------------------ */
static void hop_block(const int* L, int tap, const cplx* U, int64_t x, int mu, int dir,
                      cplx H[12][12], int64_t* y_out) {
    init_gamma();
    int64_t V = vol(L);
    double sign;
    int64_t y = neighbour(L, tap, x, mu, dir, &sign);
    cplx W[3][3];                                     /* colour part */
    if (dir > 0) {
        const cplx* u = U + 9 * (mu * V + x);           /* U^mu_x */
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) W[a][b] = u[3 * a + b];
    } else {
        const cplx* u = U + 9 * (mu * V + y);           /* U^mu_{x-mu}, daggered */
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) W[a][b] = conj(u[3 * b + a]);
    }
    for (int al = 0; al < 4; ++al)
        for (int be = 0; be < 4; ++be) {
            cplx spin = (al == be ? 1.0 : 0.0) - (double)dir * GAMMA[mu][al][be];   /* 1 -/+ gamma */
            cplx f = -0.5 * sign * spin;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) H[3 * al + a][3 * be + b] = f * W[a][b];
        }
    *y_out = y;
}

/* eq. (2): out = D(U) in.  Each hop applies the colour matrix (U^mu_x or
 * U^{mu dag}_{x-mu}) to every spin component of the neighbour, then the spin
 * matrix -(1 -/+ gamma_mu)/2 (times -1 across the antiperiodic t face). */
OR_API void or_dslash(const int* L, int tap, const double* Ur, double m, const double* inr, double* outr) {
    const cplx* U = (const cplx*)Ur;
    const cplx* in = (const cplx*)inr;
    cplx* out = (cplx*)outr;
    int64_t V = vol(L);
    init_gamma();
    cplx S[4][2][4][4];                       /* S[mu][fwd 0 / bwd 1] = (1 -/+ gamma_mu)/2 */
    for (int mu = 0; mu < 4; ++mu)
        for (int f = 0; f < 2; ++f)
            for (int al = 0; al < 4; ++al)
                for (int be = 0; be < 4; ++be)
                    S[mu][f][al][be] = 0.5 * ((al == be ? 1.0 : 0.0) - (f == 0 ? 1.0 : -1.0) * GAMMA[mu][al][be]);
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < V; ++x) {
        cplx acc[4][3];
        for (int al = 0; al < 4; ++al)
            for (int a = 0; a < 3; ++a) acc[al][a] = (4.0 + m) * in[12 * x + 3 * al + a];
        for (int mu = 0; mu < 4; ++mu)
            for (int f = 0; f < 2; ++f) {
                double sign;
                int64_t y = neighbour(L, tap, x, mu, f == 0 ? 1 : -1, &sign);
                const cplx* u = U + 9 * (mu * V + (f == 0 ? x : y));
                cplx w[4][3];                 /* colour matrix on every spin component of psi(y) */
                for (int be = 0; be < 4; ++be)
                    for (int a = 0; a < 3; ++a) {
                        cplx t = 0;
                        for (int b = 0; b < 3; ++b) {
                            cplx uab = (f == 0) ? u[3 * a + b] : conj(u[3 * b + a]);
                            t += uab * in[12 * y + 3 * be + b];
                        }
                        w[be][a] = t;
                    }
                for (int al = 0; al < 4; ++al)
                    for (int a = 0; a < 3; ++a) {
                        cplx t = 0;
                        for (int be = 0; be < 4; ++be) t += S[mu][f][al][be] * w[be][a];
                        acc[al][a] -= sign * t;
                    }
            }
        for (int al = 0; al < 4; ++al)
            for (int a = 0; a < 3; ++a) out[12 * x + 3 * al + a] = acc[al][a];
    }
}

/* gamma5 = gamma1 gamma2 gamma3 gamma4 = diag(1,1,-1,-1) in this basis (checked in tests) */
OR_API void or_gamma5(int64_t V, const double* inr, double* outr) {
    const cplx* in = (const cplx*)inr;
    cplx* out = (cplx*)outr;
    for (int64_t x = 0; x < V; ++x)
        for (int sp = 0; sp < 4; ++sp)
            for (int c = 0; c < 3; ++c)
                out[12 * x + 3 * sp + c] = (sp < 2 ? 1.0 : -1.0) * in[12 * x + 3 * sp + c];
}

/* ------------------------------------------------------------------ */
/* vector helpers (fixed serial summation order)                       */
/* ------------------------------------------------------------------ */
static cplx vdot(int64_t n, const cplx* a, const cplx* b) {         /* a^dag b */
    cplx s = 0;
    for (int64_t i = 0; i < n; ++i) s += conj(a[i]) * b[i];
    return s;
}
static double vnorm2(int64_t n, const cplx* a) {
    double s = 0;
    for (int64_t i = 0; i < n; ++i) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}
static void vaxpy(int64_t n, cplx a, const cplx* x, cplx* y) {      /* y += a x */
    for (int64_t i = 0; i < n; ++i) y[i] += a * x[i];
}

OR_API void or_dot(int64_t n, const double* a, const double* b, double* out2) {
    cplx s = vdot(n, (const cplx*)a, (const cplx*)b);
    out2[0] = creal(s); out2[1] = cimag(s);
}

/* ------------------------------------------------------------------ */
/* aggregates (geometric blocks), Sec. "Formulating an algorithm"      */
/* ------------------------------------------------------------------ */
typedef struct {
    int L[4], B[4], Lc[4];
    int64_t V, Vc;
    int nv, nc;
} blocking_t;

static int blocking_init(blocking_t* bk, const int* L, const int* B, int nv) {
    for (int m = 0; m < 4; ++m) {
        if (B[m] <= 0 || L[m] % B[m] != 0) return OR_ERR_ARG;
        bk->L[m] = L[m]; bk->B[m] = B[m]; bk->Lc[m] = L[m] / B[m];
    }
    bk->V = vol(L); bk->Vc = vol(bk->Lc); bk->nv = nv; bk->nc = 2 * nv;
    return OR_OK;
}
static int64_t block_of(const blocking_t* bk, int64_t x) {
    int c[4];
    coords(bk->L, x, c);
    for (int m = 0; m < 4; ++m) c[m] /= bk->B[m];
    return index_of(bk->Lc, c);
}
/* list of fine sites of each block, in increasing site order: sites[X*Vb + k] */
static int64_t* block_sites(const blocking_t* bk) {
    int64_t Vb = bk->V / bk->Vc;
    int64_t* sites = (int64_t*)malloc(sizeof(int64_t) * bk->V);
    int64_t* fill = (int64_t*)calloc(bk->Vc, sizeof(int64_t));
    for (int64_t x = 0; x < bk->V; ++x) {
        int64_t X = block_of(bk, x);
        sites[X * Vb + fill[X]++] = x;
    }
    free(fill);
    return sites;
}

/*
 * Block orthonormalisation, eq. (4) and the chirality split of Sec. III:
 * for every aggregate X and chirality s, the columns w_i = (v_i restricted to X
 * and to the spins of chirality s), i = 0..Nv-1, are orthonormalised by
 * modified Gram-Schmidt (two passes, index order).  The result is the Q of a
 * QR factorisation with positive real diag(R), so P^dag P = I_c and
 * P V_c = V.  Output P[i][site][spin][colour] holds column (X, s, i) on the
 * sites of X and spins of chirality s.  Returns OR_ERR_NUMERIC when a column's
 * norm drops below 1e-12 of its original norm (rank deficiency).
 */
OR_API int or_block_orthonormalize(const int* L, const int* B, int nv, const double* vr, double* Pr) {
    blocking_t bk;
    if (blocking_init(&bk, L, B, nv) != OR_OK || nv <= 0) return OR_ERR_ARG;
    const cplx* v = (const cplx*)vr;
    cplx* P = (cplx*)Pr;
    int64_t Vb = bk.V / bk.Vc;
    int64_t len = Vb * 6;                               /* sites x 2 spins x 3 colours */
    int64_t* sites = block_sites(&bk);
    int status = OR_OK;
    cplx* W = (cplx*)malloc(sizeof(cplx) * len * nv);
    double* orig = (double*)malloc(sizeof(double) * nv);
    for (int64_t X = 0; X < bk.Vc; ++X)
        for (int s = 0; s < 2; ++s) {
            for (int i = 0; i < nv; ++i)                /* gather */
                for (int64_t k = 0; k < Vb; ++k)
                    for (int sp = 0; sp < 2; ++sp)
                        for (int c = 0; c < 3; ++c)
                            W[i * len + 6 * k + 3 * sp + c] =
                                v[(int64_t)i * bk.V * 12 + 12 * sites[X * Vb + k] + 3 * (2 * s + sp) + c];
            for (int i = 0; i < nv; ++i) {
                cplx* wi = W + i * len;
                orig[i] = sqrt(vnorm2(len, wi));
                for (int pass = 0; pass < 2; ++pass)
                    for (int j = 0; j < i; ++j) {
                        cplx* qj = W + j * len;
                        cplx c = vdot(len, qj, wi);
                        vaxpy(len, -c, qj, wi);
                    }
                double n = sqrt(vnorm2(len, wi));
                if (!(n > 1e-12 * orig[i])) { status = OR_ERR_NUMERIC; n = 1.0; }
                for (int64_t k = 0; k < len; ++k) wi[k] /= n;
            }
            for (int i = 0; i < nv; ++i)                /* scatter */
                for (int64_t k = 0; k < Vb; ++k)
                    for (int sp = 0; sp < 2; ++sp)
                        for (int c = 0; c < 3; ++c)
                            P[(int64_t)i * bk.V * 12 + 12 * sites[X * Vb + k] + 3 * (2 * s + sp) + c] =
                                W[i * len + 6 * k + 3 * sp + c];
        }
    free(W); free(orig); free(sites);
    return status;
}

/* Restriction r_c = P^dag r (eq. 8 with R = P^dag, chirality kept):
 * r_c[X][s*Nv+i] = sum over x in X, spins of chirality s, colours of conj(P_i(x)) r(x). */
OR_API int or_restrict(const int* L, const int* B, int nv, const double* Pr, const double* rr, double* rcr) {
    blocking_t bk;
    if (blocking_init(&bk, L, B, nv) != OR_OK) return OR_ERR_ARG;
    const cplx* P = (const cplx*)Pr;
    const cplx* r = (const cplx*)rr;
    cplx* rc = (cplx*)rcr;
    int64_t Vb = bk.V / bk.Vc;
    int64_t* sites = block_sites(&bk);
#pragma omp parallel for schedule(static)
    for (int64_t X = 0; X < bk.Vc; ++X)
        for (int s = 0; s < 2; ++s)
            for (int i = 0; i < nv; ++i) {
                cplx acc = 0;
                for (int64_t k = 0; k < Vb; ++k) {
                    int64_t x = sites[X * Vb + k];
                    for (int sp = 2 * s; sp < 2 * s + 2; ++sp)
                        for (int c = 0; c < 3; ++c)
                            acc += conj(P[(int64_t)i * bk.V * 12 + 12 * x + 3 * sp + c]) * r[12 * x + 3 * sp + c];
                }
                rc[X * bk.nc + s * nv + i] = acc;
            }
    free(sites);
    return OR_OK;
}

/* Prolongation e = P y: e(x, spin, c) = sum_i P_i(x, spin, c) y[X(x)][s(spin)*Nv + i]. */
OR_API int or_prolong(const int* L, const int* B, int nv, const double* Pr, const double* ycr, double* er) {
    blocking_t bk;
    if (blocking_init(&bk, L, B, nv) != OR_OK) return OR_ERR_ARG;
    const cplx* P = (const cplx*)Pr;
    const cplx* yc = (const cplx*)ycr;
    cplx* e = (cplx*)er;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < bk.V; ++x) {
        int64_t X = block_of(&bk, x);
        for (int sp = 0; sp < 4; ++sp) {
            int s = sp < 2 ? 0 : 1;
            for (int c = 0; c < 3; ++c) {
                cplx acc = 0;
                for (int i = 0; i < nv; ++i)
                    acc += P[(int64_t)i * bk.V * 12 + 12 * x + 3 * sp + c] * yc[X * bk.nc + s * nv + i];
                e[12 * x + 3 * sp + c] = acc;
            }
        }
    }
    return OR_OK;
}

/*
 * Galerkin coarse operator D_c = P^dag D P (Sec. II, "A_c = P^dag A P"; its
 * nearest-neighbour form with 2Nv x 2Nv links, Sec. III):
 *   A[X][d][a][b] = sum_{x in X} sum_y conj(P_a(x)) D^{(d)}_{x,y} P_b(y)
 * where D^{(0)} is the diagonal term of eq. (2) plus every hop that stays
 * inside X, and D^{(+mu)} / D^{(-mu)} are the hops that leave X through its
 * +mu / -mu face.  Keeping the face of exit (rather than the target block)
 * makes the 9-term sum exact even when the coarse extent is 1 or 2.
 */
OR_API int or_coarse_build(const int* L, const int* B, int nv, int tap, const double* Ur, double m,
                           const double* Pr, double* Ar) {
    blocking_t bk;
    if (blocking_init(&bk, L, B, nv) != OR_OK) return OR_ERR_ARG;
    const cplx* U = (const cplx*)Ur;
    const cplx* P = (const cplx*)Pr;
    cplx* A = (cplx*)Ar;
    int nc = bk.nc;
    int64_t Vb = bk.V / bk.Vc;
    int64_t* sites = block_sites(&bk);
    memset(A, 0, sizeof(cplx) * bk.Vc * 9 * nc * nc);
#pragma omp parallel
    {
        cplx* HP = (cplx*)malloc(sizeof(cplx) * 12 * nc);
#pragma omp for schedule(static)
        for (int64_t X = 0; X < bk.Vc; ++X)
            for (int64_t k = 0; k < Vb; ++k) {
                int64_t x = sites[X * Vb + k];
                int cx[4];
                coords(L, x, cx);
                for (int term = 0; term < 9; ++term) {
                    cplx H[12][12];
                    int64_t y;
                    int d;
                    if (term == 0) {
                        memset(H, 0, sizeof(H));
                        for (int q = 0; q < 12; ++q) H[q][q] = 4.0 + m;
                        y = x;
                        d = 0;
                    } else {
                        int mu = (term - 1) / 2, dir = (term % 2 == 1) ? 1 : -1;
                        hop_block(L, tap, U, x, mu, dir, H, &y);
                        int leaves = (dir > 0) ? (cx[mu] % B[mu] == B[mu] - 1) : (cx[mu] % B[mu] == 0);
                        d = leaves ? term : 0;
                    }
                    /* HP[q][b] = (H P_b)(x) restricted to row q; P_b(y) is column b at site y */
                    for (int q = 0; q < 12; ++q)
                        for (int b = 0; b < nc; ++b) {
                            int sb = b / nv, ib = b % nv;
                            cplx acc = 0;
                            for (int sp = 2 * sb; sp < 2 * sb + 2; ++sp)
                                for (int c = 0; c < 3; ++c)
                                    acc += H[q][3 * sp + c] * P[(int64_t)ib * bk.V * 12 + 12 * y + 3 * sp + c];
                            HP[q * nc + b] = acc;
                        }
                    cplx* Ad = A + (X * 9 + d) * nc * nc;
                    for (int a = 0; a < nc; ++a) {
                        int sa = a / nv, ia = a % nv;
                        for (int b = 0; b < nc; ++b) {
                            cplx acc = 0;
                            for (int sp = 2 * sa; sp < 2 * sa + 2; ++sp)
                                for (int c = 0; c < 3; ++c)
                                    acc += conj(P[(int64_t)ia * bk.V * 12 + 12 * x + 3 * sp + c]) * HP[(3 * sp + c) * nc + b];
                            Ad[a * nc + b] += acc;
                        }
                    }
                }
            }
        free(HP);
    }
    free(sites);
    return OR_OK;
}

/* neighbour of coarse site X for stencil slot d (0 = X itself) */
static int64_t coarse_neighbour(const int* Lc, int64_t X, int d) {
    if (d == 0) return X;
    int mu = (d - 1) / 2, dir = (d % 2 == 1) ? 1 : -1;
    int c[4];
    coords(Lc, X, c);
    c[mu] = (c[mu] + dir + Lc[mu]) % Lc[mu];
    return index_of(Lc, c);
}

/* y = D_c x : y[X] = sum_d A[X][d] x[X+d] */
OR_API void or_coarse_apply(const int* Lc, int nc, const double* Ar, const double* xr, double* yr) {
    const cplx* A = (const cplx*)Ar;
    const cplx* x = (const cplx*)xr;
    cplx* y = (cplx*)yr;
    int64_t Vc = vol(Lc);
#pragma omp parallel for schedule(static)
    for (int64_t X = 0; X < Vc; ++X) {
        for (int a = 0; a < nc; ++a) {
            cplx acc = 0;
            for (int d = 0; d < 9; ++d) {
                int64_t Y = coarse_neighbour(Lc, X, d);
                const cplx* Ad = A + (X * 9 + d) * nc * nc;
                for (int b = 0; b < nc; ++b) acc += Ad[a * nc + b] * x[Y * nc + b];
            }
            y[X * nc + a] = acc;
        }
    }
}

/* sigma3 on coarse vectors: +1 on the first Nv dof of a site, -1 on the last Nv */
static void sigma3(int64_t Vc, int nc, const cplx* x, cplx* y) {
    for (int64_t X = 0; X < Vc; ++X)
        for (int a = 0; a < nc; ++a) y[X * nc + a] = (a < nc / 2 ? 1.0 : -1.0) * x[X * nc + a];
}

/* y = D_c^dag x = sigma3 D_c sigma3 x, from P^dag gamma5 = sigma3 P^dag (Sec. III) */
OR_API void or_coarse_apply_dag(const int* Lc, int nc, const double* Ar, const double* xr, double* yr) {
    int64_t Vc = vol(Lc);
    cplx* t = (cplx*)malloc(sizeof(cplx) * Vc * nc);
    sigma3(Vc, nc, (const cplx*)xr, t);
    or_coarse_apply(Lc, nc, Ar, (const double*)t, yr);
    sigma3(Vc, nc, (const cplx*)yr, (cplx*)yr);
    free(t);
}

/* ------------------------------------------------------------------ */
/* solver parameters and the multigrid state                          */
/* ------------------------------------------------------------------ */
typedef struct {
    int L[4];
    int B[4];
    int nv;
    int tap;
    double m;
    int mr_steps;        /* post-smoothing steps, V(0, mr_steps) */
    double omega;        /* under-relaxation of the smoother */
    double coarse_tol;   /* relative residual of the coarse normal-equation CG */
    int coarse_maxit;
    int gcr_restart;
    double tol;          /* outer relative true residual */
    int max_outer;
    int use_mg;          /* 0: unpreconditioned GCR (M = I) */
    int smoother;        /* 0: mr_steps MR steps; 1: one GMRES(mr_steps) application */
    /* third level (Sec. IV's 3-level W-cycle); levels = 2 ignores the rest */
    int levels;          /* 2 or 3 */
    int B2[4];           /* aggregates of the first coarse lattice (level 1 -> level 2) */
    int nv2;             /* prototypes of level 2 (2 nv2 dof per level-2 site) */
    int smoother1;       /* level-1 post-smoother: 0 MR steps, 1 one GMRES(steps1) */
    int steps1;
    int cycles1;         /* level-1 V-cycles per fine-grid correction (2: the W-cycle) */
} or_params;

typedef struct {
    int outer_iters;
    int coarse_iters;
    int fine_matvecs;
    int restarts;
    double true_rel_res;
    int status;
} or_info;

typedef struct {
    const or_params* p;
    blocking_t bk;
    const cplx* U;
    const cplx* P;
    const cplx* A;
    const cplx* P2;      /* third level (levels = 3): level-2 prolongator and operator */
    const cplx* A2;
    or_info* info;
} mg_t;

static void kcycle_l1(const mg_t* g, const cplx* r1, cplx* e1);

static void D_apply(const mg_t* g, const cplx* in, cplx* out) {
    or_dslash(g->p->L, g->p->tap, (const double*)g->U, g->p->m, (const double*)in, (double*)out);
    if (g->info) g->info->fine_matvecs++;
}

/*
 * Minimal-residual relaxation with under-relaxation omega (the smoother of
 * Sec. III, GMRES with omega = 0.9, in its one-vector restarted form):
 *   repeat n times: q = D r; alpha = omega <q,r>/<q,q>; e += alpha r; r -= alpha q
 * e and r are updated in place.
 */
OR_API void or_mr(const int* L, int tap, const double* Ur, double m, int nsteps, double omega,
                  double* er, double* rr) {
    int64_t n = vol(L) * 12;
    cplx* e = (cplx*)er;
    cplx* r = (cplx*)rr;
    cplx* q = (cplx*)malloc(sizeof(cplx) * n);
    for (int k = 0; k < nsteps; ++k) {
        or_dslash(L, tap, Ur, m, (const double*)r, (double*)q);
        cplx qr = vdot(n, q, r);
        double qq = vnorm2(n, q);
        if (!(qq > 0)) break;
        cplx alpha = omega * qr / qq;
        vaxpy(n, alpha, r, e);
        vaxpy(n, -alpha, q, r);
    }
    free(q);
}

static void mr_internal(const mg_t* g, int nsteps, cplx* e, cplx* r) {
    int64_t n = g->bk.V * 12;
    cplx* q = (cplx*)malloc(sizeof(cplx) * n);
    for (int k = 0; k < nsteps; ++k) {
        D_apply(g, r, q);
        cplx qr = vdot(n, q, r);
        double qq = vnorm2(n, q);
        if (!(qq > 0)) break;
        cplx alpha = g->p->omega * qr / qq;
        vaxpy(n, alpha, r, e);
        vaxpy(n, -alpha, q, r);
    }
    free(q);
}

/*
 * GMRES(k) post-smoothing with under-relaxation (Sec. III: GMRES as the
 * smoother with omega = 0.9; Sec. IV: the post-relaxation is one application
 * of GMRES(4)).  With r = r_in - D e: Arnoldi on the Krylov space
 * K_k(D, r), beta = ||r||, v_0 = r / beta, for j < k: w = D v_j,
 * h_ij = <v_i, w> (i <= j), w -= sum_i h_ij v_i (one classical Gram-Schmidt
 * pass), h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}; then
 * y = argmin || beta e_1 - Hbar y || (Givens rotations) and e += omega V_k y.
 * A zero h_{j+1,j} ends the space at dimension j + 1 (exact solution in it).
 */
static void gmres_smooth(const mg_t* g, int k, cplx* e, const cplx* r) {
    int64_t n = g->bk.V * 12;
    double beta = sqrt(vnorm2(n, r));
    if (!(beta > 0) || k <= 0) return;
    cplx* V = (cplx*)malloc(sizeof(cplx) * n * (k + 1));
    cplx* H = (cplx*)calloc((size_t)(k + 1) * k, sizeof(cplx));   /* H[i * k + j] */
    for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
    int dim = k;
    for (int j = 0; j < k; ++j) {
        cplx* w = V + (int64_t)(j + 1) * n;
        D_apply(g, V + (int64_t)j * n, w);
        for (int i = 0; i <= j; ++i) H[i * k + j] = vdot(n, V + (int64_t)i * n, w);
        for (int i = 0; i <= j; ++i) vaxpy(n, -H[i * k + j], V + (int64_t)i * n, w);
        double hn = sqrt(vnorm2(n, w));
        H[(j + 1) * k + j] = hn;
        if (!(hn > 0)) { dim = j + 1; break; }
        for (int64_t i = 0; i < n; ++i) w[i] /= hn;
    }
    /* least squares by Givens rotations: R y = Q^dag beta e_1 */
    cplx* g1 = (cplx*)calloc((size_t)dim + 1, sizeof(cplx));
    g1[0] = beta;
    for (int j = 0; j < dim; ++j) {
        cplx a = H[j * k + j], b = H[(j + 1) * k + j];
        double nrm = sqrt(creal(a) * creal(a) + cimag(a) * cimag(a) + creal(b) * creal(b) + cimag(b) * cimag(b));
        if (!(nrm > 0)) continue;
        cplx c = a / nrm, s = b / nrm;   /* [conj(c) conj(s); -s c] maps (a, b) to (nrm, 0) */
        for (int jj = j; jj < dim; ++jj) {
            cplx x1 = H[j * k + jj], x2 = H[(j + 1) * k + jj];
            H[j * k + jj] = conj(c) * x1 + conj(s) * x2;
            H[(j + 1) * k + jj] = -s * x1 + c * x2;
        }
        cplx t1 = g1[j], t2 = g1[j + 1];
        g1[j] = conj(c) * t1 + conj(s) * t2;
        g1[j + 1] = -s * t1 + c * t2;
    }
    cplx* y = (cplx*)calloc((size_t)dim, sizeof(cplx));
    for (int i = dim - 1; i >= 0; --i) {
        cplx acc = g1[i];
        for (int jj = i + 1; jj < dim; ++jj) acc -= H[i * k + jj] * y[jj];
        y[i] = acc / H[i * k + i];
    }
    for (int j = 0; j < dim; ++j) vaxpy(n, g->p->omega * y[j], V + (int64_t)j * n, e);
    free(V); free(H); free(g1); free(y);
}

/* e += omega * argmin_{d in K_k(D, r)} ||r - D d|| (the GMRES(k) smoother on
 * its own: e and r given, r = the residual of e; e is updated in place). */
OR_API void or_gmres_smooth(const int* L, int tap, const double* Ur, double m, int k, double omega, double* er,
                            const double* rr) {
    or_params p;
    memset(&p, 0, sizeof(p));
    for (int i = 0; i < 4; ++i) p.L[i] = L[i];
    p.tap = tap;
    p.m = m;
    p.omega = omega;
    mg_t g;
    memset(&g, 0, sizeof(g));
    g.p = &p;
    g.U = (const cplx*)Ur;
    g.bk.V = vol(L);
    gmres_smooth(&g, k, (cplx*)er, (const cplx*)rr);
}

/*
 * Coarsest-grid solve: conjugate gradients on the normal equations
 * (D_c^dag D_c y = D_c^dag r_c), CGLS form, from y = 0, stopping when the
 * residual of the original system ||r_c - D_c y|| <= tol ||r_c|| (Sec. IV:
 * "CG on the normal equations to a relative accuracy of 1e-3") or after maxit
 * iterations.  tol = 0 runs exactly maxit iterations.  Returns the count.
 */
OR_API int or_cgnr(const int* Lc, int nc, const double* Ar, const double* rcr, double* yr,
                   double tol, int maxit, double* final_rel) {
    int64_t Vc = vol(Lc);
    int64_t n = Vc * nc;
    const cplx* rc = (const cplx*)rcr;
    cplx* y = (cplx*)yr;
    cplx* r = (cplx*)malloc(sizeof(cplx) * n);
    cplx* s = (cplx*)malloc(sizeof(cplx) * n);
    cplx* p = (cplx*)malloc(sizeof(cplx) * n);
    cplx* q = (cplx*)malloc(sizeof(cplx) * n);
    memset(y, 0, sizeof(cplx) * n);
    memcpy(r, rc, sizeof(cplx) * n);
    double rc_norm = sqrt(vnorm2(n, rc));
    or_coarse_apply_dag(Lc, nc, Ar, (const double*)r, (double*)s);
    memcpy(p, s, sizeof(cplx) * n);
    double gamma = vnorm2(n, s);
    int it = 0;
    double rel = rc_norm > 0 ? 1.0 : 0.0;
    if (rc_norm > 0) {
        while (it < maxit) {
            or_coarse_apply(Lc, nc, Ar, (const double*)p, (double*)q);
            double qq = vnorm2(n, q);
            if (!(qq > 0)) break;
            double alpha = gamma / qq;
            vaxpy(n, alpha, p, y);
            vaxpy(n, -alpha, q, r);
            ++it;
            rel = sqrt(vnorm2(n, r)) / rc_norm;
            if (rel <= tol) break;
            or_coarse_apply_dag(Lc, nc, Ar, (const double*)r, (double*)s);
            double gnew = vnorm2(n, s);
            double beta = gnew / gamma;
            gamma = gnew;
            for (int64_t i = 0; i < n; ++i) p[i] = s[i] + beta * p[i];
        }
    }
    if (final_rel) *final_rel = rel;
    free(r); free(s); free(p); free(q);
    return it;
}

/*
 * Two-level V(0, n) cycle used as the preconditioner M (Sec. II-III):
 *   r_c = P^dag r;  y = CGNR(D_c, r_c);  e = P y;  r' = r - D e;
 *   n MR steps on (e, r');  return z = e.
 * (Coarse-grid correction eq. (8) with R = P^dag, then post-relaxation only.)
 */
static void vcycle(const mg_t* g, const cplx* r_in, cplx* z) {
    int64_t n = g->bk.V * 12, nC = g->bk.Vc * g->bk.nc;
    const or_params* p = g->p;
    cplx* rc = (cplx*)malloc(sizeof(cplx) * nC);
    cplx* yc = (cplx*)malloc(sizeof(cplx) * nC);
    cplx* r = (cplx*)malloc(sizeof(cplx) * n);
    cplx* De = (cplx*)malloc(sizeof(cplx) * n);
    or_restrict(p->L, p->B, p->nv, (const double*)g->P, (const double*)r_in, (double*)rc);
    if (p->levels == 3 && g->P2) {
        kcycle_l1(g, rc, yc);                  /* Sec. IV: V-cycles on the intermediate grid */
    } else {
        int it = or_cgnr(g->bk.Lc, g->bk.nc, (const double*)g->A, (const double*)rc, (double*)yc,
                         p->coarse_tol, p->coarse_maxit, NULL);
        if (g->info) g->info->coarse_iters += it;
    }
    or_prolong(p->L, p->B, p->nv, (const double*)g->P, (const double*)yc, (double*)z);
    D_apply(g, z, De);
    for (int64_t i = 0; i < n; ++i) r[i] = r_in[i] - De[i];
    if (p->smoother == 1)
        gmres_smooth(g, p->mr_steps, z, r);
    else
        mr_internal(g, p->mr_steps, z, r);
    free(rc); free(yc); free(r); free(De);
}

OR_API void or_vcycle(const or_params* p, const double* U, const double* P, const double* A,
                      const double* r, double* z, or_info* info) {
    mg_t g;
    blocking_init(&g.bk, p->L, p->B, p->nv);
    g.p = p; g.U = (const cplx*)U; g.P = (const cplx*)P; g.A = (const cplx*)A; g.info = info;
    g.P2 = NULL; g.A2 = NULL;
    vcycle(&g, (const cplx*)r, (cplx*)z);
}

/* one fine-grid cycle of the three-level method (p->levels = 3) */
OR_API void or_vcycle3(const or_params* p, const double* U, const double* P, const double* A, const double* P2,
                       const double* A2, const double* r, double* z, or_info* info) {
    mg_t g;
    blocking_init(&g.bk, p->L, p->B, p->nv);
    g.p = p; g.U = (const cplx*)U; g.P = (const cplx*)P; g.A = (const cplx*)A; g.info = info;
    g.P2 = (const cplx*)P2; g.A2 = (const cplx*)A2;
    vcycle(&g, (const cplx*)r, (cplx*)z);
}

/*
 * Flexible GCR(k) preconditioned by the multigrid cycle (Sec. III: "GCR(8)";
 * the restart length k is a parameter).  x starts at 0.  Per iteration:
 *   z_k = M r;  p_k = D z_k;  p_k -= sum_{j<k} <p_j,p_k> p_j (one classical
 *   Gram-Schmidt pass);  R_kk = ||p_k||, p_k /= R_kk;  c_k = <p_k, r>;
 *   r -= c_k p_k.
 * At a restart (k iterations) or when ||r|| <= tol ||b||: solve R y = c
 * (upper triangular), x += sum_k y_k z_k, r = b - D x (true residual).
 * Converged when the true relative residual is <= tol.
 */
static int gcr_solve_impl(const or_params* p, const double* Ur, const double* Pr, const double* Ar,
                          const double* P2r, const double* A2r, const double* br, double* xr, or_info* info);

OR_API int or_gcr_solve(const or_params* p, const double* Ur, const double* Pr, const double* Ar,
                        const double* br, double* xr, or_info* info) {
    return gcr_solve_impl(p, Ur, Pr, Ar, NULL, NULL, br, xr, info);
}

/* the same with the third level: P2r, A2r from or_setup_level2 (p->levels = 3) */
OR_API int or_gcr_solve3(const or_params* p, const double* Ur, const double* Pr, const double* Ar,
                         const double* P2r, const double* A2r, const double* br, double* xr, or_info* info) {
    return gcr_solve_impl(p, Ur, Pr, Ar, P2r, A2r, br, xr, info);
}

static int gcr_solve_impl(const or_params* p, const double* Ur, const double* Pr, const double* Ar,
                          const double* P2r, const double* A2r, const double* br, double* xr, or_info* info) {
    mg_t g;
    if (p->use_mg) {
        if (blocking_init(&g.bk, p->L, p->B, p->nv) != OR_OK) return OR_ERR_ARG;
    } else {
        memset(&g.bk, 0, sizeof(g.bk));
        g.bk.V = vol(p->L);
    }
    or_info local;
    memset(&local, 0, sizeof(local));
    g.p = p; g.U = (const cplx*)Ur; g.P = (const cplx*)Pr; g.A = (const cplx*)Ar; g.info = &local;
    g.P2 = (const cplx*)P2r; g.A2 = (const cplx*)A2r;
    int64_t n = g.bk.V * 12;
    int K = p->gcr_restart;
    const cplx* b = (const cplx*)br;
    cplx* x = (cplx*)xr;
    cplx* r = (cplx*)malloc(sizeof(cplx) * n);
    cplx* Z = (cplx*)malloc(sizeof(cplx) * n * K);
    cplx* Pk = (cplx*)malloc(sizeof(cplx) * n * K);
    cplx* R = (cplx*)calloc((size_t)K * K, sizeof(cplx));
    cplx* c = (cplx*)malloc(sizeof(cplx) * K);
    cplx* yk = (cplx*)malloc(sizeof(cplx) * K);
    cplx* t = (cplx*)malloc(sizeof(cplx) * n);
    memset(x, 0, sizeof(cplx) * n);
    memcpy(r, b, sizeof(cplx) * n);
    double bnorm = sqrt(vnorm2(n, b));
    double rel = bnorm > 0 ? 1.0 : 0.0;
    int status = OR_ERR_NOT_CONVERGED;
    if (bnorm == 0) status = OR_OK;
    while (status == OR_ERR_NOT_CONVERGED && local.outer_iters < p->max_outer) {
        int k = 0;
        for (; k < K && local.outer_iters < p->max_outer;) {
            cplx* zk = Z + (int64_t)k * n;
            cplx* pk = Pk + (int64_t)k * n;
            if (p->use_mg) vcycle(&g, r, zk);
            else memcpy(zk, r, sizeof(cplx) * n);
            D_apply(&g, zk, pk);
            for (int j = 0; j < k; ++j) R[j * K + k] = vdot(n, Pk + (int64_t)j * n, pk);
            for (int j = 0; j < k; ++j) vaxpy(n, -R[j * K + k], Pk + (int64_t)j * n, pk);
            double nk = sqrt(vnorm2(n, pk));
            if (!(nk > 0) || !isfinite(nk)) { status = OR_ERR_NUMERIC; break; }
            R[k * K + k] = nk;
            for (int64_t i = 0; i < n; ++i) pk[i] /= nk;
            c[k] = vdot(n, pk, r);
            vaxpy(n, -c[k], pk, r);
            ++k;
            local.outer_iters++;
            if (sqrt(vnorm2(n, r)) <= p->tol * bnorm) break;
        }
        if (status == OR_ERR_NUMERIC) break;
        for (int i = k - 1; i >= 0; --i) {                 /* back substitution R y = c */
            cplx s = c[i];
            for (int j = i + 1; j < k; ++j) s -= R[i * K + j] * yk[j];
            yk[i] = s / R[i * K + i];
        }
        for (int i = 0; i < k; ++i) vaxpy(n, yk[i], Z + (int64_t)i * n, x);
        D_apply(&g, x, t);                                  /* true residual */
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
        local.restarts++;
        rel = sqrt(vnorm2(n, r)) / bnorm;
        if (!isfinite(rel)) { status = OR_ERR_NUMERIC; break; }
        if (rel <= p->tol) status = OR_OK;
    }
    local.true_rel_res = rel;
    local.status = status;
    if (info) *info = local;
    free(r); free(Z); free(Pk); free(R); free(c); free(yk); free(t);
    return status;
}

/*
 * Adaptive setup (Sec. II, the alpha-SA loop, in the two-step practical form
 * of Sec. IV):
 *  (i)   start from the given random vectors v_i (i = 0..Nv-1);
 *  (ii)  relaxation of each on D v = 0: init_relax MR steps with the error
 *        e = v_i and residual r = -D v_i, then normalise;
 *  (iii) refinement by groups: the Nv prototypes are split into consecutive
 *        groups of group_size.  One group at a time is taken out of V; the
 *        truncated two-level method is built from the remaining prototypes
 *        (P_t = block-orthonormalised V without the group, D_c,t = P_t^dag D P_t)
 *        and iterated n_iter times on D x = 0 starting from each prototype of
 *        the group, v <- (I - M_t D) v (normalised after each iteration); the
 *        group is then put back.  Groups are processed in order, each seeing
 *        the already refined earlier groups.
 *  (iv)  P = block-orthonormalised V, D_c = P^dag D P.
 * V is overwritten with the final prototypes; P and A receive the final
 * prolongator and coarse operator.  n_iter = 0 (or group_size >= Nv) skips
 * step (iii).
 */
/*
 * The truncated level of the group refinement (Sec. IV: a group is removed
 * from V and the multigrid method built from the remaining prototypes):
 * Vt = V without prototypes g0 .. g0 + group_size - 1 (order kept),
 * Pt = block-orthonormalised Vt (eq. 4), At = Pt^dag D Pt.  Vt, Pt hold
 * nv - group_size fine vectors; At the coarse operator of that many.
 */
OR_API int or_setup_truncated_level(const or_params* p, const double* Ur, const double* Vr, int g0,
                                    int group_size, double* Vtr, double* Ptr, double* Atr) {
    int64_t n = vol(p->L) * 12;
    int nv = p->nv, nt = nv - group_size;
    if (group_size <= 0 || nt <= 0 || g0 < 0 || g0 + group_size > nv) return OR_ERR_ARG;
    const cplx* V = (const cplx*)Vr;
    cplx* Vt = (cplx*)Vtr;
    int k = 0;
    for (int i = 0; i < nv; ++i)
        if (i < g0 || i >= g0 + group_size) memcpy(Vt + (int64_t)(k++) * n, V + (int64_t)i * n, sizeof(cplx) * n);
    int st = or_block_orthonormalize(p->L, p->B, nt, Vtr, Ptr);
    if (st != OR_OK) return st;
    or_coarse_build(p->L, p->B, nt, p->tap, Ur, p->m, Ptr, Atr);
    return OR_OK;
}

OR_API int or_setup_counted(const or_params* p, const double* Ur, double* Vr, int init_relax, int n_iter,
                            int group_size, double* Pr, double* Ar, or_info* info);

OR_API int or_setup(const or_params* p, const double* Ur, double* Vr, int init_relax, int n_iter,
                    int group_size, double* Pr, double* Ar) {
    return or_setup_counted(p, Ur, Vr, init_relax, n_iter, group_size, Pr, Ar, NULL);
}

/* or_setup that also reports its work (info may be NULL): fine_matvecs counts
 * the operator applications of the relaxation and of the truncated cycles,
 * coarse_iters the coarse CG iterations of those cycles. */
OR_API int or_setup_counted(const or_params* p, const double* Ur, double* Vr, int init_relax, int n_iter,
                            int group_size, double* Pr, double* Ar, or_info* info) {
    or_info local;
    memset(&local, 0, sizeof(local));
    blocking_t bk;
    if (blocking_init(&bk, p->L, p->B, p->nv) != OR_OK) return OR_ERR_ARG;
    if (group_size <= 0 || p->nv % group_size != 0) return OR_ERR_ARG;
    int64_t n = bk.V * 12;
    int nv = p->nv;
    cplx* V = (cplx*)Vr;
    cplx* r = (cplx*)malloc(sizeof(cplx) * n);
    cplx* z = (cplx*)malloc(sizeof(cplx) * n);
    int st = OR_OK;
    for (int i = 0; i < nv; ++i) {
        cplx* v = V + (int64_t)i * n;
        or_dslash(p->L, p->tap, Ur, p->m, (const double*)v, (double*)r);
        for (int64_t k = 0; k < n; ++k) r[k] = -r[k];
        or_mr(p->L, p->tap, Ur, p->m, init_relax, p->omega, (double*)v, (double*)r);
        local.fine_matvecs += 1 + init_relax;
        double nrm = sqrt(vnorm2(n, v));
        for (int64_t k = 0; k < n; ++k) v[k] /= nrm;
    }
    int nt = nv - group_size;
    if (n_iter > 0 && nt > 0) {
        blocking_t bt;
        blocking_init(&bt, p->L, p->B, nt);
        or_params pt = *p;
        pt.nv = nt;
        cplx* Vt = (cplx*)malloc(sizeof(cplx) * n * nt);
        cplx* Pt = (cplx*)malloc(sizeof(cplx) * n * nt);
        cplx* At = (cplx*)malloc(sizeof(cplx) * bt.Vc * 9 * bt.nc * bt.nc);
        for (int g0 = 0; g0 < nv && st == OR_OK; g0 += group_size) {
            st = or_setup_truncated_level(p, Ur, Vr, g0, group_size, (double*)Vt, (double*)Pt, (double*)At);
            if (st != OR_OK) break;
            mg_t g;
            g.bk = bt; g.p = &pt; g.U = (const cplx*)Ur; g.P = Pt; g.A = At; g.info = &local;
            g.P2 = NULL; g.A2 = NULL;
            pt.levels = 2;                     /* the truncated method is two-level */
            for (int i = g0; i < g0 + group_size; ++i) {
                cplx* v = V + (int64_t)i * n;
                for (int it = 0; it < n_iter; ++it) {
                    D_apply(&g, v, r);                  /* residual of D x = 0 at x = v is -D v */
                    for (int64_t q = 0; q < n; ++q) r[q] = -r[q];
                    vcycle(&g, r, z);
                    for (int64_t q = 0; q < n; ++q) v[q] += z[q];
                    double nrm = sqrt(vnorm2(n, v));
                    for (int64_t q = 0; q < n; ++q) v[q] /= nrm;
                }
            }
        }
        free(Vt); free(Pt); free(At);
    }
    if (st == OR_OK) st = or_block_orthonormalize(p->L, p->B, nv, Vr, Pr);
    if (st == OR_OK) or_coarse_build(p->L, p->B, nv, p->tap, Ur, p->m, Pr, Ar);
    free(r); free(z);
    local.status = st;
    if (info) *info = local;
    return st;
}

/* ------------------------------------------------------------------ */
/* Red-black (even-odd) preconditioned CG on the normal equations: the  */
/* comparison solver of Sec. IV (Fig. 1 counts its Wilson matrix-vector */
/* products, Fig. 2 its flops against MG-GCR).  The paper names it and  */
/* uses it; the construction below is the standard one it refers to.    */
/*                                                                     */
/* With H the hopping part of eq. 2 (D = (4+m) I - H) and sites split   */
/* by parity (x+y+z+t) mod 2, H couples only opposite parities on a     */
/* lattice of even extents.  Eliminating the odd sites leaves the Schur */
/* complement on the even sites                                          */
/*     Dhat = (4+m) I - H_eo H_oe / (4+m),                               */
/*     Dhat x_e = bhat,  bhat = b_e + H_eo b_o / (4+m),                  */
/*     x_o = (b_o + H_oe x_e) / (4+m),                                   */
/* and b - D x vanishes on the odd sites and equals bhat - Dhat x_e on   */
/* the even ones.  Dhat^dag = gamma5 Dhat gamma5 (gamma5-hermiticity of  */
/* D carries over, H_eo^dag = gamma5 H_oe gamma5).                       */
/* ------------------------------------------------------------------ */
static int site_parity(const int* L, int64_t s) {
    int c[4];
    coords(L, s, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* out = H in on the sites of parity p (zero on the others), in read on the
 * sites of parity 1 - p.  H in = -D(m = -4) in (eq. 2 with 4 + m = 0). */
static void hop_to_parity(const int* L, int tap, const double* U, int p, const cplx* in, cplx* out, cplx* tmp) {
    int64_t V = vol(L);
    for (int64_t s = 0; s < V; ++s)
        for (int k = 0; k < 12; ++k) tmp[12 * s + k] = site_parity(L, s) == 1 - p ? in[12 * s + k] : 0;
    or_dslash(L, tap, U, -4.0, (const double*)tmp, (double*)out);
    for (int64_t s = 0; s < V; ++s)
        for (int k = 0; k < 12; ++k) out[12 * s + k] = site_parity(L, s) == p ? -out[12 * s + k] : 0;
}

/* out = Dhat xe (even sites; xe read on the even sites), dag: gamma5 Dhat gamma5 */
static void schur_apply(const int* L, int tap, const double* U, double m, int dag, const cplx* xe, cplx* out,
                        cplx* t1, cplx* t2, cplx* t3) {
    int64_t V = vol(L);
    const double a = 4.0 + m;
    const cplx* x = xe;
    if (dag) {
        or_gamma5(V, (const double*)xe, (double*)t3);
        x = t3;
    }
    hop_to_parity(L, tap, U, 1, x, t1, t2);       /* t1 = H_oe x (odd sites) */
    hop_to_parity(L, tap, U, 0, t1, out, t2);     /* out = H_eo H_oe x (even sites) */
    for (int64_t s = 0; s < V; ++s)
        for (int k = 0; k < 12; ++k)
            out[12 * s + k] = site_parity(L, s) == 0 ? a * x[12 * s + k] - out[12 * s + k] / a : 0;
    if (dag) or_gamma5(V, (const double*)out, (double*)out);
}

OR_API void or_eo_schur(const int* L, int tap, const double* U, double m, int dag, const double* xe, double* out) {
    int64_t n = vol(L) * 12;
    cplx* t = (cplx*)malloc(sizeof(cplx) * 3 * n);
    schur_apply(L, tap, U, m, dag, (const cplx*)xe, (cplx*)out, t, t + n, t + 2 * n);
    free(t);
}

/*
 * Solve D x = b: CGLS on Dhat from x_e = 0 (r = bhat, s = Dhat^dag r, p = s;
 * per iteration q = Dhat p, alpha = |s|^2 / |q|^2, x_e += alpha p,
 * r -= alpha q, stop when |r| <= tol |b|, else s = Dhat^dag r,
 * beta = |s_new|^2 / |s|^2, p = s + beta p), then x_o from x_e and the true
 * residual |b - D x| / |b| with the full operator.  If the recursive residual
 * has drifted above the true one's target, the solve restarts on the true
 * residual (the correction is added to x).  iters counts CG iterations;
 * matvecs counts applications of Dhat or Dhat^dag (each two half-lattice
 * hops: one full-lattice hopping term) plus the full-lattice products of the
 * source preparation, the odd-site reconstruction and the residual checks.
 */
OR_API int or_eo_cg(const int* L, int tap, const double* Ur, double m, const double* br, double* xr, double tol,
                    int maxit, int* iters_out, int* matvecs_out, double* rel_out) {
    int64_t V = vol(L), n = V * 12;
    for (int mu = 0; mu < 4; ++mu)
        if (L[mu] % 2) return OR_ERR_ARG;
    const double a = 4.0 + m;
    const cplx* b = (const cplx*)br;
    cplx* x = (cplx*)xr;
    cplx* w = (cplx*)malloc(sizeof(cplx) * n * 10);
    cplx *bh = w, *xe = w + n, *r = w + 2 * n, *s = w + 3 * n, *p = w + 4 * n, *q = w + 5 * n, *res = w + 6 * n;
    cplx *t1 = w + 7 * n, *t2 = w + 8 * n, *t3 = w + 9 * n;
    double bnorm = sqrt(vnorm2(n, b));
    int it = 0, mv = 0, st = OR_ERR_NOT_CONVERGED;
    double rel = bnorm > 0 ? 1.0 : 0.0;
    memset(x, 0, sizeof(cplx) * n);
    memcpy(res, b, sizeof(cplx) * n);                 /* residual of the current x */
    if (bnorm == 0) st = OR_OK;
    while (st == OR_ERR_NOT_CONVERGED && it < maxit) {
        /* bhat from the current residual (x = 0 at the start) */
        hop_to_parity(L, tap, Ur, 0, res, t1, t2);    /* t1 = H_eo res_o */
        for (int64_t i = 0; i < n; ++i) bh[i] = site_parity(L, i / 12) == 0 ? res[i] + t1[i] / a : 0;
        mv += 1;
        memset(xe, 0, sizeof(cplx) * n);
        memcpy(r, bh, sizeof(cplx) * n);
        schur_apply(L, tap, Ur, m, 1, r, s, t1, t2, t3);
        mv += 1;
        memcpy(p, s, sizeof(cplx) * n);
        double gamma = vnorm2(n, s);
        while (it < maxit && gamma > 0) {
            schur_apply(L, tap, Ur, m, 0, p, q, t1, t2, t3);
            mv += 1;
            double qq = vnorm2(n, q);
            if (!(qq > 0)) break;
            double alpha = gamma / qq;
            vaxpy(n, alpha, p, xe);
            vaxpy(n, -alpha, q, r);
            ++it;
            if (sqrt(vnorm2(n, r)) <= tol * bnorm) break;
            schur_apply(L, tap, Ur, m, 1, r, s, t1, t2, t3);
            mv += 1;
            double gnew = vnorm2(n, s);
            double beta = gnew / gamma;
            gamma = gnew;
            for (int64_t i = 0; i < n; ++i) p[i] = s[i] + beta * p[i];
        }
        /* x_o = (res_o + H_oe x_e) / (4 + m); x += (x_e, x_o) */
        hop_to_parity(L, tap, Ur, 1, xe, t1, t2);
        mv += 1;
        for (int64_t i = 0; i < n; ++i)
            x[i] += site_parity(L, i / 12) == 0 ? xe[i] : (res[i] + t1[i]) / a;
        or_dslash(L, tap, Ur, m, (const double*)x, (double*)t1);
        mv += 1;
        for (int64_t i = 0; i < n; ++i) res[i] = b[i] - t1[i];
        rel = sqrt(vnorm2(n, res)) / bnorm;
        if (!isfinite(rel)) { st = OR_ERR_NUMERIC; break; }
        if (rel <= tol) st = OR_OK;
    }
    free(w);
    if (iters_out) *iters_out = it;
    if (matvecs_out) *matvecs_out = mv;
    if (rel_out) *rel_out = rel;
    return st;
}

/* ------------------------------------------------------------------ */
/* The next level down.  Sec. III: the coarsening is recursed with the   */
/* chiral components kept separate, so every level is a nearest-        */
/* neighbour operator with 2Nv x 2Nv links.  Sec. IV: a 3-level cycle,  */
/* GMRES post-relaxation on each level, and a W-cycle -- for every      */
/* correction to the fine grid two V-cycles update the intermediate     */
/* grid -- with CG on the normal equations to 1e-3 on the coarsest.     */
/*                                                                     */
/* Level-1 vectors: [x1][2 nv1] complex, dof a of chirality a / nv1.    */
/* Level-2 prolongator P2: nv2 level-1 vectors [i][x1][2 nv1]; column   */
/* (X2, s, i) is vector i on the level-1 sites of aggregate X2 and the  */
/* dof of chirality s.  Level-2 operator A2[X2][d][a][b] like D_c.      */
/* ------------------------------------------------------------------ */

/* Block orthonormalisation of level-1 vectors (eq. 4 one level down): per
 * aggregate X2 and chirality s, MGS twice in index order over the entries
 * (x1 in X2, j < nv1) of dof s*nv1 + j; positive real R diagonal. */
OR_API int or_cblock_orthonormalize(const int* Lc1, const int* B2, int nv1, int nv2, const double* vr, double* Pr) {
    blocking_t bk;
    if (blocking_init(&bk, Lc1, B2, nv2) != OR_OK || nv1 <= 0 || nv2 <= 0) return OR_ERR_ARG;
    const int nc1 = 2 * nv1;
    const cplx* v = (const cplx*)vr;
    cplx* P = (cplx*)Pr;
    int64_t Vb = bk.V / bk.Vc, len = Vb * nv1;
    int64_t* sites = block_sites(&bk);
    int status = OR_OK;
    cplx* W = (cplx*)malloc(sizeof(cplx) * len * nv2);
    double* orig = (double*)malloc(sizeof(double) * nv2);
    for (int64_t X = 0; X < bk.Vc; ++X)
        for (int s = 0; s < 2; ++s) {
            for (int i = 0; i < nv2; ++i)
                for (int64_t k = 0; k < Vb; ++k)
                    for (int j = 0; j < nv1; ++j)
                        W[i * len + k * nv1 + j] = v[((int64_t)i * bk.V + sites[X * Vb + k]) * nc1 + s * nv1 + j];
            for (int i = 0; i < nv2; ++i) {
                cplx* wi = W + i * len;
                orig[i] = sqrt(vnorm2(len, wi));
                for (int pass = 0; pass < 2; ++pass)
                    for (int j = 0; j < i; ++j) {
                        cplx c = vdot(len, W + j * len, wi);
                        vaxpy(len, -c, W + j * len, wi);
                    }
                double nn = sqrt(vnorm2(len, wi));
                if (!(nn > 1e-12 * orig[i])) { status = OR_ERR_NUMERIC; nn = 1.0; }
                for (int64_t k = 0; k < len; ++k) wi[k] /= nn;
            }
            for (int i = 0; i < nv2; ++i)
                for (int64_t k = 0; k < Vb; ++k)
                    for (int j = 0; j < nv1; ++j)
                        P[((int64_t)i * bk.V + sites[X * Vb + k]) * nc1 + s * nv1 + j] = W[i * len + k * nv1 + j];
        }
    free(W); free(orig); free(sites);
    return status;
}

/* r2 = P2^dag r1: r2[X2][s nv2 + i] = sum over x1 in X2, j < nv1 of conj(P2_i(x1, s nv1 + j)) r1(x1, s nv1 + j) */
OR_API int or_crestrict(const int* Lc1, const int* B2, int nv1, int nv2, const double* Pr, const double* rr,
                        double* r2r) {
    blocking_t bk;
    if (blocking_init(&bk, Lc1, B2, nv2) != OR_OK) return OR_ERR_ARG;
    const int nc1 = 2 * nv1, nc2 = 2 * nv2;
    const cplx* P = (const cplx*)Pr;
    const cplx* r = (const cplx*)rr;
    cplx* r2 = (cplx*)r2r;
    int64_t Vb = bk.V / bk.Vc;
    int64_t* sites = block_sites(&bk);
    for (int64_t X = 0; X < bk.Vc; ++X)
        for (int s = 0; s < 2; ++s)
            for (int i = 0; i < nv2; ++i) {
                cplx acc = 0;
                for (int64_t k = 0; k < Vb; ++k) {
                    int64_t x = sites[X * Vb + k];
                    for (int j = 0; j < nv1; ++j)
                        acc += conj(P[((int64_t)i * bk.V + x) * nc1 + s * nv1 + j]) * r[x * nc1 + s * nv1 + j];
                }
                r2[X * nc2 + s * nv2 + i] = acc;
            }
    free(sites);
    return OR_OK;
}

/* e1 = P2 y2: e1(x1, s nv1 + j) = sum_i P2_i(x1, s nv1 + j) y2[X2(x1)][s nv2 + i] */
OR_API int or_cprolong(const int* Lc1, const int* B2, int nv1, int nv2, const double* Pr, const double* yr,
                       double* er) {
    blocking_t bk;
    if (blocking_init(&bk, Lc1, B2, nv2) != OR_OK) return OR_ERR_ARG;
    const int nc1 = 2 * nv1, nc2 = 2 * nv2;
    const cplx* P = (const cplx*)Pr;
    const cplx* y = (const cplx*)yr;
    cplx* e = (cplx*)er;
    for (int64_t x = 0; x < bk.V; ++x) {
        int64_t X = block_of(&bk, x);
        for (int a = 0; a < nc1; ++a) {
            int s = a / nv1;
            cplx acc = 0;
            for (int i = 0; i < nv2; ++i) acc += P[((int64_t)i * bk.V + x) * nc1 + a] * y[X * nc2 + s * nv2 + i];
            e[x * nc1 + a] = acc;
        }
    }
    return OR_OK;
}

/*
 * Galerkin operator one level down, A2 = P2^dag A1 P2 in nearest-neighbour
 * form: A2[X2][d][a][b] = sum over x1 in X2 and stencil terms t of A1 of
 * conj(P2_a(x1)) A1[x1][t] P2_b(x1 + t), where term t lands in slot d = 0
 * when t = 0 or the term stays inside X2, and in slot d = t when it leaves X2
 * through the face of direction t (exact for any level-2 extent, as the
 * fine-to-level-1 build).
 */
OR_API int or_ccoarse_build(const int* Lc1, const int* B2, int nv1, int nv2, const double* A1r, const double* Pr,
                            double* A2r) {
    blocking_t bk;
    if (blocking_init(&bk, Lc1, B2, nv2) != OR_OK) return OR_ERR_ARG;
    const int nc1 = 2 * nv1, nc2 = 2 * nv2;
    const cplx* A1 = (const cplx*)A1r;
    const cplx* P = (const cplx*)Pr;
    cplx* A2 = (cplx*)A2r;
    int64_t Vb = bk.V / bk.Vc;
    int64_t* sites = block_sites(&bk);
    memset(A2, 0, sizeof(cplx) * bk.Vc * 9 * nc2 * nc2);
    cplx* HP = (cplx*)malloc(sizeof(cplx) * nc1 * nc2);
    for (int64_t X = 0; X < bk.Vc; ++X)
        for (int64_t k = 0; k < Vb; ++k) {
            int64_t x = sites[X * Vb + k];
            int cx[4];
            coords(Lc1, x, cx);
            for (int t = 0; t < 9; ++t) {
                int64_t y = coarse_neighbour(Lc1, x, t);
                int d = 0;
                if (t > 0) {
                    int mu = (t - 1) / 2, dir = (t % 2 == 1) ? 1 : -1;
                    int leaves = (dir > 0) ? (cx[mu] % B2[mu] == B2[mu] - 1) : (cx[mu] % B2[mu] == 0);
                    d = leaves ? t : 0;
                }
                const cplx* At = A1 + (x * 9 + t) * nc1 * nc1;
                /* HP[q][b] = (A1[x][t] P2_b(y))_q, b = (sb, ib) */
                for (int q = 0; q < nc1; ++q)
                    for (int b = 0; b < nc2; ++b) {
                        int sb = b / nv2, ib = b % nv2;
                        cplx acc = 0;
                        for (int j = 0; j < nv1; ++j)
                            acc += At[q * nc1 + sb * nv1 + j] * P[((int64_t)ib * bk.V + y) * nc1 + sb * nv1 + j];
                        HP[q * nc2 + b] = acc;
                    }
                cplx* Ad = A2 + (X * 9 + d) * nc2 * nc2;
                for (int a = 0; a < nc2; ++a) {
                    int sa = a / nv2, ia = a % nv2;
                    for (int b = 0; b < nc2; ++b) {
                        cplx acc = 0;
                        for (int j = 0; j < nv1; ++j)
                            acc += conj(P[((int64_t)ia * bk.V + x) * nc1 + sa * nv1 + j]) * HP[(sa * nv1 + j) * nc2 + b];
                        Ad[a * nc2 + b] += acc;
                    }
                }
            }
        }
    free(HP); free(sites);
    return OR_OK;
}

/* ---- level-1 relaxation: the smoothers of Sec. III on the operator A1 ---- */
typedef struct {
    const int* Lc;
    int nc;
    const cplx* A;
} cop_t;

static void cop_apply(const cop_t* c, const cplx* in, cplx* out) {
    or_coarse_apply(c->Lc, c->nc, (const double*)c->A, (const double*)in, (double*)out);
}

/* MR steps with under-relaxation on (e, r), operator A1 (as mr_internal) */
static void cmr(const cop_t* c, int nsteps, double omega, cplx* e, cplx* r) {
    int64_t n = vol(c->Lc) * c->nc;
    cplx* q = (cplx*)malloc(sizeof(cplx) * n);
    for (int k = 0; k < nsteps; ++k) {
        cop_apply(c, r, q);
        cplx qr = vdot(n, q, r);
        double qq = vnorm2(n, q);
        if (!(qq > 0)) break;
        cplx alpha = omega * qr / qq;
        vaxpy(n, alpha, r, e);
        vaxpy(n, -alpha, q, r);
    }
    free(q);
}

/* one GMRES(k) application with under-relaxation, operator A1 (as gmres_smooth):
 * e += omega argmin over K_k(A1, r) of |r - A1 d| */
static void cgmres(const cop_t* c, int k, double omega, cplx* e, const cplx* r) {
    int64_t n = vol(c->Lc) * c->nc;
    double beta = sqrt(vnorm2(n, r));
    if (!(beta > 0) || k <= 0) return;
    cplx* V = (cplx*)malloc(sizeof(cplx) * n * (k + 1));
    cplx* H = (cplx*)calloc((size_t)(k + 1) * k, sizeof(cplx));
    for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
    int dim = k;
    for (int j = 0; j < k; ++j) {
        cplx* w = V + (int64_t)(j + 1) * n;
        cop_apply(c, V + (int64_t)j * n, w);
        for (int i = 0; i <= j; ++i) H[i * k + j] = vdot(n, V + (int64_t)i * n, w);
        for (int i = 0; i <= j; ++i) vaxpy(n, -H[i * k + j], V + (int64_t)i * n, w);
        double hn = sqrt(vnorm2(n, w));
        H[(j + 1) * k + j] = hn;
        if (!(hn > 0)) { dim = j + 1; break; }
        for (int64_t i = 0; i < n; ++i) w[i] /= hn;
    }
    /* least squares min |beta e_1 - Hbar y| by Givens rotations */
    cplx* g = (cplx*)calloc(dim + 1, sizeof(cplx));
    g[0] = beta;
    cplx* R = (cplx*)malloc(sizeof(cplx) * (dim + 1) * dim);
    for (int i = 0; i <= dim; ++i)
        for (int j = 0; j < dim; ++j) R[i * dim + j] = H[i * k + j];
    for (int j = 0; j < dim; ++j) {
        cplx a = R[j * dim + j], b = R[(j + 1) * dim + j];
        double den = sqrt(creal(a * conj(a)) + creal(b * conj(b)));
        if (!(den > 0)) continue;
        cplx cs = a / den, sn = b / den;   /* [conj(cs) conj(sn); -sn cs] zeroes b */
        for (int jj = j; jj < dim; ++jj) {
            cplx u = R[j * dim + jj], v = R[(j + 1) * dim + jj];
            R[j * dim + jj] = conj(cs) * u + conj(sn) * v;
            R[(j + 1) * dim + jj] = -sn * u + cs * v;
        }
        cplx u = g[j], v = g[j + 1];
        g[j] = conj(cs) * u + conj(sn) * v;
        g[j + 1] = -sn * u + cs * v;
    }
    cplx* y = (cplx*)calloc(dim, sizeof(cplx));
    for (int i = dim - 1; i >= 0; --i) {
        cplx acc = g[i];
        for (int j = i + 1; j < dim; ++j) acc -= R[i * dim + j] * y[j];
        y[i] = acc / R[i * dim + i];
    }
    for (int j = 0; j < dim; ++j) vaxpy(n, omega * y[j], V + (int64_t)j * n, e);
    free(V); free(H); free(g); free(R); free(y);
}

/* level-1 post-smoothing on (e, r = r_in - A1 e) by the configured smoother */
static void csmooth(const or_params* p, const cop_t* c, cplx* e, cplx* r) {
    if (p->smoother1 == 1) cgmres(c, p->steps1, p->omega, e, r);
    else cmr(c, p->steps1, p->omega, e, r);
}

/* M1: one V(0, steps1) cycle on level 1 (the two-grid cycle of level 1 and
 * level 2): r2 = P2^dag r; y2 = CGNR(A2, r2) to coarse_tol; z = P2 y2; then
 * post-smoothing on A1 from z with the residual r - A1 z. */
static void vcycle_l1(const mg_t* g, const cplx* r, cplx* z) {
    const or_params* p = g->p;
    int Lc2[4];
    for (int m = 0; m < 4; ++m) Lc2[m] = g->bk.Lc[m] / p->B2[m];
    const int nc1 = g->bk.nc, nc2 = 2 * p->nv2;
    int64_t n1 = g->bk.Vc * nc1, n2 = vol(Lc2) * nc2;
    cplx* r2 = (cplx*)malloc(sizeof(cplx) * n2);
    cplx* y2 = (cplx*)malloc(sizeof(cplx) * n2);
    cplx* rr = (cplx*)malloc(sizeof(cplx) * n1);
    or_crestrict(g->bk.Lc, p->B2, p->nv, p->nv2, (const double*)g->P2, (const double*)r, (double*)r2);
    int it = or_cgnr(Lc2, nc2, (const double*)g->A2, (const double*)r2, (double*)y2, p->coarse_tol, p->coarse_maxit,
                     NULL);
    if (g->info) g->info->coarse_iters += it;
    or_cprolong(g->bk.Lc, p->B2, p->nv, p->nv2, (const double*)g->P2, (const double*)y2, (double*)z);
    cop_t c = {g->bk.Lc, nc1, g->A};
    cop_apply(&c, z, rr);
    for (int64_t i = 0; i < n1; ++i) rr[i] = r[i] - rr[i];
    csmooth(p, &c, z, rr);
    free(r2); free(y2); free(rr);
}

/* The coarse-grid correction of the three-level method: cycles1 V-cycles on
 * A1 e = r1 from e = 0 (Sec. IV: two, the W-cycle), e += M1 (r1 - A1 e). */
static void kcycle_l1(const mg_t* g, const cplx* r1, cplx* e1) {
    const int nc1 = g->bk.nc;
    int64_t n1 = g->bk.Vc * nc1;
    cplx* res = (cplx*)malloc(sizeof(cplx) * n1);
    cplx* z = (cplx*)malloc(sizeof(cplx) * n1);
    cop_t c = {g->bk.Lc, nc1, g->A};
    memset(e1, 0, sizeof(cplx) * n1);
    for (int k = 0; k < g->p->cycles1; ++k) {
        cop_apply(&c, e1, res);
        for (int64_t i = 0; i < n1; ++i) res[i] = r1[i] - res[i];
        vcycle_l1(g, res, z);
        for (int64_t i = 0; i < n1; ++i) e1[i] += z[i];
    }
    free(res); free(z);
}

/* level-1 smoothing as a routine of its own (tests): e, r updated in place */
OR_API void or_csmooth(const or_params* p, const int* Lc1, const double* A1, double* er, double* rr) {
    cop_t c = {Lc1, 2 * p->nv, (const cplx*)A1};
    csmooth(p, &c, (cplx*)er, (cplx*)rr);
}

/* the coarse-grid correction of the three-level method as a routine (tests):
 * e1 = K1 r1 with p->cycles1 level-1 V-cycles */
OR_API void or_kcycle_l1(const or_params* p, const double* A1, const double* P2, const double* A2, const double* r1,
                         double* e1, or_info* info) {
    mg_t g;
    blocking_init(&g.bk, p->L, p->B, p->nv);
    g.p = p; g.U = NULL; g.P = NULL; g.A = (const cplx*)A1; g.P2 = (const cplx*)P2; g.A2 = (const cplx*)A2;
    g.info = info;
    kcycle_l1(&g, (const cplx*)r1, (cplx*)e1);
}

/*
 * Adaptive setup of level 2 (Sec. II's loop in the two-step form of Sec. IV,
 * applied to A1 as the operator to coarsen): init_relax MR steps on A1 v = 0
 * from each random start, normalise; then groups of group_size prototypes
 * refined one group at a time with the truncated two-level method of levels
 * 1 and 2 built from the other prototypes (n_iter iterations of
 * v <- v + M1_t (-A1 v), normalised); finally P2 and A2 = P2^dag A1 P2.
 * V2 (nv2 level-1 vectors) is overwritten with the prototypes.
 */
OR_API int or_setup_level2(const or_params* p, const double* A1r, double* V2r, int init_relax, int n_iter,
                           int group_size, double* P2r, double* A2r, or_info* info) {
    or_info local;
    memset(&local, 0, sizeof(local));
    blocking_t bk;
    if (blocking_init(&bk, p->L, p->B, p->nv) != OR_OK) return OR_ERR_ARG;
    const int nv2 = p->nv2, nc1 = bk.nc;
    if (group_size <= 0 || nv2 % group_size != 0) return OR_ERR_ARG;
    int Lc2[4];
    for (int m = 0; m < 4; ++m) {
        if (p->B2[m] <= 0 || bk.Lc[m] % p->B2[m]) return OR_ERR_ARG;
        Lc2[m] = bk.Lc[m] / p->B2[m];
    }
    int64_t n1 = bk.Vc * nc1;
    cplx* V = (cplx*)V2r;
    cplx* r = (cplx*)malloc(sizeof(cplx) * n1);
    cplx* z = (cplx*)malloc(sizeof(cplx) * n1);
    cop_t c = {bk.Lc, nc1, (const cplx*)A1r};
    for (int i = 0; i < nv2; ++i) {
        cplx* v = V + (int64_t)i * n1;
        cop_apply(&c, v, r);
        for (int64_t k = 0; k < n1; ++k) r[k] = -r[k];
        cmr(&c, init_relax, p->omega, v, r);
        double nrm = sqrt(vnorm2(n1, v));
        for (int64_t k = 0; k < n1; ++k) v[k] /= nrm;
    }
    int st = OR_OK;
    int nt = nv2 - group_size;
    if (n_iter > 0 && nt > 0) {
        or_params pt = *p;
        pt.nv2 = nt;
        pt.levels = 3;
        cplx* Vt = (cplx*)malloc(sizeof(cplx) * n1 * nt);
        cplx* Pt = (cplx*)malloc(sizeof(cplx) * n1 * nt);
        cplx* At = (cplx*)malloc(sizeof(cplx) * vol(Lc2) * 9 * (2 * nt) * (2 * nt));
        for (int g0 = 0; g0 < nv2 && st == OR_OK; g0 += group_size) {
            int k = 0;
            for (int i = 0; i < nv2; ++i)
                if (i < g0 || i >= g0 + group_size) memcpy(Vt + (int64_t)(k++) * n1, V + (int64_t)i * n1, sizeof(cplx) * n1);
            st = or_cblock_orthonormalize(bk.Lc, p->B2, p->nv, nt, (const double*)Vt, (double*)Pt);
            if (st != OR_OK) break;
            or_ccoarse_build(bk.Lc, p->B2, p->nv, nt, A1r, (const double*)Pt, (double*)At);
            mg_t g;
            g.bk = bk; g.p = &pt; g.U = NULL; g.P = NULL; g.A = (const cplx*)A1r; g.P2 = Pt; g.A2 = At;
            g.info = &local;
            for (int i = g0; i < g0 + group_size; ++i) {
                cplx* v = V + (int64_t)i * n1;
                for (int it = 0; it < n_iter; ++it) {
                    cop_apply(&c, v, r);
                    for (int64_t q = 0; q < n1; ++q) r[q] = -r[q];
                    vcycle_l1(&g, r, z);
                    for (int64_t q = 0; q < n1; ++q) v[q] += z[q];
                    double nrm = sqrt(vnorm2(n1, v));
                    for (int64_t q = 0; q < n1; ++q) v[q] /= nrm;
                }
            }
        }
        free(Vt); free(Pt); free(At);
    }
    if (st == OR_OK) st = or_cblock_orthonormalize(bk.Lc, p->B2, p->nv, nv2, V2r, P2r);
    if (st == OR_OK) or_ccoarse_build(bk.Lc, p->B2, p->nv, nv2, A1r, P2r, A2r);
    free(r); free(z);
    local.status = st;
    if (info) *info = local;
    return st;
}
